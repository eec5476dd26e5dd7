"""Serving loop (pnuc_server): continuous batching with memory-based admission. Every
request's results equal those of the same events run alone; overflowing requests are re-run;
admission respects the arena; queue limits, errors and timeouts are reported."""
import numpy as np
import pytest

from paper_1309_7963_gb300 import driver, inputs, pnuc

pytestmark = pytest.mark.gpu


def serving_tids(ctx):
    return np.array([ctx.create_target(*za) for za in inputs.SERVING_TARGETS], np.int32)


def alone(ctx, req, tids, seed, precision="fp32"):
    sec, res = ctx.simulate_host(req["energies"], tids[req["tidx"]], seed=seed, first_event_id=req["first_event_id"],
                                 precision=precision, method="persistent")
    return pnuc.sort_secondaries(sec), res


def test_each_result_equals_its_events_run_alone(ctx):
    tids = serving_tids(ctx)
    reqs = inputs.serving_requests(24, rate_hz=1e6, seed=7, min_batch=500, max_batch=20_000)
    srv = pnuc.Server(ctx, precision="fp32", streams=4, arena_bytes=256 << 20)
    try:
        tickets = [srv.submit(r["energies"], tids[r["tidx"]], 11, r["first_event_id"]) for r in reqs]
        for tk, r in zip(tickets, reqs):
            n = srv.wait(tk)
            sec, res = srv.fetch(tk, n)
            ref_sec, ref_res = alone(ctx, r, tids, 11)
            assert np.array_equal(res, ref_res)
            assert np.array_equal(pnuc.sort_secondaries(sec), ref_sec)
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["failed"] == 0
        assert st["latency_p99_ms"] >= st["latency_p50_ms"] > 0
    finally:
        srv.close()


def test_overflowing_requests_are_rerun_identically(ctx):
    tids = serving_tids(ctx)
    reqs = inputs.serving_requests(6, rate_hz=1e6, seed=8, min_batch=1000, max_batch=5000)
    srv = pnuc.Server(ctx, precision="fp64", streams=2, arena_bytes=64 << 20, sec_per_event=1)
    try:
        tickets = [srv.submit(r["energies"], tids[r["tidx"]], 3, r["first_event_id"]) for r in reqs]
        for tk, r in zip(tickets, reqs):
            sec, res = srv.fetch(tk, srv.wait(tk))
            ref_sec, ref_res = alone(ctx, r, tids, 3, precision="fp64")
            assert np.array_equal(res, ref_res) and np.array_equal(pnuc.sort_secondaries(sec), ref_sec)
        assert srv.stats()["reruns"] >= len(reqs)
    finally:
        srv.close()


def test_admission_respects_the_arena(ctx):
    tids = serving_tids(ctx)
    arena = 8 << 20
    srv = pnuc.Server(ctx, precision="fp32", streams=8, arena_bytes=arena, sec_per_event=12)
    try:
        reqs = inputs.serving_requests(10, rate_hz=1e6, seed=9, min_batch=9000, max_batch=9000)
        tickets = [srv.submit(r["energies"], tids[r["tidx"]], 5, r["first_event_id"]) for r in reqs]
        for tk in tickets:
            srv.fetch(tk, srv.wait(tk))
        st = srv.stats()
        # one 9000-event request reserves ~4.1 MB (inputs, residuals, 12 secondaries per event):
        # two fit the 8 MiB arena at once, never three
        one = 256 + 9000 * (8 + 4 + 64) + 9000 * 12 * 32
        assert st["completed"] == 10 and one <= st["arena_peak_bytes"] <= arena
        assert st["arena_peak_bytes"] < 3 * one
    finally:
        srv.close()


def test_submit_errors_queue_limit_and_timeout(ctx):
    tids = serving_tids(ctx)
    srv = pnuc.Server(ctx, precision="fp32", streams=1, arena_bytes=256 << 20, max_pending=2)
    try:
        with pytest.raises(pnuc.PnucError):
            srv.submit(np.zeros(0), np.zeros(0, np.int32), 0)
        with pytest.raises(pnuc.PnucError):  # can never fit the 256 MiB arena
            srv.submit(np.full(1_500_000, 100.0), np.full(1_500_000, tids[0], np.int32), 0)
        big = srv.submit(np.full(150_000, 200.0), np.full(150_000, tids[2], np.int32), 0)
        assert srv.wait(big, 0) is None  # still running: the wait times out
        q1 = srv.submit(np.full(1000, 100.0), np.full(1000, tids[1], np.int32), 0, 1 << 32)
        q2 = srv.submit(np.full(1000, 100.0), np.full(1000, tids[1], np.int32), 0, 2 << 32)
        with pytest.raises(pnuc.PnucError) as e:
            srv.submit(np.full(1000, 100.0), np.full(1000, tids[1], np.int32), 0, 3 << 32)
        assert e.value.status == 3
        for tk in (big, q1, q2):
            srv.fetch(tk, srv.wait(tk))
    finally:
        srv.close()


def test_driver_reports_latency_and_throughput(ctx):
    tids = serving_tids(ctx)
    reqs = inputs.serving_requests(60, rate_hz=300.0, seed=10)
    srv = pnuc.Server(ctx, precision="fp32", streams=4, arena_bytes=1 << 30)
    seen = []
    try:
        rep = driver.run(srv, reqs, tids, seed=1, keep=lambda req, sec, res: seen.append(len(res)))
        assert rep["requests"] == 60 and sum(seen) == rep["events"] == sum(len(r["energies"]) for r in reqs)
        assert 0 < rep["p50_ms"] <= rep["p99_ms"]
        st = srv.stats()
        assert st["completed"] == 60 and st["latency_p50_ms"] > 0
    finally:
        srv.close()


def test_zero_copy_view_and_release(ctx):
    tids = serving_tids(ctx)
    reqs = inputs.serving_requests(5, rate_hz=1e6, seed=12, min_batch=2000, max_batch=8000)
    srv = pnuc.Server(ctx, precision="fp32", streams=2, arena_bytes=64 << 20)
    try:
        tickets = [srv.submit(r["energies"], tids[r["tidx"]], 13, r["first_event_id"]) for r in reqs]
        for tk, r in zip(tickets, reqs):
            srv.wait(tk)
            sec, res = srv.view(tk)
            ref_sec, ref_res = alone(ctx, r, tids, 13)
            assert np.array_equal(res, ref_res)
            assert np.array_equal(pnuc.sort_secondaries(sec.copy()), ref_sec)
            srv.release(tk)
            with pytest.raises(pnuc.PnucError):  # released: the ticket is gone
                srv.release(tk)
        big = srv.submit(np.full(100_000, 200.0), np.full(100_000, tids[2], np.int32), 13)
        with pytest.raises(pnuc.PnucError) as e:  # still running
            srv.view(big)
        assert e.value.status == 6
        srv.wait(big)
        srv.release(big)
        assert srv.stats()["completed"] == len(reqs) + 1
    finally:
        srv.close()


def test_small_requests_are_merged_and_split_back(ctx):
    """Many small same-seed requests share launches (fewer launches than requests); requests
    with other seeds in between are never merged with them; every request's residuals and
    secondaries (renumbered to its own events) equal its events run alone."""
    tids = serving_tids(ctx)
    reqs = inputs.serving_requests(96, rate_hz=1e6, seed=14, min_batch=50, max_batch=3000)
    seeds = [21 if k % 8 else 22 for k in range(len(reqs))]
    srv = pnuc.Server(ctx, precision="fp32", streams=2, arena_bytes=256 << 20, max_merge=16)
    try:
        tickets = [srv.submit(r["energies"], tids[r["tidx"]], s, r["first_event_id"]) for r, s in zip(reqs, seeds)]
        for tk, r, s in zip(tickets, reqs, seeds):
            sec, res = srv.fetch(tk, srv.wait(tk))
            ref_sec, ref_res = alone(ctx, r, tids, s)
            assert np.array_equal(res, ref_res)
            assert np.array_equal(pnuc.sort_secondaries(sec), ref_sec)
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["failed"] == 0 and st["reruns"] == 0
        # seed changes cut the queue into 12 runs of 7 same-seed requests and 12 single ones
        assert 24 <= st["launches"] < len(reqs)
    finally:
        srv.close()


def test_merging_can_be_switched_off(ctx):
    tids = serving_tids(ctx)
    reqs = inputs.serving_requests(12, rate_hz=1e6, seed=15, min_batch=200, max_batch=2000)
    srv = pnuc.Server(ctx, precision="fp32", streams=1, arena_bytes=64 << 20, max_merge=1)
    try:
        tickets = [srv.submit(r["energies"], tids[r["tidx"]], 4, r["first_event_id"]) for r in reqs]
        for tk, r in zip(tickets, reqs):
            sec, res = srv.fetch(tk, srv.wait(tk))
            ref_sec, ref_res = alone(ctx, r, tids, 4)
            assert np.array_equal(res, ref_res) and np.array_equal(pnuc.sort_secondaries(sec), ref_sec)
        assert srv.stats()["launches"] == len(reqs)
    finally:
        srv.close()


def test_overflow_inside_a_merged_launch(ctx):
    """One secondary reserved per event: merged requests overflow their ranges (and the
    launch its reservation); each is run again alone and still equals its events run alone."""
    tids = serving_tids(ctx)
    reqs = inputs.serving_requests(20, rate_hz=1e6, seed=16, min_batch=100, max_batch=1500)
    srv = pnuc.Server(ctx, precision="fp64", streams=1, arena_bytes=64 << 20, sec_per_event=1, max_merge=8)
    try:
        tickets = [srv.submit(r["energies"], tids[r["tidx"]], 6, r["first_event_id"]) for r in reqs]
        for tk, r in zip(tickets, reqs):
            sec, res = srv.fetch(tk, srv.wait(tk))
            ref_sec, ref_res = alone(ctx, r, tids, 6, precision="fp64")
            assert np.array_equal(res, ref_res) and np.array_equal(pnuc.sort_secondaries(sec), ref_sec)
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["reruns"] >= len(reqs)
    finally:
        srv.close()


def test_server_configuration_is_checked(ctx):
    for bad in (dict(max_merge=0), dict(max_merge=65), dict(merge_events=0), dict(merge_events=(1 << 22) + 1),
                dict(lane_events=0), dict(lane_events=1025), dict(streams=65), dict(sec_per_event=0)):
        with pytest.raises(pnuc.PnucError):
            pnuc.Server(ctx, precision="fp32", arena_bytes=64 << 20, **bad)
    srv = pnuc.Server(ctx, precision="fp32", arena_bytes=64 << 20, max_merge=64, merge_events=1 << 22, lane_events=1024)
    srv.close()


def test_wait_any_returns_each_finished_request_once(ctx):
    tids = serving_tids(ctx)
    reqs = inputs.serving_requests(10, rate_hz=1e6, seed=17, min_batch=500, max_batch=50_000)
    srv = pnuc.Server(ctx, precision="fp32", streams=3, arena_bytes=256 << 20, max_merge=1)
    try:
        tickets = [srv.submit(r["energies"], tids[r["tidx"]], 8, r["first_event_id"]) for r in reqs]
        by_ticket = dict(zip(tickets, reqs))
        # one request waited for and released directly: wait_any must skip it
        srv.wait(tickets[3])
        srv.release(tickets[3])
        seen = []
        while len(seen) < len(tickets) - 1:
            tk = srv.wait_any(10_000)
            assert tk is not None and tk not in seen and tk != tickets[3]
            seen.append(tk)
            sec, res = srv.view(tk)
            ref_sec, ref_res = alone(ctx, by_ticket[tk], tids, 8)
            assert np.array_equal(res, ref_res)
            assert np.array_equal(pnuc.sort_secondaries(sec.copy()), ref_sec)
            srv.release(tk)
        assert sorted(seen) == sorted(t for t in tickets if t != tickets[3])
        assert srv.wait_any(50) is None  # nothing left: the wait times out
    finally:
        srv.close()


def test_neutron_requests_merge_with_proton_requests(ctx):
    """Requests with incident neutrons (a transport code's secondary neutrons) merge with
    proton requests; each result equals its events run alone with the same species."""
    import torch
    tids = serving_tids(ctx)
    reqs = inputs.serving_requests(12, rate_hz=1e6, seed=18, min_batch=300, max_batch=3000)
    rng = np.random.default_rng(19)
    species = [None if k % 3 == 0 else rng.integers(0, 2, len(r["energies"])).astype(np.uint8)
               for k, r in enumerate(reqs)]
    srv = pnuc.Server(ctx, precision="fp32", streams=1, arena_bytes=128 << 20)
    try:
        tickets = [srv.submit(r["energies"], tids[r["tidx"]], 12, r["first_event_id"], projectiles=pj)
                   for r, pj in zip(reqs, species)]
        for tk, r, pj in zip(tickets, reqs, species):
            sec, res = srv.fetch(tk, srv.wait(tk))
            proj = None if pj is None else torch.tensor(pj, device="cuda")
            ref = ctx.simulate(torch.tensor(r["energies"], device="cuda"),
                               torch.tensor(tids[r["tidx"]], device="cuda"), seed=12,
                               first_event_id=r["first_event_id"], capacity=40 * len(r["energies"]), projectiles=proj)
            torch.cuda.synchronize()
            assert np.array_equal(res, ref.residuals_np())
            assert np.array_equal(pnuc.sort_secondaries(sec), pnuc.sort_secondaries(ref.secondaries_np()))
        assert srv.stats()["launches"] < len(reqs)
    finally:
        srv.close()


def test_inflight_cap_still_serves_every_request(ctx):
    tids = serving_tids(ctx)
    reqs = inputs.serving_requests(16, rate_hz=1e6, seed=20, min_batch=1000, max_batch=20_000)
    srv = pnuc.Server(ctx, precision="fp32", streams=8, arena_bytes=256 << 20, max_inflight_events=15_000)
    try:
        tickets = [srv.submit(r["energies"], tids[r["tidx"]], 13, r["first_event_id"]) for r in reqs]
        for tk, r in zip(tickets, reqs):
            sec, res = srv.fetch(tk, srv.wait(tk))
            ref_sec, ref_res = alone(ctx, r, tids, 13)
            assert np.array_equal(res, ref_res) and np.array_equal(pnuc.sort_secondaries(sec), ref_sec)
        assert srv.stats()["completed"] == len(reqs)
    finally:
        srv.close()


def test_trace_orders_each_requests_phases(ctx):
    """pnuc_server_trace: one entry per released request, whose times follow the request
    through the server (submit, admission, launch enqueued, GPU start and end, completion seen,
    release; the GPU times aligned to the host clock within a fraction of a millisecond), and
    whose phases add up to its latency."""
    tids = serving_tids(ctx)
    reqs = inputs.serving_requests(40, rate_hz=2000.0, seed=12, min_batch=1000, max_batch=30_000)
    srv = pnuc.Server(ctx, precision="fp32", streams=4, arena_bytes=512 << 20)
    try:
        srv.trace(True)
        driver.run(srv, reqs, tids, seed=5)
        srv.trace(False)
        tr = srv.trace_read()
    finally:
        srv.close()
    assert len(tr) == len(reqs) and np.all(tr["status"] == 0) and np.all(tr["launch"] > 0)
    slack = 0.5  # ms: alignment of the device clock to the host's
    assert np.all(tr["t_submit"] <= tr["t_admit"]) and np.all(tr["t_admit"] <= tr["t_launched"])
    assert np.all(tr["t_gpu_start"] <= tr["t_gpu_end"])
    assert np.all(tr["t_gpu_start"] >= tr["t_admit"] - slack)
    assert np.all(tr["t_gpu_end"] <= tr["t_complete"] + slack)
    assert np.all(tr["t_complete"] <= tr["t_release"])
    ph = driver.phase_times(tr)
    total = sum(ph[k] for k in driver.PHASES)
    assert np.allclose(total, tr["t_release"] - tr["t_submit"], atol=1e-6)
    where = driver.attribute(tr, slow_ms=0.0)
    assert where["slow"] == len(tr) and sum(where["dominant"].values()) == len(tr)
