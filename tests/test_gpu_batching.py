"""Batched method: tuning never changes results; CUDA-graph plans replay the launch exactly;
the autotuner and its JSON cache (through the C ABI)."""
import json

import numpy as np
import pytest

from paper_1309_7963_gb300 import inputs, pnuc

pytestmark = pytest.mark.gpu


def device_inputs(ctx, w):
    import torch
    tids = np.array([ctx.create_target(*za) for za in w.targets], np.int32)
    return (torch.tensor(w.energies, dtype=torch.float64, device="cuda"),
            torch.tensor(tids[w.tidx], dtype=torch.int32, device="cuda"))


def results(r):
    return r.residuals_np().copy(), pnuc.sort_secondaries(r.secondaries_np())


def same(a, b):
    return np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_tuning_variants_give_identical_results(ctx):
    import torch
    w = inputs.mixed(30_000, seed=21)
    e, t = device_inputs(ctx, w)
    saved = ctx.get_tuning("fp32")
    try:
        ref = results(ctx.simulate(e, t, seed=21, precision="fp32", method="plain"))
        for tun in [dict(block_size=256, kin_batch=1, refill_threshold=1, chunk=64),
                    dict(block_size=128, kin_batch=32, refill_threshold=16, chunk=1024),
                    dict(block_size=64, kin_batch=8, refill_threshold=4, chunk=256)]:
            ctx.set_tuning("fp32", **tun)
            got = results(ctx.simulate(e, t, seed=21, precision="fp32", method="persistent"))
            torch.cuda.synchronize()
            assert same(got, ref), tun
    finally:
        ctx.set_tuning("fp32", **saved)


def test_invalid_tuning_rejected(ctx):
    for bad in [dict(block_size=96), dict(kin_batch=0), dict(kin_batch=33), dict(chunk=8),
                dict(refill_threshold=40), dict(blocks_per_sm=0)]:
        with pytest.raises(pnuc.PnucError):
            ctx.set_tuning("fp32", **bad)


def test_a_refused_launch_leaves_the_next_one_clean(ctx):
    """A launch refused for its tuning (the sorted method's FP64 slots at 512 threads do not fit
    an SM's shared memory) fails with PNUC_ERR_ARG and leaves no CUDA error behind: the next
    launch of the same context, with a tuning that fits, succeeds and matches a fresh run."""
    import torch
    w = inputs.oxygen_calcium(n_each=2_000)
    e, t = device_inputs(ctx, w)
    saved = ctx.get_tuning("fp64")
    ref = results(ctx.simulate(e, t, seed=5, precision="fp64", method="persistent"))
    try:
        ctx.set_tuning("fp64", block_size=512)
        with pytest.raises(pnuc.PnucError) as err:
            ctx.simulate(e, t, seed=5, precision="fp64", method="sorted")
        assert err.value.status == 1  # PNUC_ERR_ARG
    finally:
        ctx.set_tuning("fp64", **saved)
    got = results(ctx.simulate(e, t, seed=5, precision="fp64", method="persistent"))
    torch.cuda.synchronize()
    assert same(got, ref)


def test_graph_plan_replays_and_updates(ctx):
    import torch
    w = inputs.mixed(20_000, seed=4)
    e, t = device_inputs(ctx, w)
    out = ctx.alloc(w.n)
    g = ctx.graph(e, t, seed=4, out=out)
    for _ in range(2):
        g.launch()
        torch.cuda.synchronize()
        got = results(out)
        ref = results(ctx.simulate(e, t, seed=4, precision="fp32", method="persistent"))
        assert same(got, ref)
    # new seed and new buffers through an update
    w2 = inputs.mixed(7_000, seed=5)
    e2, t2 = device_inputs(ctx, w2)
    out2 = ctx.alloc(w2.n)
    g.update(e2, t2, seed=5, out=out2, first_event_id=1000)
    g.launch()
    torch.cuda.synchronize()
    ref2 = results(ctx.simulate(e2, t2, seed=5, first_event_id=1000, precision="fp32", method="persistent"))
    assert same(results(out2), ref2)
    g.close()


def test_autotune_and_cache_roundtrip(ctx, tmp_path):
    import torch
    w = inputs.oxygen_calcium(n_each=40_000)
    e, t = device_inputs(ctx, w)
    saved = ctx.get_tuning("fp32")
    try:
        best, ms = ctx.autotune(e, t, seed=0, precision="fp32", reps=1)
        assert ms > 0 and best == {**ctx.get_tuning("fp32")}
        ref = results(ctx.simulate(e, t, seed=0, precision="fp32", method="plain"))
        got = results(ctx.simulate(e, t, seed=0, precision="fp32", method="persistent"))
        torch.cuda.synchronize()
        assert same(got, ref)
        path = tmp_path / "tuning.json"
        path.write_text(json.dumps({"Some Other GPU": {"fp32": {"block_size": 64}}}))
        ctx.save_tuning(str(path))
        data = json.loads(path.read_text())
        assert "Some Other GPU" in data and len(data) == 2
        ctx.set_tuning("fp32", kin_batch=3)
        ctx.load_tuning(str(path))
        assert ctx.get_tuning("fp32") == best
        # a cache without this device's entry is refused and leaves the tuning alone
        other = tmp_path / "other.json"
        other.write_text(json.dumps({"Some Other GPU": {"fp32": {"block_size": 64}}}))
        with pytest.raises(pnuc.PnucError):
            ctx.load_tuning(str(other))
        assert ctx.get_tuning("fp32") == best
    finally:
        ctx.set_tuning("fp32", **saved)


def test_kernel_timing_records_each_launch(ctx):
    import torch
    w = inputs.oxygen_calcium(n_each=20_000)
    e, t = device_inputs(ctx, w)
    out = ctx.alloc(w.n)
    ctx.kernel_timing(True)
    for _ in range(3):
        ctx.simulate(e, t, seed=1, precision="fp32", method="persistent", out=out)
    kt = ctx.kernel_times()
    assert kt["launches"] == 3 and kt["cascade_ms"] > 0 and kt["evaporation_ms"] > 0
    # a graph launch is not recorded; the plain method records one kernel
    g = ctx.graph(e, t, seed=1, out=out)
    g.launch()
    torch.cuda.synchronize()
    g.close()
    assert ctx.kernel_times()["launches"] == 3
    ctx.kernel_timing(True)
    ctx.simulate(e, t, seed=1, precision="fp32", method="plain", out=out)
    ctx.kernel_timing(False)
    ctx.simulate(e, t, seed=1, precision="fp32", method="plain", out=out)
    kt = ctx.kernel_times()
    assert kt["launches"] == 1 and kt["cascade_ms"] > 0 and kt["evaporation_ms"] == 0.0


def test_small_batches_leave_idle_lanes_quiet(ctx):
    """A batch much smaller than the resident grid leaves most lanes without an event; those
    lanes must not touch their (unset) draw streams, and every launch ends promptly."""
    import time

    import torch
    w = inputs.oxygen_calcium(n_each=3)
    e, t = device_inputs(ctx, w)
    out = ctx.alloc(w.n)
    ref = results(ctx.simulate(e, t, seed=9, precision="fp32", method="plain"))
    t0 = time.perf_counter()
    for _ in range(50):
        ctx.simulate(e, t, seed=9, precision="fp32", method="persistent", out=out)
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < 5.0
    assert same(results(out), ref)


def test_sorted_method_tiny_and_ragged_batches(ctx):
    """The sorted method on batches smaller than a block, of one event, and ragged against the
    block size, with per-event parity to the plain kernel; it is refused by the entry point
    that allocates nothing."""
    import torch
    for n in (1, 3, 127, 129, 5000):
        w = inputs.mixed(n, seed=n)
        e, t = device_inputs(ctx, w)
        a = results(ctx.simulate(e, t, seed=n, precision="fp64", method="plain"))
        b = results(ctx.simulate(e, t, seed=n, precision="fp64", method="sorted"))
        torch.cuda.synchronize()
        assert same(a, b), n
    import ctypes as C
    e, t = np.full(4, 100.0), np.zeros(4, np.int32)
    sec, res, cnt = np.empty(64, pnuc.SECONDARY_DTYPE), np.empty(4, pnuc.RESIDUAL_DTYPE), C.c_uint64()
    st = ctx.lib.pnuc_simulate_host_noalloc(ctx.handle, pnuc.PRECISION["fp32"], pnuc.METHOD["sorted"], e.ctypes.data,
                                            t.ctypes.data, 4, 1, 0, sec.ctypes.data, 64, C.byref(cnt),
                                            res.ctypes.data, None)
    assert st == 1
