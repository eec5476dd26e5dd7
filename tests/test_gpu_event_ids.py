"""Per-event ids (pnuc_batch.event_ids): event i of a batch with ids runs exactly the event
that a batch with contiguous ids runs at id ids[i], whatever their order and repeats; a run
of one repeated id gives the same records on every lane (the divergence-free bound of the
paper's same-seed experiment, §3); FP64 results at given ids match the oracle."""
import numpy as np
import pytest

from paper_1309_7963_gb300 import inputs, pnuc

from .parity import compare, gpu_subset, oracle_at

pytestmark = pytest.mark.gpu


def expected_secondaries(sec_ref, n_ref, pos):
    """The reference run's secondaries of events pos, renumbered to 0..len(pos)-1."""
    s = pnuc.sort_secondaries(sec_ref)
    b = np.searchsorted(s["event"], np.arange(n_ref + 1))
    idx = np.concatenate([np.arange(b[p], b[p + 1]) for p in pos])
    out = s[idx].copy()
    out["event"] = np.repeat(np.arange(len(pos)), (b[1:] - b[:-1])[pos])
    return out


@pytest.mark.parametrize("precision,method", [("fp32", "persistent"), ("fp64", "plain"), ("fp64", "sorted")])
def test_ids_in_any_order_and_repeated(ctx, precision, method):
    import torch
    w = inputs.mixed(4000, seed=2)
    n = w.n
    tids = np.array([ctx.create_target(*za) for za in w.targets], np.int32)
    e = torch.tensor(w.energies, device="cuda")
    t = torch.tensor(tids[w.tidx], device="cuda")
    ref = ctx.simulate(e, t, seed=w.seed, first_event_id=w.first_event_id, precision=precision, method=method,
                       capacity=40 * n)
    rng = np.random.default_rng(3)
    # repeats at random, a run of 700 lanes on one id, the last 300 ids in reverse order
    pos = np.concatenate([rng.integers(0, n, 3000), np.full(700, 17), np.arange(n - 300, n)[::-1]])
    p_dev = torch.tensor(pos, device="cuda")
    ids = torch.tensor(w.first_event_id + pos, dtype=torch.int64, device="cuda")
    r = ctx.simulate(e[p_dev], t[p_dev], seed=w.seed, first_event_id=987654321, precision=precision, method=method,
                     capacity=40 * len(pos), event_ids=ids)
    torch.cuda.synchronize()
    res_ref, res = ref.residuals_np(), r.residuals_np()
    assert np.array_equal(res, res_ref[pos])
    assert np.array_equal(pnuc.sort_secondaries(r.secondaries_np()),
                          expected_secondaries(ref.secondaries_np(), n, pos))


def test_ids_match_the_oracle_fp64(ctx):
    import torch
    w = inputs.mixed(2000, seed=4)
    tids = np.array([ctx.create_target(*za) for za in w.targets], np.int32)
    pos = np.concatenate([np.full(40, 1234), np.random.default_rng(5).integers(0, w.n, 160)])
    r = ctx.simulate(torch.tensor(w.energies[pos], device="cuda"), torch.tensor(tids[w.tidx][pos], device="cuda"),
                     seed=w.seed, precision="fp64", method="persistent", capacity=40 * len(pos),
                     event_ids=torch.tensor(w.first_event_id + pos, dtype=torch.int64, device="cuda"))
    torch.cuda.synchronize()
    gres, gsec = gpu_subset(r.residuals_np(), r.secondaries_np(), np.arange(len(pos)))
    c = compare(gres, gsec, oracle_at(w, pos), len(pos))
    assert c["frac_same"] >= 0.995, c


def test_event_ids_are_checked(ctx):
    import torch
    tid = ctx.create_target(8, 16)
    e = torch.full((8,), 100.0, dtype=torch.float64, device="cuda")
    t = torch.full((8,), tid, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        ctx.simulate(e, t, seed=1, event_ids=torch.arange(8, device="cuda", dtype=torch.int32))
    with pytest.raises(ValueError):
        ctx.simulate(e, t, seed=1, event_ids=torch.arange(7, device="cuda", dtype=torch.int64))


def test_graph_plan_with_ids_and_projectiles(ctx):
    """A CUDA-graph plan carries per-event ids and incident species like a direct launch."""
    import torch
    w = inputs.mixed(3000, seed=8)
    tids = np.array([ctx.create_target(*za) for za in w.targets], np.int32)
    e = torch.tensor(w.energies, device="cuda")
    t = torch.tensor(tids[w.tidx], device="cuda")
    rng = np.random.default_rng(9)
    ids = torch.tensor(rng.integers(0, 1 << 40, w.n), dtype=torch.int64, device="cuda")
    proj = torch.tensor(rng.integers(0, 2, w.n), dtype=torch.uint8, device="cuda")
    ref = ctx.simulate(e, t, seed=w.seed, capacity=40 * w.n, projectiles=proj, event_ids=ids)
    out = ctx.alloc(w.n, capacity=40 * w.n)
    g = ctx.graph(e, t, seed=w.seed, out=out, projectiles=proj, event_ids=ids)
    try:
        g.launch()
        torch.cuda.synchronize()
    finally:
        g.close()
    assert np.array_equal(out.residuals_np(), ref.residuals_np())
    assert np.array_equal(pnuc.sort_secondaries(out.secondaries_np()), pnuc.sort_secondaries(ref.secondaries_np()))
