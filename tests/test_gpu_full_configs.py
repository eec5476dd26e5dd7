"""The workloads at their full sizes, in the launch configurations they name: 2e6 p-16O +
p-40Ca events with the plain FP32 kernel, 4e6 mixed-target events (one autotuned persistent
launch replayed from a CUDA graph) and 1e6 events on each heavy target. Checked against the
oracle run on every event on the host cores (spectra, angles, the paper's Fig. 2 windows,
residual (Z, A), multiplicities), on sampled events it computes one by one (per-event
integers), and, over every event, by properties that hold at any size: baryon number and
charge conservation, flags."""
import os

import numpy as np
import pytest

from paper_1309_7963_gb300 import inputs, pnuc

import oracle

from .parity import assert_observables, compare, gpu_subset, observable_table, oracle_at

pytestmark = pytest.mark.gpu

EJ_Z = np.array([0, 1, 1, 1, 2, 2])
EJ_A = np.array([1, 1, 2, 3, 3, 4])


def conservation(w, res, sec):
    """Events (flags 0 or no-excitation) whose target + proton = residual + secondaries in
    charge and baryon number; returns the fraction of such events that conserve both."""
    n = w.n
    zt = np.array([za[0] for za in w.targets])[w.tidx]
    at = np.array([za[1] for za in w.targets])[w.tidx]
    ev = sec["event"].astype(np.int64)
    zs = np.bincount(ev, weights=EJ_Z[sec["species"]], minlength=n)
    as_ = np.bincount(ev, weights=EJ_A[sec["species"]], minlength=n)
    ok = (res["flags"] & ~np.uint32(32)) == 0
    good = (zt + 1 == res["Z_final"] + zs) & (at + 1 == res["A_final"] + as_)
    return ok, good


def sample_ids(n, k, seed):
    return np.unique(np.concatenate([np.linspace(0, n - 1, k).astype(np.int64), [0, n - 1],
                                     np.random.default_rng(seed).integers(0, n, k // 10)]))


def test_mixed_targets_4e6_graph_replay_autotuned(ctx):
    import torch
    w = inputs.mixed(4_000_000, seed=0)
    tids = np.array([ctx.create_target(*za) for za in w.targets], np.int32)
    e = torch.tensor(w.energies, device="cuda")
    t = torch.tensor(tids[w.tidx], device="cuda")
    saved = ctx.get_tuning("fp32")
    try:
        ctx.autotune(e, t, seed=w.seed, precision="fp32", reps=1)
        out = ctx.alloc(w.n, capacity=8 * w.n)
        g = ctx.graph(e, t, seed=w.seed, out=out, precision="fp32")
        g.launch()
        torch.cuda.synchronize()
        g.close()
    finally:
        ctx.set_tuning("fp32", **saved)
    res, sec = out.residuals_np(), out.secondaries_np()
    assert out.n_secondaries() <= 8 * w.n
    ok, good = conservation(w, res, sec)
    assert ok.mean() > 0.995 and good[ok].all()
    ids = sample_ids(w.n, 1500, 1)
    gres, gsec = gpu_subset(res, sec, ids)
    c = compare(gres, gsec, oracle_at(w, ids), len(ids))
    assert c["frac_same"] >= 0.97, c["frac_same"]
    # every event against the oracle run on all of them: spectra, angles, Fig. 2 windows,
    # residual (Z, A), multiplicities
    orc = oracle.simulate_parallel(w.targets, w.energies, w.tidx, seed=w.seed)
    row = observable_table(res, sec, orc["residuals"], orc["secondaries"], w.n)
    assert_observables(row, "mixed targets 4e6")
    assert row["residual_ZA_identical"] > 0.99
    record("full size: mixed targets 20-250 MeV, 4e6 events, autotuned graph replay", row)


def record(name, row):
    path = os.environ.get("PNUC_OBSERVABLES_OUT")
    if path:
        import json
        data = json.load(open(path)) if os.path.exists(path) else {}
        data[name] = row
        json.dump(data, open(path, "w"), indent=1)


def test_plain_fp32_o16_ca40_2e6_against_the_oracle(ctx):
    import torch
    w = inputs.oxygen_calcium(n_each=1_000_000)
    tids = np.array([ctx.create_target(*za) for za in w.targets], np.int32)
    r = ctx.simulate(torch.tensor(w.energies, device="cuda"), torch.tensor(tids[w.tidx], device="cuda"), seed=w.seed,
                     precision="fp32", method="plain", capacity=8 * w.n)
    torch.cuda.synchronize()
    res, sec = r.residuals_np(), r.secondaries_np()
    ok, good = conservation(w, res, sec)
    assert ok.mean() > 0.995 and good[ok].all()
    orc = oracle.simulate_parallel(w.targets, w.energies, w.tidx, seed=w.seed)
    row = observable_table(res, sec, orc["residuals"], orc["secondaries"], w.n)
    record("full size: p-16O + p-40Ca 200 MeV, 2e6 events, plain FP32 kernel", row)
    assert_observables(row, "plain fp32 2e6")
    assert row["residual_ZA_identical"] > 0.99


@pytest.mark.parametrize("target", [inputs.TI48, inputs.FE56, inputs.PB208], ids=["48Ti", "56Fe", "208Pb"])
def test_heavy_targets_1e6(ctx, target):
    import torch
    w = inputs.heavy(target, 1_000_000, seed=3)
    tids = np.array([ctx.create_target(*za) for za in w.targets], np.int32)
    e = torch.tensor(w.energies, device="cuda")
    t = torch.tensor(tids[w.tidx], device="cuda")
    r = ctx.simulate(e, t, seed=w.seed, precision="fp32", method="persistent", capacity=24 * w.n)
    torch.cuda.synchronize()
    res, sec = r.residuals_np(), r.secondaries_np()
    ok, good = conservation(w, res, sec)
    assert ok.mean() > 0.995 and good[ok].all()
    orc = oracle.simulate_parallel(w.targets, w.energies, w.tidx, seed=w.seed)
    row = observable_table(res, sec, orc["residuals"], orc["secondaries"], w.n)
    assert_observables(row, f"{target} 1e6")
    assert row["residual_ZA_identical"] > 0.99
    ids = sample_ids(w.n, 500, 2)
    gres, gsec = gpu_subset(res, sec, ids)
    c = compare(gres, gsec, oracle_at(w, ids), len(ids))
    assert c["frac_same"] >= 0.97, c["frac_same"]
    record(f"full size: p-{target} 100-250 MeV, 1e6 events", row)
