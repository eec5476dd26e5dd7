"""Neutron-induced events (pnuc_batch.projectiles = 0): the incident nucleon's species,
mass and entry well change, and the residual keeps the target's charge. FP64 mode equals the
oracle event by event, alone and mixed with proton-induced events in one batch; FP32 mode
matches it observable by observable; other projectile values are flagged as bad input."""
import numpy as np
import pytest

import oracle
from paper_1309_7963_gb300 import inputs, pnuc

from .parity import assert_observables, compare, observable_table

pytestmark = pytest.mark.gpu


def run(ctx, w, proj, precision, method="persistent"):
    import torch
    tids = np.array([ctx.create_target(*za) for za in w.targets], np.int32)
    r = ctx.simulate(torch.tensor(w.energies, device="cuda"), torch.tensor(tids[w.tidx], device="cuda"), seed=w.seed,
                     first_event_id=w.first_event_id, precision=precision, method=method,
                     projectiles=torch.tensor(proj, dtype=torch.uint8, device="cuda"))
    torch.cuda.synchronize()
    return r


@pytest.mark.parametrize("method", ["plain", "persistent"])
def test_fp64_neutron_events_equal_the_oracle(ctx, method):
    w = inputs.fixed(inputs.O16, 200.0, 5000, seed=4)
    proj = np.zeros(w.n, np.uint8)
    r = run(ctx, w, proj, "fp64", method)
    orc = oracle.simulate(w.targets, w.energies, w.tidx, seed=w.seed, projectiles=proj)
    c = compare(r.residuals_np(), r.secondaries_np(), orc, w.n)
    assert c["frac_match"] >= 0.999, c["frac_match"]


def test_fp64_mixed_neutron_proton_batch(ctx):
    w = inputs.mixed(8000, seed=6)
    proj = np.random.default_rng(6).integers(0, 2, w.n).astype(np.uint8)
    r = run(ctx, w, proj, "fp64")
    orc = oracle.simulate_parallel(w.targets, w.energies, w.tidx, seed=w.seed, projectiles=proj)
    c = compare(r.residuals_np(), r.secondaries_np(), orc, w.n)
    assert c["frac_match"] >= 0.999, c["frac_match"]
    res = r.residuals_np()
    ok = (res["flags"] & 1) == 0
    # the neutrons' residuals after the cascade carry one unit of charge less on average
    zt = np.array([za[0] for za in w.targets])[w.tidx]
    dz = (res["Z_cascade"].astype(np.int64) - zt)
    assert dz[ok & (proj == 0)].mean() < dz[ok & (proj == 1)].mean() - 0.5


def test_fp32_neutron_observables(ctx):
    w = inputs.mixed(40_000, seed=7)
    proj = np.zeros(w.n, np.uint8)
    r = run(ctx, w, proj, "fp32")
    gres, gsec = r.residuals_np(), r.secondaries_np()
    orc = oracle.simulate_parallel(w.targets, w.energies, w.tidx, seed=w.seed, projectiles=proj)
    row = observable_table(gres, gsec, orc["residuals"], orc["secondaries"], w.n)
    assert_observables(row, "neutron-induced, mixed targets")
    assert compare(gres, gsec, orc, w.n)["frac_same"] >= 0.9


def test_bad_projectile_is_flagged(ctx):
    w = inputs.fixed(inputs.O16, 100.0, 64)
    proj = np.ones(w.n, np.uint8)
    proj[::4] = 2
    res = run(ctx, w, proj, "fp32").residuals_np()
    assert np.all((res["flags"][::4] & pnuc.FLAGS["bad_input"]) != 0)
    assert np.all((res["flags"][1::4] & pnuc.FLAGS["bad_input"]) == 0)
