"""The FP32 modes stay finite. Over the bench workload and a mixed-target batch (3e6 events in
all) every secondary has a finite, non-negative kinetic energy and a unit direction, and every
residual a finite E* after the cascade and at the end. The case this guards: the emission
energy of an evaporation step (§2.4) is E* - Q less the daughter's excitation U_d, and for a
channel without barrier a draw of t close to 0 can put U_d an FP32 rounding above E* - Q;
the FP32 decay then takes the release as 0 instead of computing a NaN momentum."""
import numpy as np
import pytest

from paper_1309_7963_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "fp32_scaled"])
@pytest.mark.parametrize("workload", ["oxygen_calcium", "mixed"])
def test_fp32_outputs_finite(ctx, workload, precision):
    import torch
    w = inputs.oxygen_calcium(500_000, seed=5) if workload == "oxygen_calcium" else inputs.mixed(2_000_000, seed=6)
    n = w.n
    tids = np.array([ctx.create_target(*za) for za in w.targets], np.int32)
    e = torch.tensor(w.energies, device="cuda")
    t = torch.tensor(tids[w.tidx], device="cuda")
    r = ctx.simulate(e, t, seed=w.seed, first_event_id=w.first_event_id, precision=precision, method="persistent")
    sec, res = r.secondaries_np(), r.residuals_np()
    assert len(sec) > 3 * n
    u = np.stack([sec["ux"], sec["uy"], sec["uz"]], 1).astype(np.float64)
    assert np.isfinite(sec["T"]).all() and np.isfinite(u).all()
    assert (sec["T"] >= -1e-6).all()
    assert np.abs(np.sqrt((u * u).sum(1)) - 1.0).max() < 1e-3
    assert np.isfinite(res["Estar_cascade"]).all() and np.isfinite(res["Estar_final"]).all()
