"""FP32 modes against the FP64 oracle, observable by observable, on the same events: the FP32
mode (FP64 evaporation widths) and the scaled FP32 mode (FP32 widths scaled by the largest
channel's exponential).

For each workload: the fraction of events whose integer outcomes are identical, the mean
multiplicity of every species (cascade and evaporation) with the difference in units of its
standard error, binned kinetic-energy spectra and angular distributions, the evaporated n and
p spectra in 1-degree windows at the angles of the paper's Fig. 2, the residual (Z, A)
distribution (two-sample chi-square p-values), and the mean E* after the cascade. Bounds
asserted: identical integers on >= 90% of events, multiplicities within 3 sigma, chi-square
p > 0.01. The table is written as JSON to the path in the environment variable
PNUC_OBSERVABLES_OUT when it is set.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1309_7963_gb300 import inputs

from .parity import assert_observables, compare, observable_table

pytestmark = pytest.mark.gpu

WORKLOADS = [
    ("p-16O + p-40Ca 200 MeV", lambda: inputs.oxygen_calcium(n_each=25_000)),
    ("mixed tissue targets 20-250 MeV", lambda: inputs.mixed(40_000, seed=2)),
    ("p-48Ti 100-250 MeV", lambda: inputs.heavy(inputs.TI48, 10_000, seed=3)),
    ("p-56Fe 100-250 MeV", lambda: inputs.heavy(inputs.FE56, 10_000, seed=4)),
    ("p-208Pb 100-250 MeV", lambda: inputs.heavy(inputs.PB208, 6_000, seed=5)),
]


@pytest.mark.parametrize("precision", ["fp32", "fp32_scaled"])
@pytest.mark.parametrize("name,make", WORKLOADS, ids=[w[0] for w in WORKLOADS])
def test_fp32_observables_against_fp64_oracle(ctx, name, make, precision):
    import torch
    w = make()
    tids = np.array([ctx.create_target(*za) for za in w.targets], np.int32)
    r = ctx.simulate(torch.tensor(w.energies, device="cuda"), torch.tensor(tids[w.tidx], device="cuda"), seed=w.seed,
                     first_event_id=w.first_event_id, precision=precision, method="persistent")
    torch.cuda.synchronize()
    gres, gsec = r.residuals_np(), r.secondaries_np()
    orc = oracle.simulate_parallel(w.targets, w.energies, w.tidx, seed=w.seed, first_event_id=w.first_event_id)
    ores, osec = orc["residuals"], orc["secondaries"]
    c = compare(gres, gsec, orc, w.n, rel_tol=1e-4)
    row = observable_table(gres, gsec, ores, osec, w.n)
    row.update(workload=name, precision=precision, identical_integers=c["frac_same"], **{"identical_within_1e-4": c["frac_match"]})
    row["mean_A_final"] = {"fp32": float(gres["A_final"].mean()), "oracle": float(ores["Af"].mean())}
    assert_observables(row, name)
    assert c["frac_same"] >= 0.90, c["frac_same"]
    record(f"{name} [{precision}]", row)


def record(name, row):
    path = os.environ.get("PNUC_OBSERVABLES_OUT")
    if path:
        data = json.load(open(path)) if os.path.exists(path) else {}
        data[name] = row
        json.dump(data, open(path, "w"), indent=1)
