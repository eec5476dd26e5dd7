"""Reading M26 on the GPU (pnuc_config.level_density = 1: GEM's constant-temperature level
density below U_x = 2.5 + 150/A_d MeV, the Fermi gas above, §2.4): the FP64 mode reproduces
the oracle run with the same option event by event (integer outcomes identical and energies
within 1e-9 on >= 99.9% of events), with every method; the FP32 mode matches the oracle's
observables; the scaled FP32 widths refuse the option."""
import numpy as np
import pytest

import oracle
from paper_1309_7963_gb300 import inputs, pnuc

from .parity import assert_observables, compare, observable_table

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx_ct():
    c = pnuc.Context(0, level_density=1)
    yield c
    c.close()


def run(ctx, w, precision, method):
    import torch
    tids = np.array([ctx.create_target(*za) for za in w.targets], np.int32)
    r = ctx.simulate(torch.tensor(w.energies, device="cuda"), torch.tensor(tids[w.tidx], device="cuda"), seed=w.seed,
                     first_event_id=w.first_event_id, precision=precision, method=method, capacity=40 * w.n)
    torch.cuda.synchronize()
    return r


def oracle_ct(w):
    return oracle.simulate_parallel(w.targets, w.energies, w.tidx, seed=w.seed, first_event_id=w.first_event_id,
                                    limits={"level_density": 1}, chunk=512)


@pytest.mark.parametrize("method", ["plain", "persistent", "sorted"])
@pytest.mark.parametrize("workload", ["o16", "mixed", "pb208"])
def test_fp64_per_event_parity_with_the_composite_level_density(ctx_ct, workload, method):
    w = {"o16": lambda: inputs.plain_fp64(6000), "mixed": lambda: inputs.mixed(6000, seed=3),
         "pb208": lambda: inputs.heavy(inputs.PB208, 3000, seed=7)}[workload]()
    r = run(ctx_ct, w, "fp64", method)
    orc = oracle_ct(w)
    c = compare(r.residuals_np(), r.secondaries_np(), orc, w.n)
    assert c["frac_match"] >= 0.999, c["frac_match"]
    assert c["max_rel_energy_same"] < 1e-6
    # the option changes the evaporation (the same events with the Fermi gas differ)
    orc0 = oracle.simulate_parallel(w.targets, w.energies, w.tidx, seed=w.seed, first_event_id=w.first_event_id,
                                    chunk=512)
    assert not np.array_equal(orc0["residuals"]["Af"], orc["residuals"]["Af"])


@pytest.mark.parametrize("workload", ["oxygen_calcium", "heavy"])
def test_fp32_observables_with_the_composite_level_density(ctx_ct, workload):
    w = inputs.oxygen_calcium(n_each=25_000) if workload == "oxygen_calcium" else inputs.heavy(inputs.FE56, 20_000, seed=4)
    r = run(ctx_ct, w, "fp32", "persistent")
    gres, gsec = r.residuals_np(), r.secondaries_np()
    orc = oracle_ct(w)
    row = observable_table(gres, gsec, orc["residuals"], orc["secondaries"], w.n)
    assert_observables(row, f"level density M26, {workload}")
    assert compare(gres, gsec, orc, w.n, rel_tol=1e-4)["frac_same"] >= 0.97


def test_scaled_fp32_widths_refuse_the_composite_level_density(ctx_ct):
    w = inputs.plain_fp64(64)
    with pytest.raises(pnuc.PnucError):
        run(ctx_ct, w, "fp32_scaled", "persistent")
