"""The statistical checks the FP32-mode tests apply (tests/parity.py: multiplicities and mean
kinetic energies within 3 standard errors, chi-square and Kolmogorov-Smirnov p > 0.01, and the
paired comparison of the same events' records) have the power to see plausible mistakes: on
the CPU, oracle results recast as the library's records pass against themselves (kinetic
energies and directions rounded as the FP32 records store them) and fail once a mistake is
planted in the copy: a 2% or a 0.5% energy scale, a mirrored angular distribution, lost
emissions, and one in five of the rare tritons or 3He dropped."""
import numpy as np
import pytest

from paper_1309_7963_gb300 import inputs, pnuc

import oracle

from .parity import assert_observables, observable_table


@pytest.fixture(scope="module")
def ca40():
    w = inputs.fixed(inputs.CA40, 200.0, 20_000, seed=9)
    r = oracle.simulate(w.targets, w.energies, w.tidx, seed=w.seed)
    return w.n, r["residuals"], r["secondaries"]


def as_library_records(res, sec):
    """Oracle records in the library's record layout (FP32 directions, as stored)."""
    g = np.zeros(len(sec), pnuc.SECONDARY_DTYPE)
    for f in ("event", "species", "origin", "index", "T", "ux", "uy", "uz"):
        g[f] = sec[f]
    r = np.zeros(len(res), pnuc.RESIDUAL_DTYPE)
    r["Z_final"], r["A_final"], r["flags"] = res["Zf"], res["Af"], res["flags"]
    r["Estar_cascade"] = res["Estar_c"]
    return r, g


def test_identical_results_pass(ca40):
    n, res, sec = ca40
    gres, gsec = as_library_records(res, sec)
    row = observable_table(gres, gsec, res, sec, n)
    assert row["multiplicity"] and row["ks_T_p"] and row["fig2_p"]
    assert_observables(row, "oracle against itself")


def planted(ca40, how):
    n, res, sec = ca40
    gres, gsec = as_library_records(res, sec)
    if how == "energy scale":
        sel = (gsec["species"] == 1) & (gsec["origin"] == 1)  # evaporated protons 2% hot
        gsec["T"][sel] *= 1.02
    elif how == "mirrored angles":
        sel = (gsec["species"] == 0) & (gsec["origin"] == 0)  # cascade neutrons backwards
        gsec["uz"][sel] = -gsec["uz"][sel]
    elif how == "half-percent energy scale":
        sel = (gsec["species"] == 1) & (gsec["origin"] == 1)  # evaporated protons 0.5% hot
        gsec["T"][sel] *= 1.005
    elif how == "lost emissions":
        alpha = np.flatnonzero((gsec["species"] == 5) & (gsec["origin"] == 1))
        gsec = np.delete(gsec, alpha[::5])  # every fifth evaporated alpha dropped
    elif how in ("lost tritons", "lost 3He"):
        sp = 3 if how == "lost tritons" else 4
        rare = np.flatnonzero((gsec["species"] == sp) & (gsec["origin"] == 1))
        gsec = np.delete(gsec, rare[::5])  # every fifth evaporated t (3He) dropped
    return observable_table(gres, gsec, res, sec, n)


@pytest.mark.parametrize("how", ["energy scale", "half-percent energy scale", "mirrored angles", "lost emissions",
                                 "lost tritons", "lost 3He"])
def test_planted_mistakes_fail(ca40, how):
    with pytest.raises(AssertionError):
        assert_observables(planted(ca40, how), how)
