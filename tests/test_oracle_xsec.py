"""Pins of the oracle's NN cross sections (§2.3, Cugnon et al. parametrisations) and of
the collision-rate majorant (Metropolis et al.'s maximum-cross-section sequence)."""
import json
import os

import numpy as np
import pytest

import oracle

DATA = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "nuclear_data.json")))
MP, MN = oracle.M_P, oracle.M_N


def plab_gev(T_mev, m=MP):
    return np.sqrt(T_mev * T_mev + 2 * T_mev * m) * 1e-3


@pytest.mark.parametrize("pair,like", [("pp", True), ("np", False)])
def test_total_cross_sections_against_measured(pair, like):
    ref = DATA["nn_total_cross_section_mb"][pair]
    assert oracle.sigma(like, plab_gev(200.0)) == pytest.approx(ref["200"], rel=0.10)
    assert oracle.sigma(like, plab_gev(100.0)) == pytest.approx(ref["100"], rel=0.25)


def test_parametrisation_fixed_points_and_branch_joins():
    assert oracle.sigma(True, 0.4) == pytest.approx(34.0, rel=1e-15)
    assert oracle.sigma(True, 0.7) == pytest.approx(23.5, rel=1e-15)
    e = 1e-12
    for like, p in [(True, 0.44), (True, 0.8), (False, 0.8)]:
        lo, hi = oracle.sigma(like, p - e), oracle.sigma(like, p + e)
        assert abs(lo - hi) / hi < 0.012, (like, p, lo, hi)
    # clamped to [0.1, 2] GeV/c
    assert oracle.sigma(True, 0.01) == oracle.sigma(True, 0.1)
    assert oracle.sigma(False, 5.0) == oracle.sigma(False, 2.0)


def test_np_slope_branches_join():
    # the np slope's pieces join (to 0.3% at 0.6 GeV/c, to 1e-12 at 1.6); the slopes are pinned
    # against measured angular distributions in test_oracle_nn_angular.py
    for p, tol in ((0.6, 0.004), (1.6, 1e-9)):
        a, b = oracle.slope(False, p - 1e-12), oracle.slope(False, p + 1e-12)
        assert abs(a - b) / b < tol, (p, a, b)


def test_g_pieces_bound_p_sigma():
    # the majorant's piecewise bound of g(p) = p sigma(p) on a fine grid (brute force)
    p = np.linspace(0.001, 2.0, 200001)
    gpp = np.array([x * oracle.sigma(True, x) for x in p[::20]])
    gnp = np.array([x * oracle.sigma(False, x) for x in p[::20]])
    pc = p[::20]
    assert gnp[pc < 0.8].max() < 31.0
    assert (oracle.sigma(True, 0.44) <= 28.1) and max(oracle.sigma(True, x) for x in np.linspace(0.44, 2, 2001)) <= 28.1
    assert np.all(np.diff(gpp[(pc > 0.1) & (pc < 0.44)]) < 0)
    assert np.all(np.diff(gnp[pc > 0.8]) > 0)


def _fermi_partners(pF, n, rng):
    q = pF * rng.random(n) ** (1 / 3)
    ct = 2 * rng.random(n) - 1
    ph = 2 * np.pi * rng.random(n)
    st = np.sqrt(1 - ct * ct)
    return np.stack([q * st * np.cos(ph), q * st * np.sin(ph), q * ct], 1)


@pytest.mark.parametrize("Z,A", [(8, 16), (82, 208)])
def test_majorant_bounds_every_partner(Z, A):
    # brute force: sigma * v_rel * E1 never exceeds g_hat, for projectiles of 5-400 MeV,
    # partners from every shell's Fermi spheres, including the worst (collinear) partners
    t = oracle.target(Z, A)
    rng = np.random.default_rng(1)
    worst = 0.0
    for i in range(15):
        vF = t["vF"][i]
        for s1, m1 in ((0, MN), (1, MP)):
            for T1 in (5.0, 20.0, 35.0, 50.0, 80.0, 150.0, 250.0, 400.0):
                p1m = np.sqrt(T1 * T1 + 2 * T1 * m1)
                E1 = T1 + m1
                gh = oracle.g_hat(p1m, E1, vF)
                p1 = np.array([0.0, 0.0, p1m])
                for s2, m2 in ((0, MN), (1, MP)):
                    pF = t["pF"][s2][i]
                    P = _fermi_partners(pF, 4000, rng)
                    P = np.concatenate([P, [[0, 0, pF], [0, 0, -pF], [0, 0, 0.5 * pF]]])
                    E2 = np.sqrt((P * P).sum(1) + m2 * m2)
                    X = np.maximum((E1 * E2 - P @ p1) - m1 * m2, 0)
                    k = np.sqrt(X * (X + 2 * m1 * m2))
                    plab = k / m2 * 1e-3
                    sig = np.array([oracle.sigma(s1 == s2, x) for x in plab])
                    ratio = (sig * k / (E1 * E2) * E1 * 1e-3) / gh
                    worst = max(worst, ratio.max())
    assert worst <= 1.0
    assert worst > 0.3  # and it is not absurdly loose
