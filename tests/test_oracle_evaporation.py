"""Pins of the oracle's evaporation (§2.4: GEM-style emission of n, p, d, t, 3He, alpha,
isotropic in the nucleus rest frame): width integrals against adaptive quadrature, channel
thresholds, the emission-energy sampler against its normalised density."""
import numpy as np
import pytest
from scipy import integrate, stats

import oracle


def width_ref(a, Y, b):
    f = lambda U: (Y + b - U) * np.exp(2 * np.sqrt(a * U))
    # substitution U = s^2 removes the square-root kink at U = 0
    g = lambda s: f(s * s) * 2 * s
    return integrate.quad(g, 0, np.sqrt(Y), epsabs=0, epsrel=1e-13, limit=400)[0]


@pytest.mark.parametrize("a", [0.5, 2.0, 5.0, 26.0])
@pytest.mark.parametrize("Y", [1e-6, 0.01, 0.1249, 0.1251, 0.5, 3.0, 20.0, 120.0])
@pytest.mark.parametrize("b", [0.0, 0.3])
def test_width_integral_against_quadrature(a, Y, b):
    got = oracle.width_integral(a, Y, b)
    ref = width_ref(a, Y, b)
    tol = 1e-10 if 2 * np.sqrt(a * Y) > 1e-2 else 1e-8
    assert got == pytest.approx(ref, rel=tol)


def test_width_series_and_closed_form_join_at_x_one():
    # x = 2 sqrt(aY) = 1 is where the series hands over to the closed form
    a = 2.0
    Y = 1.0 / (4 * a)
    lo, hi = oracle.width_integral(a, Y * (1 - 1e-13), 0.2), oracle.width_integral(a, Y * (1 + 1e-13), 0.2)
    assert abs(hi - lo) / hi < 1e-11


def test_channel_thresholds_and_q_values():
    # 16O: Q_n and Q_p are the SEMF separation energies, close to measured 15.66 and 12.13 MeV
    c_n = oracle.channel(8, 16, 30.0, 0)
    c_p = oracle.channel(8, 16, 30.0, 1)
    c_a = oracle.channel(8, 16, 30.0, 5)
    assert c_n["Q"] == pytest.approx(15.66, abs=2.5)
    assert c_p["Q"] == pytest.approx(12.13, abs=2.0)
    assert c_a["Q"] == pytest.approx(7.16, abs=4.0)
    # charged barrier of alpha on 12C: e^2 2 6 / (1.5 (4^1/3 + 12^1/3)) MeV
    assert c_a["V"] == pytest.approx(1.44 * 12 / (1.5 * (4 ** (1 / 3) + 12 ** (1 / 3))), rel=1e-12)
    for j in range(6):
        c = oracle.channel(8, 16, 30.0, j)
        thr = c["Q"] + c["V"]
        assert oracle.channel(8, 16, thr - 1e-9, j)["width"] == 0.0
        assert oracle.channel(8, 16, thr + 1e-6, j)["width"] > 0.0
    # closed channels: daughter lighter than A = 5, or without protons / neutrons
    assert oracle.channel(3, 6, 50.0, 5)["width"] == 0.0
    assert oracle.channel(2, 6, 50.0, 4)["width"] == 0.0


@pytest.mark.parametrize("a,Y,b", [(2.0, 0.2, 0.0), (2.0, 0.2, 0.35), (2.0, 30.0, 0.0), (3.0, 10.0, 0.25),
                                   (26.0, 12.0, 0.0), (0.75, 0.9, 0.2)])
def test_emission_sampler_matches_normalised_density(a, Y, b):
    x = 2 * np.sqrt(a * Y)
    U, trials = oracle.sample_U(a, x, b, 200000, seed=4, event=int(100 * a + Y))
    assert U.min() >= 0 and U.max() <= Y * (1 + 1e-12)
    assert trials / len(U) < 12  # acceptance never collapses near threshold
    # chi-square of 40 equal-width bins against the exact integral of the density
    edges = np.linspace(0, Y, 41)
    f = lambda u: (Y + b - u) * np.exp(2 * np.sqrt(a * u))
    g = lambda s: f(s * s) * 2 * s
    mass = np.array([integrate.quad(g, np.sqrt(lo), np.sqrt(hi), epsrel=1e-12)[0] for lo, hi in zip(edges[:-1], edges[1:])])
    expect = mass / mass.sum() * len(U)
    h, _ = np.histogram(U, bins=edges)
    keep = expect > 5
    chi2 = (((h - expect) ** 2) / expect)[keep].sum()
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-3


def test_single_open_channel_spectrum():
    # 11C at 9 MeV: find the (Z,A,E*) where only the neutron channel is open, then the
    # chosen channel must always be n and the U density is the neutron integrand
    Z, A = 6, 12
    thr = sorted((oracle.channel(Z, A, 0.0, j)["Q"] + oracle.channel(Z, A, 0.0, j)["V"], j) for j in range(6))
    lowest, second = thr[0], thr[1]
    E = 0.5 * (lowest[0] + second[0])
    widths = [oracle.channel(Z, A, E, j)["width"] for j in range(6)]
    assert sum(w > 0 for w in widths) == 1 and widths[lowest[1]] > 0
