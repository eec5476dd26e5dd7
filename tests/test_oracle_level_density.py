"""Pins of reading M26, the option of a composite level density in the evaporation (§2.4:
GEM after Furihata, whose level density is Gilbert and Cameron's): constant temperature below
the matching energy U_x = 2.5 + 150/A_d MeV, M20's Fermi gas exp(2 sqrt(aU)) above, joined
in value and slope. Checked: the switch energy against the Gilbert-Cameron systematics, the
joint (value and slope, by finite differences from both sides), the constant-temperature part
(log-linear), the width integrals against adaptive quadrature of the density, the emission
sampler against its normalised density (chi-square), and whole events in that mode
(conservation and the evaporation invariants)."""
import json
import os

import numpy as np
import pytest
from scipy import integrate, stats

import oracle

GC = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "level_density.json")))[
    "gilbert_cameron_matching_energy_MeV"]
AD = [6, 16, 40, 56, 120, 206]  # daughter mass numbers


def Ux_of(Ad):
    return GC["constant"] + GC["over_A"] / Ad


@pytest.mark.parametrize("Ad", AD)
def test_constant_temperature_below_the_gilbert_cameron_energy_and_fermi_gas_above(Ad):
    a = Ad / 8.0
    Ux = Ux_of(Ad)
    # above U_x the two modes coincide; below, the composite density differs
    for U in (Ux * (1 + 1e-9), 1.5 * Ux, 3 * Ux, 100.0):
        assert oracle.level_density(a, U, 1) == oracle.level_density(a, U, 0)
    for U in (0.0, 0.3 * Ux, 0.9 * Ux, Ux * (1 - 1e-6)):
        assert oracle.level_density(a, U, 1) != oracle.level_density(a, U, 0)
    # below U_x: a constant temperature, log rho linear in U (zero second differences)
    us = np.linspace(0.05 * Ux, 0.95 * Ux, 9)
    lr = np.log([oracle.level_density(a, u, 1) for u in us])
    assert np.abs(np.diff(lr, 2)).max() < 1e-11 * np.abs(lr).max()


@pytest.mark.parametrize("Ad", AD)
def test_value_and_slope_join_at_the_matching_energy(Ad):
    a = Ad / 8.0
    Ux = Ux_of(Ad)
    h = 1e-5 * Ux
    lo = [np.log(oracle.level_density(a, Ux - k * h, 1)) for k in (1, 2)]
    hi = [np.log(oracle.level_density(a, Ux + k * h, 1)) for k in (1, 2)]
    # value: both one-sided extrapolations to U_x agree
    v_lo, v_hi = 2 * lo[0] - lo[1], 2 * hi[0] - hi[1]
    assert v_lo == pytest.approx(v_hi, rel=1e-9)
    # slope of log rho (1/T) from either side
    s_lo, s_hi = (lo[0] - lo[1]) / h, (hi[1] - hi[0]) / h
    assert s_lo == pytest.approx(s_hi, rel=2e-4)


def width_ct_ref(a, Y, b):
    f = lambda U: (Y + b - U) * oracle.level_density(a, U, 1)
    Ux = Ux_of(8 * a)
    if Y <= Ux:
        return integrate.quad(f, 0, Y, epsabs=0, epsrel=1e-13, limit=400)[0], None
    g = lambda s: f(s * s) * 2 * s  # U = s^2 above U_x
    ct = integrate.quad(f, 0, Ux, epsabs=0, epsrel=1e-13, limit=400)[0]
    fg = integrate.quad(g, np.sqrt(Ux), np.sqrt(Y), epsabs=0, epsrel=1e-13, limit=400)[0]
    return ct + fg, ct


@pytest.mark.parametrize("Ad", [6, 16, 56, 206])
@pytest.mark.parametrize("frac", [1e-6, 0.02, 0.5, 0.999, 1.001, 2.0, 10.0])
@pytest.mark.parametrize("b", [0.0, 0.3])
def test_width_integral_against_quadrature(Ad, frac, b):
    a = Ad / 8.0
    Y = frac * Ux_of(Ad)
    got, got_ct = oracle.width_integral_ct(a, Y, b)
    ref, ref_ct = width_ct_ref(a, Y, b)
    assert got == pytest.approx(ref, rel=1e-10)
    if ref_ct is not None:
        assert got_ct == pytest.approx(ref_ct, rel=1e-10)
    else:
        assert got_ct == got


def test_fermi_gas_widths_unchanged_by_default():
    for j in range(6):
        c0 = oracle.channel(20, 40, 45.0, j)
        assert oracle.channel(20, 40, 45.0, j, level_density=0)["width"] == c0["width"]
    # M26 changes them (below and across U_x) but not the thresholds
    c = oracle.channel(20, 40, 45.0, 0, level_density=1)
    assert c["width"] > 0 and c["width"] != oracle.channel(20, 40, 45.0, 0)["width"]


@pytest.mark.parametrize("Ad,frac,b", [(16, 0.05, 0.0), (16, 0.6, 0.4), (40, 0.9, 0.0), (56, 3.0, 0.0),
                                       (56, 1.2, 0.3), (206, 25.0, 0.0), (6, 0.3, 0.2)])
def test_emission_sampler_matches_normalised_density(Ad, frac, b):
    a = Ad / 8.0
    Ux = Ux_of(Ad)
    Y = frac * Ux
    U, trials = oracle.sample_U_ct(a, Y, b, 200000, seed=6, event=Ad * 100 + int(10 * frac))
    assert U.min() >= 0 and U.max() <= Y * (1 + 1e-12)
    assert trials / len(U) < 12
    edges = np.linspace(0, Y, 41)
    if 0 < Ux < Y:
        edges = np.unique(np.concatenate([edges, [Ux]]))
    f = lambda u: (Y + b - u) * oracle.level_density(a, u, 1)
    mass = np.array([integrate.quad(f, lo, hi, epsrel=1e-12)[0] for lo, hi in zip(edges[:-1], edges[1:])])
    expect = mass / mass.sum() * len(U)
    h, _ = np.histogram(U, bins=edges)
    keep = expect > 5
    chi2 = (((h - expect) ** 2) / expect)[keep].sum()
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-3


@pytest.mark.parametrize("za,energy", [((8, 16), 200.0), ((20, 40), 150.0), ((82, 208), 120.0)])
def test_events_with_the_composite_density_conserve_and_respect_thresholds(za, energy):
    Z, A = za
    n = 1000
    r = oracle.simulate([za], np.full(n, energy), np.zeros(n, np.int32), seed=2,
                        limits={"level_density": 1}, trace=True, trace_cap=1 << 22)
    sec, res = r["secondaries"], r["residuals"]
    ok = (res["flags"] & ~np.uint32(32 | 16)) == 0
    assert ok.mean() > 0.95
    za_ej, m_ej = np.array(oracle.EJECTILE_ZA), np.array(oracle.EJECTILE_MASS)
    ev = sec["event"]
    sa = np.bincount(ev, weights=za_ej[sec["species"], 1], minlength=n)
    sz = np.bincount(ev, weights=za_ej[sec["species"], 0], minlength=n)
    assert np.all(sa[ok] + res["Af"][ok] == A + 1) and np.all(sz[ok] + res["Zf"][ok] == Z + 1)
    Ein = energy + oracle.M_P + oracle.semf_mass(Z, A)
    Eout = np.bincount(ev, weights=sec["T"] + m_ej[sec["species"]], minlength=n) + res["Ef"]
    assert np.allclose(Eout[ok], Ein, rtol=1e-12, atol=0)
    tr = r["trace"]
    evp = tr[tr["kind"] == oracle.TRACE_KINDS["evap"]]
    assert len(evp) > n
    eps, V, Q, Es = evp["T"], evp["x"], evp["y"], evp["z"]
    assert np.all(eps >= V - 1e-9) and np.all(Es >= Q + V) and np.all(eps <= Es - Q + 1e-9)
    # the mode changes the evaporation, not the cascade
    r0 = oracle.simulate([za], np.full(n, energy), np.zeros(n, np.int32), seed=2)
    assert np.array_equal(r0["residuals"]["Ac"], res["Ac"]) and np.array_equal(r0["residuals"]["Zc"], res["Zc"])
    assert not np.array_equal(r0["residuals"]["Af"], res["Af"])
