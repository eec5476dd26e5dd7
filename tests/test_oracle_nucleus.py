"""Pins of the oracle's nucleus set-up (§2.2, Eq. 1): SEMF masses against measured
binding energies, shell densities against independent quadrature, Fermi-gas values."""
import json
import os

import numpy as np
import pytest
from scipy import integrate

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")
PAPER = json.load(open(os.path.join(GOLD, "paper_constants.json")))
DATA = json.load(open(os.path.join(GOLD, "nuclear_data.json")))
HBARC = 197.3269804


def binding(Z, A):
    return Z * oracle.M_P + (A - Z) * oracle.M_N - oracle.semf_mass(Z, A)


@pytest.mark.parametrize("za,b_exp", [(tuple(map(int, k.split(","))), v) for k, v in DATA["binding_energy_MeV"].items()])
def test_semf_binding_against_measured(za, b_exp):
    # the liquid-drop formula reproduces measured binding energies to ~1-3% for A >= 12;
    # a dropped term or a flipped sign misses by far more
    assert abs(binding(*za) - b_exp) / b_exp < 0.035


def test_semf_separation_energies_against_measured():
    for key, seps in DATA["separation_energy_MeV"].items():
        Z, A = map(int, key.split(","))
        t = oracle.target(Z, A)
        assert abs(t["S"][0] - seps["n"]) < 2.5, (key, t["S"][0])
        assert abs(t["S"][1] - seps["p"]) < 4.0, (key, t["S"][1])


def test_paper_constants_in_target_table():
    for Z, A in [(6, 12), (8, 16), (20, 40), (82, 208)]:
        t = oracle.target(Z, A)
        c = PAPER["density_c_coefficient_fm"]["value"] * A ** (1 / 3)
        assert t["c"] == pytest.approx(c, rel=1e-15)
        assert t["R"] == pytest.approx(c + PAPER["radius_offset_fm"]["value"], rel=1e-15)
        n = PAPER["n_shells"]["value"]
        assert np.allclose(t["r"], np.arange(n + 1) * t["R"] / n, rtol=1e-15)


@pytest.mark.parametrize("Z,A", [(6, 12), (8, 16), (20, 40), (26, 56), (82, 208)])
def test_shell_densities_against_quadrature(Z, A):
    t = oracle.target(Z, A)
    c, delta = t["c"], PAPER["density_diffuseness_fm"]["value"]
    f = lambda r: r * r / (1.0 + np.exp((r - c) / delta))
    I = np.array([integrate.quad(f, t["r"][i], t["r"][i + 1], epsabs=0, epsrel=5e-14, limit=200)[0] for i in range(15)])
    vol = 4 * np.pi / 3 * (t["r"][1:] ** 3 - t["r"][:-1] ** 3)
    rho_ref = A * (4 * np.pi * I / vol) / (4 * np.pi * I.sum())
    assert np.allclose(t["rho"], rho_ref, rtol=1e-12, atol=0)
    assert (vol * t["rho"]).sum() == pytest.approx(A, rel=1e-13)
    assert np.all(np.diff(t["rho"]) < 0)
    assert np.allclose(t["rho_s"][1] + t["rho_s"][0], t["rho"], rtol=1e-15)
    assert np.allclose(t["rho_s"][1] / t["rho"], Z / A, rtol=1e-15)


def test_saturation_density_and_well_depth():
    # heavy nuclei: central density near nuclear saturation (0.16 fm^-3; c = 1.07 A^1/3 is a
    # slightly small half-density radius, so up to ~0.19), Fermi energy 25-45 MeV, well depth
    # 40-55 MeV (textbook Fermi-gas values)
    t = oracle.target(82, 208)
    assert 0.14 < t["rho"][0] < 0.19
    assert 25 < t["EF"][0][0] < 45 and 20 < t["EF"][1][0] < 40
    assert 35 < t["V"][0][0] < 55 and 30 < t["V"][1][0] < 55
    # Coulomb barrier of lead for protons, ~13 MeV
    assert 11 < t["EC"] < 15


def test_fermi_momentum_and_energy_relation():
    # number density of one spin-1/2 species filled to p_F: rho = p_F^3 / (3 pi^2 (hbar c)^3);
    # E_F is the relativistic kinetic energy at p_F
    t = oracle.target(20, 40)
    for s, m in ((0, oracle.M_N), (1, oracle.M_P)):
        pf = t["pF"][s]
        n_from_pf = pf**3 / (3 * np.pi**2 * HBARC**3)
        assert np.allclose(n_from_pf, t["rho_s"][s], rtol=1e-13)
        assert np.allclose(t["EF"][s], np.hypot(pf, m) - m, rtol=1e-12)
        assert np.allclose(t["V"][s], t["EF"][s] + t["S"][s], rtol=1e-15)
    v = np.maximum(t["pF"][0] / np.hypot(t["pF"][0], oracle.M_N), t["pF"][1] / np.hypot(t["pF"][1], oracle.M_P))
    assert np.allclose(t["vF"], v, rtol=1e-15)


def test_unsupported_targets_rejected():
    for Z, A in [(1, 2), (2, 4), (0, 10), (5, 6), (101, 260)]:
        with pytest.raises(ValueError):
            oracle.target(Z, A)
