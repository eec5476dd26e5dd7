"""Pins of the oracle's collision kinematics (§2.3, relativistic two-body), angular
sampling, boundary geometry and refraction (after Chen et al.), and Fermi-sphere sampling
(§2.2: momentum density proportional to p^2)."""
import numpy as np
import pytest
from scipy import stats

import oracle

MP, MN = oracle.M_P, oracle.M_N
mass = {0: MN, 1: MP}


def four(p, m):
    p = np.asarray(p, float)
    return np.array([np.sqrt(p @ p + m * m), *p])


def lorentz_to_rest_of(P):
    """Boost matrix into the rest frame of four-vector P (independent construction)."""
    E, p = P[0], P[1:]
    M = np.sqrt(E * E - p @ p)
    b = p / E
    g = E / M
    b2 = b @ b
    L = np.eye(4)
    L[0, 0] = g
    L[0, 1:] = L[1:, 0] = -g * b
    if b2 > 0:
        L[1:, 1:] += (g - 1) * np.outer(b, b) / b2
    return L


def test_cos_theta_isotropic_when_slope_zero():
    u = np.linspace(0.001, 0.999, 999)
    assert np.allclose([oracle.cos_theta(0.0, 0.3, x) for x in u], 1 - 2 * u, rtol=0, atol=1e-15)


@pytest.mark.parametrize("B,pst", [(1.0, 0.3), (5.5, 0.5), (16.5, 0.25), (5.0, 0.05)])
def test_cos_theta_follows_truncated_exponential(B, pst):
    # -t = 2 p*^2 (1 - cos) is exponential with rate B truncated to [0, 4 p*^2]
    L = 4 * pst * pst
    u = (np.arange(20000) + 0.5) / 20000
    x = np.array([2 * pst * pst * (1 - oracle.cos_theta(B, pst, v)) for v in u])
    mean_ref = 1 / B - L * np.exp(-B * L) / (1 - np.exp(-B * L))
    assert x.mean() == pytest.approx(mean_ref, rel=1e-6)
    cdf = (1 - np.exp(-B * x)) / (1 - np.exp(-B * L))
    assert np.allclose(cdf, u, atol=1e-9)


def test_rotation_preserves_angle_and_covers_azimuth():
    rng = np.random.default_rng(0)
    for _ in range(50):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        ct = rng.uniform(-1, 1)
        ds = np.array([oracle.rotate(n, ct, ph) for ph in np.linspace(0, 2 * np.pi, 64, endpoint=False)])
        assert np.allclose(np.linalg.norm(ds, axis=1), 1, atol=1e-14)
        assert np.allclose(ds @ n, ct, atol=1e-14)
        assert np.allclose(ds.mean(0), ct * n, atol=1e-13)
    # the pole case
    d = oracle.rotate([0, 0, -1], 0.3, 1.0)
    assert d[2] == pytest.approx(-0.3)


@pytest.mark.parametrize("s1,s2", [(1, 1), (1, 0), (0, 1), (0, 0)])
def test_collision_conserves_four_momentum_and_sets_cm_angle(s1, s2):
    rng = np.random.default_rng(s1 * 2 + s2)
    for _ in range(200):
        p1 = rng.normal(size=3) * rng.uniform(100, 800)
        p2 = rng.normal(size=3) * rng.uniform(0, 180)
        ut, uph, uf = rng.random(3)
        q1, q2 = oracle.collide(s1, p1, s2, p2, ut, uph, uf)
        m1, m2 = mass[s1], mass[s2]
        Pin = four(p1, m1) + four(p2, m2)
        Pout = four(q1, m1) + four(q2, m2)
        assert np.allclose(Pout, Pin, rtol=1e-12, atol=1e-9)
        # angle in the CM frame, from an independent boost construction
        L = lorentz_to_rest_of(Pin)
        a, b = (L @ four(p1, m1))[1:], (L @ four(q1, m1))[1:]
        assert np.linalg.norm(b) == pytest.approx(np.linalg.norm(a), rel=1e-10)
        cos_cm = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
        s = Pin[0] ** 2 - Pin[1:] @ Pin[1:]
        pst = np.linalg.norm(a) * 1e-3
        k = np.sqrt(((s - (m1 + m2) ** 2) * (s - (m1 - m2) ** 2))) / (2 * np.sqrt(s)) * 1e-3
        assert pst == pytest.approx(k, rel=1e-9)
        plab = np.sqrt(s) * k / m2
        ct = oracle.cos_theta(oracle.slope(s1 == s2, plab), pst, ut)
        if s1 != s2:
            a_b = oracle.backward_a(plab)
            if uf < a_b / (1 + a_b):
                ct = -ct
        assert cos_cm == pytest.approx(ct, abs=1e-9)


def test_boundary_distance_lands_on_the_shell_surface():
    t = oracle.target(20, 40)
    rng = np.random.default_rng(5)
    for _ in range(400):
        i = int(rng.integers(0, 15))
        rad = rng.uniform(t["r"][i], t["r"][i + 1])
        r = rng.normal(size=3)
        r *= rad / np.linalg.norm(r)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        s, direction = oracle.boundary_distance(t, i, r, d)
        end = r + s * d
        target_r = t["r"][i + 1] if direction > 0 else t["r"][i]
        assert np.linalg.norm(end) == pytest.approx(target_r, rel=1e-12, abs=1e-12)
        # brute-force march: the chord stays inside shell i before it ends
        lam = np.linspace(0, 1, 201)[1:-1]
        rr = np.linalg.norm(r[None, :] + (lam * s)[:, None] * d[None, :], axis=1)
        assert np.all(rr >= t["r"][i] - 1e-9) and np.all(rr <= t["r"][i + 1] + 1e-9)


def test_refraction_keeps_tangential_momentum_and_shifts_energy():
    """Chen et al.'s potential step (§2.3): the tangential momentum is kept; a refraction
    changes the kinetic energy by exactly dT, its normal component taking the sign of the
    crossing; a reflection, exactly when the new normal momentum squared would be <= 0 (or
    T + dT <= 0), is specular."""
    rng = np.random.default_rng(9)
    n_reflect = 0
    for _ in range(2000):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        p = rng.normal(size=3) * rng.uniform(50, 600)
        m = MP
        dT = rng.uniform(-60, 60)
        T = np.hypot(np.linalg.norm(p), m) - m
        ok, q = oracle.refract(n, p, m, dT)
        sgn = 1.0 if p @ n >= 0 else -1.0
        pt = p - (p @ n) * n
        qt = q - (q @ n) * n
        assert np.allclose(qt, pt, atol=1e-9)  # the tangential momentum is always kept
        Tq = np.hypot(np.linalg.norm(q), m) - m
        qn2 = (p @ n) ** 2 + dT * (2 * T + dT + 2 * m)
        if ok:
            assert T + dT > 0 and qn2 > 0
            assert sgn * (q @ n) > 0  # (the crossings here go the way p points along n)
            assert (q @ n) ** 2 == pytest.approx(qn2, rel=1e-10, abs=1e-9)
            assert Tq == pytest.approx(T + dT, rel=1e-10, abs=1e-9)
        else:
            n_reflect += 1
            assert T + dT <= 0 or qn2 <= 0
            assert np.allclose(q, p - 2 * (p @ n) * n, atol=1e-9)
    assert 0 < n_reflect < 2000


def test_grazing_reflection_is_specular():
    """Reading M11 in the model (FP64): no floor on the normal momentum; a reflection at
    grazing incidence reverses the normal component exactly, however small, and keeps the
    tangential momentum; an exactly tangent momentum is unchanged."""
    n = np.array([0.0, 0.0, 1.0])
    for eps, direction in ((1e-6, 1), (0.0, 1), (-1e-7, 1), (1e-6, -1)):
        p = np.array([300.0, 40.0, eps * 300.0 * direction])
        ok, q = oracle.refract(n, p, MP, -500.0, direction)  # dT far below -T: reflection
        assert not ok
        assert q[:2] == pytest.approx(p[:2], rel=1e-15)
        assert q[2] == -p[2]


def test_fermi_sphere_sampling_moments_and_ks():
    pF = 250.0
    q = oracle.sample_fermi(pF, 200000, seed=1, event=2)
    r = np.linalg.norm(q, axis=1)
    assert r.max() <= pF
    assert r.mean() == pytest.approx(0.75 * pF, rel=3e-3)
    assert (r * r).mean() == pytest.approx(0.6 * pF * pF, rel=4e-3)
    assert stats.kstest((r / pF) ** 3, "uniform").pvalue > 0.01
    u = q / r[:, None]
    assert np.all(np.abs(u.mean(0)) < 0.01)
    assert np.allclose((u * u).mean(0), 1 / 3, atol=0.005)
