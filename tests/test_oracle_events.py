"""Whole-event pins of the oracle (§2.1-2.4): per-event conservation of baryon number,
charge and energy, momentum in the evaporation, Pauli / cutoff / Coulomb-barrier invariants
from the decision trace, a hand-traced central event, determinism by event id."""
import numpy as np
import pytest

import oracle
from paper_1309_7963_gb300 import inputs

ZA_EJ = np.array(oracle.EJECTILE_ZA)
M_EJ = np.array(oracle.EJECTILE_MASS)
K = oracle.TRACE_KINDS


def _run(za, energy, n, seed=0, **kw):
    if np.isscalar(energy):
        energy = np.full(n, float(energy))
    return oracle.simulate([za], energy, np.zeros(n, np.int32), seed=seed, **kw)


@pytest.mark.parametrize("proj", [1, 0], ids=["proton", "neutron"])
@pytest.mark.parametrize("za,energy", [((8, 16), 200.0), ((20, 40), 70.0), ((82, 208), 150.0), ((6, 12), 25.0)])
def test_conservation_per_event(za, energy, proj):
    """Per event, for proton- and neutron-induced events: baryon number and charge, energy,
    the cascade's momentum against the static field, evaporation momentum, mass shell."""
    Z, A = za
    m_proj = oracle.M_P if proj else oracle.M_N
    r = _run(za, energy, 1500, projectiles=np.full(1500, proj))
    sec, res = r["secondaries"], r["residuals"]
    ok = (res["flags"] & ~np.uint32(32 | 16)) == 0
    ev = sec["event"]
    sa = np.bincount(ev, weights=ZA_EJ[sec["species"], 1], minlength=len(res))
    sz = np.bincount(ev, weights=ZA_EJ[sec["species"], 0], minlength=len(res))
    assert np.all(sa[ok] + res["Af"][ok] == A + 1)
    assert np.all(sz[ok] + res["Zf"][ok] == Z + proj)
    Ein = energy + m_proj + oracle.semf_mass(Z, A)
    Eout = np.bincount(ev, weights=sec["T"] + M_EJ[sec["species"]], minlength=len(res)) + res["Ef"]
    assert np.allclose(Eout[ok], Ein, rtol=1e-12, atol=0)
    # momentum: the cascade's imbalance goes to the static field, the evaporation conserves it
    p0 = np.sqrt(energy ** 2 + 2 * energy * m_proj)
    casc = sec["origin"] == 0
    for k, comp in enumerate(("px", "py", "pz")):
        pc = np.bincount(ev[casc], weights=sec[comp][casc], minlength=len(res))
        pe = np.bincount(ev[~casc], weights=sec[comp][~casc], minlength=len(res))
        want = p0 if comp == "pz" else 0.0
        assert np.allclose((pc + res["Pcas"][:, k])[ok], want, atol=1e-8)
        assert np.allclose((pe + res["Pf"][:, k])[ok], 0.0, atol=1e-8)
    # the final residual sits on its mass shell: invariant mass = M(Zf, Af) + E*_f
    evap = ok & (res["n_evap"] > 0)
    inv = np.sqrt(res["Ef"] ** 2 - (res["Pf"] ** 2).sum(1))
    Mf = np.array([oracle.semf_mass(z, a) for z, a in zip(res["Zf"], res["Af"])])
    assert np.allclose(inv[evap], (Mf + res["Estar_f"])[evap], rtol=1e-12)
    # no error flags; E* <= 0 (flag 32: the cascade holds the target's separation energies,
    # so e.g. a (p,n) exchange into 12N binds the captured proton too strongly) stays rare
    assert np.all((res["flags"] & ~np.uint32(32)) == 0)
    assert np.mean(res["flags"] != 0) < 0.08


def test_pauli_cutoff_and_coulomb_invariants_from_trace():
    za = (20, 40)
    t = oracle.target(*za)
    r = _run(za, 120.0, 400, trace=True, trace_cap=1 << 22)
    tr = r["trace"]
    assert r["trace_total"] == len(tr)
    kinds = tr["kind"]
    # every accepted collision is followed by its two products, both above their Fermi energy
    idx = np.where(kinds == K["collision"])[0]
    assert len(idx) > 100
    for i in idx:
        for j in (i + 1, i + 2):
            e = tr[j]
            assert e["kind"] == K["product"]
            assert e["T"] > t["EF"][e["species"]][e["shell"]]
    # captures after collisions are below the cutoff V (+E_C for protons) of their shell
    cap = tr[kinds == K["capture"]]
    cut = t["V"][cap["species"], cap["shell"]] + np.where(cap["species"] == 1, t["EC"], 0.0)
    assert np.all(cap["T"] < cut)
    # escaped secondaries: protons left with at least the Coulomb barrier, neutrons with T >= 0
    sec = r["secondaries"]
    c = sec[sec["origin"] == 0]
    assert np.all(c["T"][c["species"] == 1] >= t["EC"] * (1 - 1e-9))
    assert np.all(c["T"][c["species"] == 0] >= 0)
    # evaporation: charged ejectiles above their barrier, every emission energetically open
    ev = tr[kinds == K["evap"]]
    assert len(ev) > 100
    eps, V, Q, Es = ev["T"], ev["x"], ev["y"], ev["z"]
    assert np.all(eps >= V - 1e-9)
    assert np.all(Es >= Q + V)
    assert np.all(eps <= Es - Q + 1e-9)


def test_hand_traced_central_event_without_collision():
    # injected draws: b ~ 0 (central), then path draws that always exceed the chord, so the
    # incident proton crosses all 29 shell boundaries along the z axis and leaves with T0
    za, T0 = (8, 16), 150.0
    t = oracle.target(*za)
    inject = [1e-30, 0.25] + [2.0 ** -53] * 29
    r = _run(za, T0, 1, inject=inject, trace=True)
    tr = r["trace"]
    first = tr[: np.where(tr["kind"] == K["escape"])[0][0] + 1]
    assert first[0]["kind"] == K["entry"]
    assert first[0]["T"] == pytest.approx(T0 + t["V"][1][14], rel=1e-12)
    shells = list(range(13, -1, -1)) + list(range(1, 15))
    refr = first[first["kind"] == K["refract"]]
    assert list(refr["shell"]) == shells
    assert np.allclose(refr["T"], T0 + t["V"][1][shells], rtol=1e-12)
    assert first[-1]["T"] == pytest.approx(T0, rel=1e-12)
    # along the axis: x = y = 0, |z| at each crossing equals the shell radius
    assert np.allclose(refr["x"], 0, atol=1e-12) and np.allclose(refr["y"], 0, atol=1e-12)
    radii = np.concatenate([t["r"][14:0:-1], t["r"][1:15]])
    assert np.allclose(np.abs(refr["z"]), radii, rtol=1e-12)
    # that attempt was elastic, so the event went on with a new entry and ended non-elastic
    assert r["residuals"][0]["n_attempts"] >= 2 and r["residuals"][0]["n_coll"] >= 1


def test_events_depend_only_on_seed_and_event_id():
    w = inputs.mixed(300, seed=5)
    a = oracle.simulate(w.targets, w.energies, w.tidx, seed=5)
    b = oracle.simulate(w.targets, w.energies[120:], w.tidx[120:], seed=5, first_event_id=120)
    sa = a["secondaries"][a["secondaries"]["event"] >= 120]
    sb = b["secondaries"]
    assert len(sa) == len(sb)
    assert np.array_equal(sa["T"], sb["T"]) and np.array_equal(sa["event"] - 120, sb["event"])
    assert np.array_equal(a["residuals"][120:], b["residuals"])
    p = oracle.simulate_parallel(w.targets, w.energies, w.tidx, seed=5, chunk=64, threads=4)
    assert np.array_equal(p["residuals"], a["residuals"])
    assert np.array_equal(p["secondaries"], a["secondaries"])


def test_secondary_order_and_bad_inputs():
    r = oracle.simulate([(8, 16)], np.array([200.0, 10.0, 300.0, 100.0]), np.array([0, 0, 0, 3], np.int32), seed=0)
    res, sec = r["residuals"], r["secondaries"]
    assert res["flags"][1] == 1 and res["flags"][2] == 1 and res["flags"][3] == 1
    assert set(sec["event"]) == {0}
    s0 = sec[sec["event"] == 0]
    assert list(s0["index"]) == list(range(len(s0)))
    assert np.all(np.diff(s0["origin"]) >= 0)
    assert res["n_casc"][0] + res["n_evap"][0] == len(s0)


def test_neutron_entry_and_residual_charge_from_trace():
    """A neutron enters through the neutron well of the surface shell: its entry record is
    species 0 with kinetic energy T0 + V_n (refraction into the well at fixed tangential
    momentum), and the residual charge after the cascade counts only escaped protons."""
    za = (8, 16)
    t = oracle.target(*za)
    n = 300
    r = _run(za, 60.0, n, trace=True, projectiles=np.zeros(n, np.int32))
    tr = r["trace"]
    ent = tr[tr["kind"] == K["entry"]]
    assert len(ent) >= n and np.all(ent["species"] == 0)
    assert np.allclose(ent["T"], 60.0 + t["V"][0][14], rtol=1e-12)
    res, sec = r["residuals"], r["secondaries"]
    ok = (res["flags"] & ~np.uint32(32 | 16)) == 0
    nps = np.bincount(sec["event"][(sec["species"] == 1) & (sec["origin"] == 0)], minlength=n)
    assert np.all((res["Zc"] == 8 - nps)[ok])
    # the same events as protons differ: the projectile species enters the stream of decisions
    rp = _run(za, 60.0, n, projectiles=np.ones(n, np.int32))
    assert not np.array_equal(rp["residuals"]["Zc"], res["Zc"])


def test_heavy_target_events_never_reach_the_step_cap():
    """Specular reflections at the shell boundaries (reading M11, no floor): no event of a
    p-208Pb sample (the heavy target with the most surface reflections) runs to the 1e5-step
    cap, and the longest stays within a few thousand steps."""
    w = inputs.heavy(inputs.PB208, 3000, seed=3)
    r = oracle.simulate(w.targets, w.energies, w.tidx, seed=w.seed)
    assert (r["residuals"]["flags"] & 4).sum() == 0
    worst = 0
    for i in range(0, 3000, 10):  # per-event step counts on every tenth event
        c = oracle.simulate(w.targets, w.energies[i:i + 1], w.tidx[i:i + 1], seed=w.seed, first_event_id=i)
        worst = max(worst, int(c["counters"]["steps"]))
    assert worst < 5000
