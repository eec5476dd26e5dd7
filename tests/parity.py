"""Per-event comparison of libpnuc outputs with the CPU oracle (used by the GPU tests)."""
import numpy as np

from paper_1309_7963_gb300 import pnuc

INT_FIELDS = [("Z_cascade", "Zc"), ("A_cascade", "Ac"), ("Z_final", "Zf"), ("A_final", "Af"),
              ("n_cascade", "n_casc"), ("n_evaporated", "n_evap"), ("n_collisions", "n_coll"),
              ("n_attempts", "n_attempts"), ("flags", "flags")]


def species_signature(sec, n):
    """Per event: tuple of (species, origin) in emission order."""
    s = pnuc.sort_secondaries(sec) if sec.dtype == pnuc.SECONDARY_DTYPE else sec
    out = [[] for _ in range(n)]
    for e, sp, o in zip(s["event"], s["species"], s["origin"]):
        out[int(e)].append((int(sp), int(o)))
    return [tuple(x) for x in out]


def compare(gpu_res, gpu_sec, orc, n, rel_tol=1e-9):
    """Per-event comparison. An event matches when its integer outcomes (residual Z/A after
    cascade and evaporation, multiplicities, collisions, attempts, flags, and the ordered
    (species, origin) list of its secondaries) are identical AND every energy (secondary
    kinetic energies, E* after the cascade and at the end) agrees within rel_tol relative
    (E* relative to max(|E*|, 1 MeV)). Returns the matching fraction and diagnostics."""
    ores, osec = orc["residuals"], orc["secondaries"]
    same = np.ones(n, bool)
    for g, o in INT_FIELDS:
        same &= gpu_res[g].astype(np.int64) == ores[o].astype(np.int64)
    gs = pnuc.sort_secondaries(gpu_sec)
    sig_g = species_signature(gs, n)
    sig_o = species_signature(osec, n)
    same &= np.array([a == b for a, b in zip(sig_g, sig_o)])
    ok_ev = np.where(same)[0]
    mask_g = np.isin(gs["event"], ok_ev)
    mask_o = np.isin(osec["event"], ok_ev)
    Tg, To = gs["T"][mask_g], osec["T"][mask_o]
    assert len(Tg) == len(To)
    ev_of = osec["event"][mask_o].astype(np.int64)
    rel_T = np.abs(Tg - To) / np.maximum(np.abs(To), 1e-300)
    worst = np.zeros(n)
    if len(rel_T):
        np.maximum.at(worst, ev_of, rel_T)
    scale_c = np.maximum(np.abs(ores["Estar_c"]), 1.0)
    scale_f = np.maximum(np.abs(ores["Estar_f"]), 1.0)
    rel_Ec = np.abs(gpu_res["Estar_cascade"] - ores["Estar_c"]) / scale_c
    rel_Ef = np.abs(gpu_res["Estar_final"] - ores["Estar_f"]) / scale_f
    worst = np.maximum(worst, np.maximum(rel_Ec, rel_Ef))
    match = same & (worst <= rel_tol)
    dir_err = 0.0
    if len(Tg):
        dg = np.stack([gs["ux"][mask_g], gs["uy"][mask_g], gs["uz"][mask_g]], 1).astype(np.float64)
        do = np.stack([osec["ux"][mask_o], osec["uy"][mask_o], osec["uz"][mask_o]], 1)
        dir_err = float(np.abs(dg - do).max())
    return dict(frac_match=float(match.mean()), frac_same=float(same.mean()), same=same, match=match,
                max_rel_energy_same=float(worst[same].max()) if same.any() else 0.0, max_dir_err=dir_err,
                worst=worst)


def oracle_at(w, ids):
    """Oracle results for the events ids (positions in workload w), one call per event;
    secondaries renumbered to positions 0..len(ids)-1."""
    import oracle
    res, secs = [], []
    for k, i in enumerate(ids):
        r = oracle.simulate(w.targets, w.energies[i:i + 1], w.tidx[i:i + 1], seed=w.seed,
                            first_event_id=w.first_event_id + int(i))
        s = r["secondaries"].copy()
        s["event"] = k
        res.append(r["residuals"])
        secs.append(s)
    return dict(residuals=np.concatenate(res), secondaries=np.concatenate(secs))


def gpu_subset(res, sec, ids):
    """GPU residuals of events ids and their secondaries renumbered to 0..len(ids)-1."""
    pos = {int(i): k for k, i in enumerate(ids)}
    keep = np.isin(sec["event"], ids)
    s = sec[keep].copy()
    s["event"] = [pos[int(e)] for e in s["event"]]
    return res[ids], s
