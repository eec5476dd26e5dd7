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


def compare(gpu_res, gpu_sec, orc, n):
    """Returns dict: fraction of events whose integer outcomes all agree, and the worst
    relative energy difference over those events."""
    ores, osec = orc["residuals"], orc["secondaries"]
    same = np.ones(n, bool)
    for g, o in INT_FIELDS:
        same &= gpu_res[g].astype(np.int64) == ores[o].astype(np.int64)
    gs = pnuc.sort_secondaries(gpu_sec)
    sig_g = species_signature(gs, n)
    sig_o = species_signature(osec, n)
    same &= np.array([a == b for a, b in zip(sig_g, sig_o)])
    # energies of the events that agree
    ok_ev = np.where(same)[0]
    mask_g = np.isin(gs["event"], ok_ev)
    mask_o = np.isin(osec["event"], ok_ev)
    Tg, To = gs["T"][mask_g], osec["T"][mask_o]
    assert len(Tg) == len(To)
    rel_T = np.abs(Tg - To) / np.maximum(np.abs(To), 1e-300)
    dir_err = 0.0
    if len(Tg):
        dg = np.stack([gs["ux"][mask_g], gs["uy"][mask_g], gs["uz"][mask_g]], 1).astype(np.float64)
        do = np.stack([osec["ux"][mask_o], osec["uy"][mask_o], osec["uz"][mask_o]], 1)
        dir_err = float(np.abs(dg - do).max())
    Eg = np.concatenate([gpu_res["Estar_cascade"][ok_ev], gpu_res["Estar_final"][ok_ev]])
    Eo = np.concatenate([ores["Estar_c"][ok_ev], ores["Estar_f"][ok_ev]])
    scale = np.maximum(np.abs(Eo), 1.0)  # E* near 0: compare on the MeV scale
    rel_E = np.abs(Eg - Eo) / scale
    return dict(frac_same=float(same.mean()), same=same,
                max_rel_T=float(rel_T.max()) if len(rel_T) else 0.0,
                max_rel_Estar=float(rel_E.max()) if len(rel_E) else 0.0, max_dir_err=dir_err)
