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


SPECIES = ("n", "p", "d", "t", "3He", "alpha")
FIG2_ANGLES = (7.5, 30.0, 60.0, 150.0)  # degrees: the paper's double-differential spectra (Fig. 2)


def chi2_p(a, b, edges):
    """Two-sample chi-square p-value of two binned samples of equal size (bins with > 10
    entries in the pair); 1.0 when fewer than two such bins."""
    from scipy import stats
    ha, _ = np.histogram(a, edges)
    hb, _ = np.histogram(b, edges)
    keep = (ha + hb) > 10
    if keep.sum() < 2:
        return 1.0
    chi2 = (((ha[keep] - hb[keep]) ** 2) / (ha[keep] + hb[keep])).sum()
    return float(stats.chi2.sf(chi2, keep.sum() - 1))


def observable_table(gres, gsec, ores, osec, n):
    """Per-observable comparison of GPU results (FP32 mode) with the oracle on the same n
    events: mean multiplicity per species and origin (difference in standard errors),
    kinetic-energy spectra (2 MeV bins) and cos(theta) spectra (0.05 bins), the spectra in 1
    degree windows at the angles of the paper's Fig. 2, the residual (Z, A) distribution after
    evaporation, and the mean E* after the cascade; per species and origin also the mean
    kinetic energy (difference in standard errors) and two-sample Kolmogorov-Smirnov p-values
    of the unbinned kinetic energies and cos(theta). Returns the table row."""
    from scipy import stats
    row = {"events": int(n), "multiplicity": {}, "spectra_p": {}, "angle_p": {}, "fig2_p": {}, "mean_T": {},
           "ks_T_p": {}, "ks_cos_p": {}}
    for origin, label in ((0, "cascade"), (1, "evaporated")):
        for sp, sname in enumerate(SPECIES):
            gm_sel = (gsec["species"] == sp) & (gsec["origin"] == origin)
            om_sel = (osec["species"] == sp) & (osec["origin"] == origin)
            om = np.bincount(osec["event"][om_sel], minlength=n)
            if om.sum() < 50:
                continue
            gm = np.bincount(gsec["event"][gm_sel], minlength=n)
            se = np.sqrt(om.var() / n + gm.var() / n)
            z = (gm.mean() - om.mean()) / se if se > 0 else 0.0
            key = f"{label} {sname}"
            row["multiplicity"][key] = {"fp32": float(gm.mean()), "oracle": float(om.mean()), "z": float(z)}
            row["spectra_p"][key] = chi2_p(gsec["T"][gm_sel], osec["T"][om_sel], np.linspace(0, 250, 126))
            row["angle_p"][key] = chi2_p(gsec["uz"][gm_sel], osec["uz"][om_sel], np.linspace(-1, 1, 41))
            gT, oT = gsec["T"][gm_sel].astype(np.float64), osec["T"][om_sel].astype(np.float64)
            se_T = np.sqrt(gT.var() / len(gT) + oT.var() / len(oT))
            row["mean_T"][key] = {"fp32": float(gT.mean()), "oracle": float(oT.mean()),
                                  "z": float((gT.mean() - oT.mean()) / se_T) if se_T > 0 else 0.0}
            row["ks_T_p"][key] = float(stats.ks_2samp(gT, oT, method="asymp").pvalue)
            row["ks_cos_p"][key] = float(stats.ks_2samp(gsec["uz"][gm_sel].astype(np.float64),
                                                        osec["uz"][om_sel].astype(np.float64), method="asymp").pvalue)
            if origin == 0 or sp > 1:
                continue
            for ang in FIG2_ANGLES:  # evaporated n and p in 1-degree windows
                lo, hi = np.cos(np.radians(ang + 0.5)), np.cos(np.radians(ang - 0.5))
                gw = gm_sel & (gsec["uz"] >= lo) & (gsec["uz"] < hi)
                ow = om_sel & (osec["uz"] >= lo) & (osec["uz"] < hi)
                row["fig2_p"][f"{key} {ang:g} deg"] = chi2_p(gsec["T"][gw], osec["T"][ow], np.linspace(0, 60, 31))
    # residual (Z, A) after evaporation: two-sample chi-square over the occupied cells
    gk = gres["Z_final"].astype(np.int64) * 1000 + gres["A_final"].astype(np.int64)
    ok = ores["Zf"].astype(np.int64) * 1000 + ores["Af"].astype(np.int64)
    cells, inv = np.unique(np.concatenate([gk, ok]), return_inverse=True)
    hg = np.bincount(inv[:n], minlength=len(cells))
    ho = np.bincount(inv[n:], minlength=len(cells))
    keep = (hg + ho) > 10
    chi2 = (((hg[keep] - ho[keep]) ** 2) / (hg[keep] + ho[keep])).sum()
    row["residual_ZA_p"] = float(stats.chi2.sf(chi2, max(keep.sum() - 1, 1))) if keep.sum() > 1 else 1.0
    row["residual_ZA_identical"] = float(np.mean(gk == ok))
    good = (ores["flags"] & 48) == 0
    row["mean_Estar_cascade"] = {"fp32": float(gres["Estar_cascade"][good].mean()),
                                 "oracle": float(ores["Estar_c"][good].mean())}
    return row


def assert_observables(row, name):
    """The bounds: multiplicities and mean kinetic energies within 3 standard errors,
    chi-square and Kolmogorov-Smirnov p > 0.01."""
    for field in ("multiplicity", "mean_T"):
        for k, v in row[field].items():
            assert abs(v["z"]) < 3.0, (name, field, k, v)
    for field in ("spectra_p", "angle_p", "fig2_p", "ks_T_p", "ks_cos_p"):
        for k, p in row[field].items():
            assert p > 0.01, (name, field, k, p)
    assert row["residual_ZA_p"] > 0.01, (name, row["residual_ZA_p"])
