"""Reference yield tallies (test infrastructure, like the rest of oracle/): the histograms
that pnuc_tally defines, written out with numpy from their definition (bin index =
floor((x - lo) * (n / (hi - lo))) in FP64, cos theta bins floor((uz + 1) * (n / 2)) capped
at n - 1) over records in the library's output layout or the oracle's."""
import numpy as np

BAD = 1 | 2  # bad input, attempt cap: no non-elastic event


def secondary_hist(T, uz, species, origin, T_range, n_T, n_cos):
    T = np.asarray(T, np.float64)
    t = (T - T_range[0]) * (float(n_T) / (T_range[1] - T_range[0]))
    keep = (t >= 0.0) & (t < n_T)
    c = (np.asarray(uz, np.float32).astype(np.float64) + 1.0) * (0.5 * n_cos)
    ic = np.minimum(np.maximum(np.floor(c), 0), n_cos - 1).astype(np.int64)
    idx = ((np.asarray(origin, np.int64) * 6 + np.asarray(species, np.int64)) * n_cos + ic) * n_T
    idx = idx[keep] + np.floor(t[keep]).astype(np.int64)
    return np.bincount(idx, minlength=12 * n_cos * n_T).reshape(2, 6, n_cos, n_T)


def secondary_window_hist(T, uz, species, origin, T_range, n_T, cos_lo, cos_hi):
    """pnuc_tally_windows (the spectra at fixed angles of the paper's Fig. 2, §4.1): window k
    holds the records with cos_lo[k] <= uz < cos_hi[k] (uz as
    its float value, compared in FP64 with the edges), T bins as in secondary_hist; histogram
    [2][6][len(cos_lo)][n_T]; records in no window or outside the T range are not counted."""
    T = np.asarray(T, np.float64)
    t = (T - T_range[0]) * (float(n_T) / (T_range[1] - T_range[0]))
    u = np.asarray(uz, np.float32).astype(np.float64)
    kw = len(cos_lo)
    win = np.full(len(u), -1, np.int64)
    for k in range(kw):
        win[(win < 0) & (u >= cos_lo[k]) & (u < cos_hi[k])] = k
    keep = (t >= 0.0) & (t < n_T) & (win >= 0)
    idx = ((np.asarray(origin, np.int64) * 6 + np.asarray(species, np.int64)) * kw + win) * n_T
    idx = idx[keep] + np.floor(t[keep]).astype(np.int64)
    return np.bincount(idx, minlength=12 * kw * n_T).reshape(2, 6, kw, n_T)


def residual_hist(Z, A, flags, energies, E_range, n_E, Z_max, A_max):
    E = np.asarray(energies, np.float64)
    e = (E - E_range[0]) * (float(n_E) / (E_range[1] - E_range[0]))
    Z = np.asarray(Z, np.int64)
    A = np.asarray(A, np.int64)
    keep = ((np.asarray(flags, np.int64) & BAD) == 0) & (e >= 0.0) & (e < n_E) & (Z <= Z_max) & (A <= A_max)
    idx = (np.floor(e[keep]).astype(np.int64) * (Z_max + 1) + Z[keep]) * (A_max + 1) + A[keep]
    return np.bincount(idx, minlength=n_E * (Z_max + 1) * (A_max + 1)).reshape(n_E, Z_max + 1, A_max + 1)
