"""The reference yield tallies (oracle/tally.py) against a brute-force loop over records and
hand-placed values at the bin edges."""
import math

import numpy as np

from oracle import tally


def brute_secondary(T, uz, sp, org, lo, hi, n_T, n_cos):
    h = np.zeros((2, 6, n_cos, n_T), np.int64)
    s = n_T / (hi - lo)
    for t, u, a, o in zip(T, uz, sp, org):
        x = (t - lo) * s
        if not (0.0 <= x < n_T):
            continue
        c = (float(np.float32(u)) + 1.0) * (0.5 * n_cos)
        ic = min(max(math.floor(c), 0), n_cos - 1)
        h[o, a, ic, math.floor(x)] += 1
    return h


def test_secondary_hist_matches_brute_force_and_edges():
    rng = np.random.default_rng(3)
    n = 3000
    T = rng.uniform(-5, 260, n)
    uz = rng.uniform(-1, 1, n).astype(np.float32)
    sp = rng.integers(0, 6, n)
    org = rng.integers(0, 2, n)
    # bin edges and the ends of the ranges
    T[:6] = [0.0, 2.0, 249.999999, 250.0, -1e-12, 124.0]
    uz[:6] = [-1.0, 1.0, 0.0, 0.5, -0.999, 1.0]
    for n_T, n_cos in ((125, 1), (50, 40), (7, 3)):
        got = tally.secondary_hist(T, uz, sp, org, (0.0, 250.0), n_T, n_cos)
        assert np.array_equal(got, brute_secondary(T, uz, sp, org, 0.0, 250.0, n_T, n_cos))
    h = tally.secondary_hist([0.0, 250.0, 2.0], [1.0, 0.0, -1.0], [0, 0, 1], [0, 0, 1], (0.0, 250.0), 125, 40)
    assert h[0, 0, 39, 0] == 1 and h.sum() == 2 and h[1, 1, 0, 1] == 1  # uz = 1 -> last bin; T = 250 out


def test_window_hist_matches_brute_force_and_edges():
    rng = np.random.default_rng(5)
    n = 4000
    lo, hi = [0.99, 0.86, -0.2, -0.871], [0.9925, 0.871, 0.1, -0.86]
    T = rng.uniform(-5, 260, n)
    uz = rng.uniform(-1, 1, n).astype(np.float32)
    # values on and next to every edge (as floats), and the ends
    edges = np.array(lo + hi, np.float64)
    near = np.concatenate([np.nextafter(edges.astype(np.float32), np.float32(d)) for d in (-2, 2)] +
                          [edges.astype(np.float32)])
    uz[:len(near)] = near
    sp, org = rng.integers(0, 6, n), rng.integers(0, 2, n)
    got = tally.secondary_window_hist(T, uz, sp, org, (0.0, 250.0), 125, lo, hi)
    want = np.zeros((2, 6, 4, 125), np.int64)
    for t, u, a, o in zip(T, uz, sp, org):
        x = (t - 0.0) * (125 / 250.0)
        k = [j for j in range(4) if lo[j] <= float(u) < hi[j]]
        if 0.0 <= x < 125 and k:
            want[o, a, k[0], math.floor(x)] += 1
    assert np.array_equal(got, want)
    # a record on a lower edge counts, on an upper edge not
    h = tally.secondary_window_hist([10.0, 10.0], [np.float32(0.5), np.float32(0.75)], [0, 0], [0, 0], (0.0, 250.0),
                                    125, [0.5], [0.75])
    assert h.sum() == 1 and h[0, 0, 0, 5] == 1


def test_residual_hist_filters_and_bins():
    Z = np.array([8, 8, 6, 7, 100, 8])
    A = np.array([15, 15, 11, 13, 250, 15])
    flags = np.array([0, 1, 0, 32, 0, 2])
    E = np.array([200.0, 200.0, 20.0, 249.9, 120.0, 100.0])
    h = tally.residual_hist(Z, A, flags, E, (20.0, 250.0), 23, 99, 250)
    assert h.shape == (23, 100, 251)
    assert h.sum() == 3  # bad input and attempt cap dropped; Z = 100 > Z_max dropped
    assert h[18, 8, 15] == 1 and h[0, 6, 11] == 1 and h[22, 7, 13] == 1
