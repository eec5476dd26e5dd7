"""The FP32 bin decision of the yield tallies (csrc/tally.cu, bin_of and bin_map) restated in
numpy float32 and checked by brute force against the FP64 definition of the bins
(floor(RN(RN(x - x0) * s)), the definition oracle/tally.py writes out): values on and a few
ulps around every bin edge, random values, zeros, subnormals, infinities and NaN, for maps
with odd ranges and offsets. The decision must agree everywhere; with the error bound taken
64 times too small it must not (the check can see an undersized bound)."""
import numpy as np

f32 = np.float32


def round_up_f32(v):
    with np.errstate(over="ignore"):
        f = f32(v)
    return np.nextafter(f, f32(np.inf)) if float(f) < v else f


def bin_map(x0, s, n, shrink=1.0):
    m = dict(x0=x0, s=s, n=n, x0f=f32(x0), sf=f32(s), errs=f32(round_up_f32(s * 2.0 ** -20) * shrink),
             abs_err=f32(max(round_up_f32(s * 2.0 ** -120), f32(2.0 ** -126)) * shrink))
    m["fast"] = bool(np.isfinite(m["x0f"]) and np.isfinite(m["sf"]) and np.isfinite(m["errs"])
                     and m["sf"] >= f32(2.0 ** -100) and n < (1 << 24) and (x0 == 0.0 or abs(x0) >= 2.0 ** -100))
    return m


def floor_bits(t):
    """The kernel's floor: -1 below zero (-0 is 0), INT_MAX from 2^31, for NaN and infinities."""
    with np.errstate(invalid="ignore"):
        out = np.floor(np.where(np.isfinite(t), t, 0.0)).astype(np.int64)
        out = np.where(np.isnan(t) | (t >= 2.0 ** 31), 2 ** 31 - 1, out)
        return np.where(t < 0, -1, out)


def exact(x, m):
    with np.errstate(all="ignore"):
        return floor_bits((x - m["x0"]) * m["s"])


def decided(xf, x, m):
    """bin_of: every float32 operation rounded to nearest, in the kernel's order"""
    with np.errstate(all="ignore"):
        t = (xf - m["x0f"]) * m["sf"]
        err = (np.abs(xf) + abs(m["x0f"])) * m["errs"] + m["abs_err"]
        assert t.dtype == np.float32 and err.dtype == np.float32
        f = np.floor(t)
        inner = ((t - f) > err) & (((f + f32(1)) - t) > err)
        out = np.where(inner, np.nan_to_num(f, posinf=0, neginf=0).astype(np.int64), -999)
        out = np.where((t - err) > f32(m["n"]), m["n"], out)
        out = np.where((t + err) < f32(0), -1, out)
    slow = out == -999
    out[slow] = exact(x[slow], m)
    return out


def in_range(b, n):
    return np.where(b < 0, -1, np.where(b >= n, n, b))


MAPS = [(0.0, 125 / 250.0, 125), (199.0, 0.5, 1), (150.0, 4 / 100.0, 4), (-1.0, 10.0, 20), (-1.0, 0.5, 1),
        (0.3, 113 / (217.7 - 0.3), 113), (20.0, 23 / 230.0, 23), (1e-3, 3e5, 1000), (-5.0, 1 / 3.0, 30),
        (1e6, 1e-3, 5000), (0.0, 1e30, 100), (0.0, 3e-30, 50), (-1e-20, 1e10, 77), (3.0, 16777215 / 10.0, 16777215)]


def points(rng, x0, s, n):
    ks = np.arange(-2, n + 3) if n < 5000 else np.concatenate([np.arange(-2, 2000), rng.integers(0, n, 2000),
                                                               np.arange(n - 2000, n + 3)])
    edges = x0 + ks / s
    e = np.repeat(edges, 16)
    k = np.tile(np.arange(-8, 8), len(edges)).astype(np.float64)
    hi = x0 + n / s
    return np.concatenate([rng.uniform(x0 - 1 / s, hi + 1 / s, 30000),
                           e + k * np.spacing(np.abs(e) + 1e-300) * rng.integers(1, 4, len(e)),
                           e * (1 + k * 2.0 ** -24),
                           np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-310, -1e-310, 1e-40, -1e-40, 1e-38, x0, hi,
                                     3.5e38, 1e300, -1e300]),
                           rng.standard_normal(5000) * 1e-30])


def to_f32(x, ftz):
    with np.errstate(over="ignore"):
        xf = x.astype(np.float32)
    if ftz:  # the kernel's double-to-float conversion flushes results below the normal range
        xf = np.where(np.abs(xf) < f32(2.0 ** -126), f32(0) * np.sign(xf), xf).astype(np.float32)
    return xf


def test_fp32_decision_equals_the_fp64_bins():
    rng = np.random.default_rng(3)
    for x0, s, n in MAPS:
        m = bin_map(x0, s, n)
        assert m["fast"], (x0, s, n)
        x = points(rng, x0, s, n)
        for ftz in (False, True):
            got = in_range(decided(to_f32(x, ftz), x, m), n)
            want = in_range(exact(x, m), n)
            bad = np.flatnonzero(got != want)
            assert bad.size == 0, (x0, s, n, ftz, x[bad[:4]], got[bad[:4]], want[bad[:4]])


def test_parameters_outside_the_bound_take_the_fp64_path():
    assert not bin_map(0.0, 1.0, 1 << 24)["fast"]      # n not exact in FP32
    assert not bin_map(1e-120, 1.0, 10)["fast"]        # x0 below the normal floats
    assert not bin_map(1e39, 1.0, 10)["fast"]          # x0 beyond them
    assert not bin_map(0.0, 1e-101, 10)["fast"]        # s too small
    assert not bin_map(0.0, 3e38 * 2 ** 21, 10)["fast"]  # s * 2^-20 overflows FP32


def test_an_undersized_bound_is_caught():
    rng = np.random.default_rng(4)
    bad = 0
    for x0, s, n in MAPS[:6]:
        m = bin_map(x0, s, n, shrink=1 / 64)
        x = points(rng, x0, s, n)
        bad += int((in_range(decided(to_f32(x, False), x, m), n) != in_range(exact(x, m), n)).sum())
    assert bad > 0
