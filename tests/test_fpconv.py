"""The integer-pipe float<->double conversions of the FP32-mode kernels (csrc/fpconv.h),
compiled as host C++ and checked bit for bit against the CPU's IEEE-754 conversions (numpy):
random bit patterns over the whole normal range, exact ties, the rounding carry into the
exponent, overflow, zeros, infinities and NaN."""
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER_DIR = os.path.join(HERE, "..", "paper_1309_7963_gb300", "csrc")

DRIVER = r"""
#include <stdio.h>
#include <stdlib.h>
#include "fpconv.h"
int main(int argc, char **argv)
{
    FILE *fi = fopen(argv[2], "rb"), *fo = fopen(argv[3], "wb");
    if (!fi || !fo) return 1;
    if (argv[1][0] == 'd') {  // double -> float
        double x;
        while (fread(&x, 8, 1, fi) == 1) { float y = pnuc::d2f(x); fwrite(&y, 4, 1, fo); }
    } else {                  // float -> double
        float x;
        while (fread(&x, 4, 1, fi) == 1) { double y = pnuc::f2d(x); fwrite(&y, 8, 1, fo); }
    }
    fclose(fi);
    fclose(fo);
    return 0;
}
"""


@pytest.fixture(scope="module")
def conv(tmp_path_factory):
    d = tmp_path_factory.mktemp("fpconv")
    src = d / "drv.cpp"
    src.write_text(DRIVER)
    exe = d / "drv"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", HEADER_DIR, str(src), "-o", str(exe)], check=True)

    def run(mode, arr):
        fi, fo = d / "in.bin", d / "out.bin"
        arr.tofile(fi)
        subprocess.run([str(exe), mode, str(fi), str(fo)], check=True)
        return np.fromfile(fo, dtype=np.float32 if mode == "d" else np.float64)
    return run


def test_double_to_float_rounds_to_nearest_even(conv):
    rng = np.random.default_rng(1)
    n = 400_000
    # random doubles with float-range exponents, both signs
    bits = rng.integers(0, 2**52, n, dtype=np.uint64)
    exp = rng.integers(1023 - 126, 1023 + 128, n).astype(np.uint64)
    sign = rng.integers(0, 2, n).astype(np.uint64)
    x = ((sign << np.uint64(63)) | (exp << np.uint64(52)) | bits).view(np.float64)
    # exact ties and neighbours: dropped 29 bits = 0x10000000 and +-1, odd and even kept bits
    t = rng.integers(0, 2**23, 20_000, dtype=np.uint64) << np.uint64(29)
    texp = rng.integers(1023 - 126, 1023 + 127, 20_000).astype(np.uint64) << np.uint64(52)
    ties = np.concatenate([(texp | t | np.uint64(0x10000000 + k)) for k in (-1, 0, 1)]).view(np.float64)
    # mantissa all ones: the rounding carry moves into the exponent
    carry = ((texp | np.uint64((2**52 - 1))) ).view(np.float64)
    big = np.array([3.4028234663852886e38, 3.4028235677973366e38, 3.40282357e38, 1e39, -1e300, 1e308], np.float64)
    special = np.array([0.0, -0.0, np.inf, -np.inf, 1.0, -2.5, 1.1754943508222875e-38], np.float64)
    allx = np.concatenate([x, ties, carry, big, special])
    got = conv("d", allx)
    with np.errstate(over="ignore"):
        want = allx.astype(np.float32)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    nan = conv("d", np.array([np.nan, -np.nan], np.float64))
    assert np.isnan(nan).all()


def test_double_to_float_flushes_below_flt_min(conv):
    x = np.array([1e-39, -1e-40, 5e-324, 1e-300, 1.1754942e-38], np.float64)
    got = conv("d", x)
    assert np.all(got == 0.0) and np.array_equal(np.signbit(got), np.signbit(x))


def test_float_to_double_is_exact(conv):
    rng = np.random.default_rng(2)
    bits = rng.integers(0, 2**32, 400_000, dtype=np.uint64).astype(np.uint32)
    f = bits.view(np.float32)
    normal = (np.abs(f) >= np.float32(1.1754944e-38)) | (f == 0) | np.isinf(f)
    got = conv("f", f[normal])
    assert np.array_equal(got.view(np.uint64), f[normal].astype(np.float64).view(np.uint64))
    sub = conv("f", np.array([1e-40, -1e-41], np.float32))
    assert np.all(sub == 0.0) and np.signbit(sub[1])
    nan = conv("f", np.array([np.nan], np.float32))
    assert np.isnan(nan).all()
