"""The FP32 mode's double-precision width exponential (paper §2.4: the evaporation widths'
e^x, x = 2 sqrt(aY)), computed on the integer pipes by a table-driven fixed-point method
(paper_1309_7963_gb300/csrc/expfixed.h). CPU: its constants equal their mathematical
definitions (log2 e, ln 2, 1/n!, 2^(j/64), each to its stated number of bits, computed here
with 80-digit decimal arithmetic), and the algorithm, as the header states it, emulated with
exact integers, is within 0.51 ulp of e^x for float arguments in [1, 256). GPU: the kernel
gives the same bits as the emulation and stays within 1 ulp of the host's exp."""
import math
import os
import re
import struct
from decimal import Decimal, getcontext

import numpy as np
import pytest

getcontext().prec = 80
HDR = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1309_7963_gb300", "csrc",
                        "expfixed.h")).read()
LN2 = Decimal(2).ln()


def const(name):
    return int(re.search(name + r"\s*=\s*0x([0-9A-F]+)ull", HDR).group(1), 16)


def array(name):
    body = re.search(name + r"\[\d+\]\s*=\s*\{([^}]*)\}", HDR).group(1)
    return [int(v, 16) for v in re.findall(r"0x([0-9A-F]+)ull", body)]


def nearest(v):
    return int(v.to_integral_value())


def test_constants_are_their_definitions():
    c = (const("kLog2eHi") << 32) | const("kLog2eLo")
    assert c == nearest(Decimal(2) ** 95 / LN2)
    assert const("kLn2Q64") == nearest(LN2 * Decimal(2) ** 64)
    assert array("kInvFact") == [nearest(Decimal(2) ** 63 / math.factorial(n)) for n in range(1, 8)]
    assert array("kExp2Q63") == [nearest(Decimal(2) ** (Decimal(j) / 64) * Decimal(2) ** 63) for j in range(64)]


def emulate(xf):
    """The header's algorithm with exact integers."""
    M64 = (1 << 64) - 1
    C_HI, C_LO, LN2Q = const("kLog2eHi"), const("kLog2eLo"), const("kLn2Q64")
    fact, tab = array("kInvFact"), array("kExp2Q63")
    u = struct.unpack("<I", struct.pack("<f", xf))[0]
    X = ((u & 0x7FFFFF) | 0x800000) << ((u >> 23) - 127)
    lo, hi = (X * C_HI) & M64, (X * C_HI) >> 64
    t = (X * C_LO) >> 32
    lo2 = (lo + t) & M64
    hi += 1 if lo2 < t else 0
    k = hi >> 22
    f = ((hi << 42) | (lo2 >> 22)) & M64
    j = f >> 58
    r = ((f & ((1 << 58) - 1)) * LN2Q) >> 64
    s = fact[6]
    for n in range(5, -1, -1):
        s = fact[n] + ((r * s) >> 64)
    er = (1 << 63) + ((r * s) >> 64)
    M = (tab[j] * er) >> 64
    q, rem = M >> 10, M & 0x3FF
    q += 1 if (rem > 512 or (rem == 512 and q & 1)) else 0
    if q >> 53:
        q, k = q >> 1, k + 1
    return struct.unpack("<d", struct.pack("<Q", ((k + 1023) << 52) | (q - (1 << 52))))[0]


def floats(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(1.0, 256.0, n).astype(np.float32)
    edge = np.array([1.0, np.nextafter(np.float32(1), np.float32(2)), 2.0, 64.0, 87.0, 128.0, 200.0,
                     np.nextafter(np.float32(256), np.float32(0))], np.float32)
    return np.concatenate([edge, x])


def ulp_error(a, xf):
    v = Decimal(float(xf)).exp()
    return float(abs(Decimal(a) - v) / Decimal(math.ulp(a)))


def test_emulated_algorithm_is_within_half_an_ulp():
    xs = floats(4000, 1)
    errs = [ulp_error(emulate(float(x)), x) for x in xs]
    assert max(errs) < 0.51
    # a plausible slip (a table entry off by one, a dropped Taylor term) is far outside that
    assert np.mean([emulate(float(x)) == float(Decimal(float(x)).exp()) for x in xs]) > 0.99


@pytest.mark.gpu
def test_kernel_matches_the_emulation_and_the_host_exp(ctx):
    import torch
    xs = floats(1 << 20, 2)
    got = ctx.width_exp(torch.tensor(xs, device="cuda")).cpu().numpy()
    ref = np.exp(xs.astype(np.float64))
    ulp = np.spacing(ref)
    assert np.all(np.abs(got - ref) <= ulp)  # within 1 ulp of the host's exp everywhere
    assert np.mean(got == ref) > 0.99
    sub = np.random.default_rng(3).choice(len(xs), 3000, replace=False)
    assert all(got[i] == emulate(float(xs[i])) for i in sub)
    bad = ctx.width_exp(torch.tensor([0.5, 256.0, -3.0], dtype=torch.float32, device="cuda")).cpu().numpy()
    assert np.all(bad == -1.0)
