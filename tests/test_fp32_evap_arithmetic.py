"""Reading M25 (the scaled FP32 evaporation arithmetic, PNUC_FP32_SCALED), checked on the CPU against the
oracle's FP64 widths (§2.4: Weisskopf–Ewing widths with closed-form integrals, channel drawn
with probability Γ_j / ΣΓ). The FP32 mode evaluates each width times e^-xm, xm the largest x
of the parent's open channels. An FP32 emulation of that formula (numpy float32) must give
the oracle's channel probabilities to FP32 accuracy for light to heavy parents and E* up to
300 MeV: where e^-xm is flushed to 0 (xm > 87; the kernels flush denormals) and the
unscaled widths overflow FP32, and where
the series branch (x < 1) is taken. A second check shows the case the clamp of the release
at 0 is for: with x rounded to FP32, a t drawn next to 0 on a channel without barrier can put
U = (x - t)^2 / (4a) above E* - Q."""
import numpy as np
import pytest

import oracle

f = np.float32


def ftz(v):
    return f(0) if 0 < abs(v) < np.finfo(np.float32).tiny else v


def oracle_channels(Z, A, Estar):
    """Open channels of the parent as the oracle computes them (None where closed), with the
    prefactor w0 = width / integral."""
    out = []
    for j in range(6):
        c = oracle.channel(Z, A, Estar, j)
        if not c["width"] > 0.0:
            out.append(None)
            continue
        Y = c["x"] ** 2 / (4.0 * c["a"])
        c["w0"] = c["width"] / oracle.width_integral(c["a"], Y, c["b"])
        out.append(c)
    return out


ULP = 2.0 ** -23  # float32 relative spacing at most


def exp_err(arg):
    """Relative error bound of the fast-math single-precision exponential at argument arg:
    2 + floor(|1.173 arg|) ulp (the CUDA Programming Guide's table of intrinsic functions)."""
    return (2 + np.floor(abs(1.173 * float(arg)))) * ULP


def scaled_widths_f32(chans, sign=None):
    """The PNUC_FP32_SCALED widths times e^-xm, in float32 arithmetic (reading M25), with the
    exponentials' denormal results flushed to 0 as the fast-math kernels do. With sign (a
    function giving +1 or -1 per approximate operation), every exponential, reciprocal and
    division is moved by its published error bound in that direction: the fast-math kernels
    compute them approximately (expf, 1/a and x/n), the products and sums exactly rounded."""
    if sign is None:
        def bump(v, rel):
            return v
    else:
        def bump(v, rel):
            return f(np.float64(v) * (1.0 + sign() * rel))
    xm = f(0)
    for c in chans:
        if c is not None and f(c["x"]) > xm:
            xm = f(c["x"])
    with np.errstate(under="ignore"):
        s = ftz(bump(np.exp(-xm, dtype=np.float32), exp_err(xm)))
        w = np.zeros(6, np.float32)
        for j, c in enumerate(chans):
            if c is None:
                continue
            x, a, b, w0 = f(c["x"]), f(c["a"]), f(c["b"]), f(c["w0"])
            if x >= f(1):
                ex = ftz(bump(np.exp(x - xm, dtype=np.float32), exp_err(x - xm)))
                F = ex * (x * x - f(3) * x + f(3)) + (f(0.5) * x * x - f(3)) * s
                G = ex * (x - f(1)) + s
            else:
                term, fs, gs = x, f(0), f(0)
                for n in range(2, 21):
                    term = term * bump(x / f(n), 2 * ULP)
                    gs = gs + f(n - 1) * term
                    if n >= 4:
                        fs = fs + f((n - 1) * (n - 3)) * term
                F, G = fs * s, gs * s
            ia = bump(f(1) / a, ULP)
            w[j] = w0 * (F * (f(0.25) * ia * ia) + G * (f(0.5) * b * ia))
    return w


PARENTS = [(6, 12), (8, 16), (20, 40), (26, 56), (50, 120), (82, 208)]
ESTARS = [0.5, 2.0, 5.0, 10.0, 20.0, 50.0, 100.0, 200.0, 300.0]


@pytest.mark.parametrize("za", PARENTS)
def test_scaled_fp32_widths_give_the_oracle_channel_probabilities(za):
    Z, A = za
    seen_underflow = False
    for Es in ESTARS:
        chans = oracle_channels(Z, A, Es)
        g64 = np.array([c["width"] if c else 0.0 for c in chans])
        if not g64.sum() > 0.0:
            continue
        w32 = scaled_widths_f32(chans)
        assert np.isfinite(w32).all() and w32.sum() > 0
        p64 = g64 / g64.sum()
        p32 = w32.astype(np.float64) / float(w32.sum(dtype=np.float32))
        assert np.abs(p32 - p64).max() < 3e-5, (za, Es, p32, p64)
        seen_underflow |= max(c["x"] for c in chans if c) > 88.0
    if za == (82, 208):
        assert seen_underflow  # the range where e^-xm is flushed to 0 is covered


@pytest.mark.parametrize("za", [(8, 16), (26, 56), (82, 208)])
def test_scaled_widths_within_the_fast_math_error_bounds(za):
    """The same bound with every approximate operation of the fast-math kernels (the
    exponentials, the reciprocal of a and the series' divisions) moved by its published
    worst-case error: all up, all down, and 16 random sign patterns per excitation."""
    Z, A = za
    rng = np.random.default_rng(4)
    for Es in ESTARS:
        chans = oracle_channels(Z, A, Es)
        g64 = np.array([c["width"] if c else 0.0 for c in chans])
        if not g64.sum() > 0.0:
            continue
        p64 = g64 / g64.sum()
        signs = [lambda: 1.0, lambda: -1.0] + [lambda: float(rng.choice((-1.0, 1.0)))] * 16
        for sg in signs:
            w32 = scaled_widths_f32(chans, sign=sg)
            p32 = w32.astype(np.float64) / float(w32.sum(dtype=np.float32))
            assert np.abs(p32 - p64).max() < 3e-5, (za, Es, p32, p64)


def test_fp32_rounding_can_put_U_above_the_excitation():
    """The channel without barrier (the neutron below A = 191) at the smallest t the FP32
    sampler can draw: U from the FP32 x exceeds E* - Q in a fraction of cases, which is why
    the FP32 decay takes the release as max(E* - Q - U, 0)."""
    Estar = np.linspace(20.0, 120.0, 4001)
    neg = 0
    for Es in Estar:
        c = oracle.channel(8, 16, float(Es), 0)
        assert c["V"] == 0.0 and Es - c["Q"] > 0.0
        X64 = Es - c["Q"]
        a = f(c["a"])
        x = f(2) * np.sqrt(a * f(X64))
        t = x * f(2.0**-24)
        xt = np.float64(x) - np.float64(t)
        U = xt * xt / (4.0 * np.float64(a))
        eps = X64 - U
        if eps < 0.0:
            neg += 1
            assert max(eps, 0.0) == 0.0
    assert 0 < neg < len(Estar) // 2
