"""FP64 CPU oracle of the proton-nucleus cascade + evaporation model (arXiv:1309.7963 §2).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()`` and by the
CPU-baseline leg of ``bench.py``. The pnuc library and its Python binding never import it.
It shares no code with the CUDA path; the only common module is the seeded input generator
(``paper_1309_7963_gb300.inputs``), which holds none of the model's arithmetic.

The C source ``pnuc_oracle.c`` is compiled with ``-ffp-contract=off`` (no fused
multiply-add) so that its FP64 arithmetic is the plain IEEE sequence the model states.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pnuc_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")

TARGET_DTYPE = np.dtype([
    ("Z", "<i4"), ("A", "<i4"), ("c", "<f8"), ("R", "<f8"), ("EC", "<f8"), ("ZoverA", "<f8"),
    ("M", "<f8"), ("S", "<f8", (2,)), ("r", "<f8", (16,)), ("rho", "<f8", (15,)),
    ("rho_s", "<f8", (2, 15)), ("pF", "<f8", (2, 15)), ("EF", "<f8", (2, 15)),
    ("V", "<f8", (2, 15)), ("vF", "<f8", (15,)),
])
SECONDARY_DTYPE = np.dtype([
    ("event", "<u4"), ("species", "<i4"), ("origin", "<i4"), ("index", "<i4"),
    ("T", "<f8"), ("ux", "<f8"), ("uy", "<f8"), ("uz", "<f8"),
    ("px", "<f8"), ("py", "<f8"), ("pz", "<f8"),
])
RESIDUAL_DTYPE = np.dtype([
    ("Zc", "<i4"), ("Ac", "<i4"), ("Zf", "<i4"), ("Af", "<i4"), ("n_casc", "<i4"),
    ("n_evap", "<i4"), ("n_coll", "<i4"), ("n_attempts", "<i4"), ("flags", "<u4"), ("pad", "<u4"),
    ("Estar_c", "<f8"), ("Estar_f", "<f8"), ("Pcas", "<f8", (3,)), ("Pf", "<f8", (3,)),
    ("Ef", "<f8"),
])
COUNTER_NAMES = ("steps", "candidates", "kinematics", "pauli_blocked", "collisions", "crossings",
                 "reflections", "escapes", "captures", "attempts", "evap_steps", "evap_trials", "draws",
                 "settled", "evap_passes", "evap_exps", "evap_series")
COUNTERS_DTYPE = np.dtype([(n, "<u8") for n in COUNTER_NAMES])
LIMITS_DTYPE = np.dtype([("max_steps", "<i4"), ("max_attempts", "<i4"), ("stack_cap", "<i4"),
                         ("max_evap_steps", "<i4"), ("max_evap_trials", "<i4"), ("level_density", "<i4")])
TRACE_DTYPE = np.dtype([("event", "<u4"), ("kind", "<i4"), ("species", "<i4"), ("shell", "<i4"),
                        ("T", "<f8"), ("x", "<f8"), ("y", "<f8"), ("z", "<f8")])
TRACE_KINDS = {"entry": 0, "null": 1, "pauli": 2, "collision": 3, "refract": 4, "reflect": 5,
               "escape": 6, "capture": 7, "evap": 8, "product": 9}

# level_density: 0 the Fermi gas of reading M20 (default), 1 the constant-temperature composite
# of reading M26
DEFAULT_LIMITS = dict(max_steps=100000, max_attempts=1000, stack_cap=64, max_evap_steps=64,
                      max_evap_trials=10000, level_density=0)

# physical constants of the model, for tests that need them (masses in MeV)
M_P, M_N = 938.272, 939.565
EJECTILE_MASS = (M_N, M_P, 1875.613, 2808.921, 2808.391, 3727.379)
EJECTILE_ZA = ((0, 1), (1, 1), (1, 2), (1, 3), (2, 3), (2, 4))

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, FP64, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                        "-shared", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _SO)
    return _SO


def lib() -> C.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            d, i32, i64, u64, vp = C.c_double, C.c_int32, C.c_int64, C.c_uint64, C.c_void_p
            L.orc_philox4x64_10.argtypes = [vp, vp, vp]
            L.orc_uniform.argtypes = [C.c_uint32]
            L.orc_uniform.restype = d
            L.orc_stream_draws.argtypes = [u64, u64, C.c_int64, vp]
            L.orc_semf_mass.argtypes = [i32, i32]
            L.orc_semf_mass.restype = d
            L.orc_target_setup.argtypes = [i32, i32, vp]
            L.orc_target_setup.restype = C.c_int
            L.orc_sigma.argtypes = [C.c_int, d]
            L.orc_sigma.restype = d
            L.orc_slope.argtypes = [C.c_int, d]
            L.orc_slope.restype = d
            L.orc_backward_a.argtypes = [d]
            L.orc_backward_a.restype = d
            L.orc_g_hat.argtypes = [d, d, d]
            L.orc_g_hat.restype = d
            L.orc_cos_theta.argtypes = [d, d, d]
            L.orc_cos_theta.restype = d
            L.orc_rotate.argtypes = [vp, d, d, d, vp]
            L.orc_collide.argtypes = [C.c_int, vp, C.c_int, vp, d, d, d, vp, vp]
            L.orc_boundary_distance.argtypes = [vp, C.c_int, vp, vp, vp]
            L.orc_boundary_distance.restype = d
            L.orc_refract.argtypes = [vp, vp, d, d, i32]
            L.orc_refract.restype = C.c_int
            L.orc_width_integral.argtypes = [d, d, d]
            L.orc_width_integral.restype = d
            L.orc_channel.argtypes = [C.c_int, C.c_int, d, C.c_int, vp, vp, vp, vp, vp, vp]
            L.orc_channel.restype = d
            L.orc_channel_ld.argtypes = [C.c_int, C.c_int, d, C.c_int, C.c_int, vp, vp, vp, vp, vp, vp]
            L.orc_channel_ld.restype = d
            L.orc_level_density.argtypes = [d, d, C.c_int]
            L.orc_level_density.restype = d
            L.orc_width_integral_ct.argtypes = [d, d, d, vp]
            L.orc_width_integral_ct.restype = d
            L.orc_sample_U_ct.argtypes = [d, d, d, u64, u64, i64, vp]
            L.orc_sample_U_ct.restype = i64
            L.orc_sample_U.argtypes = [d, d, d, u64, u64, i64, vp]
            L.orc_sample_U.restype = i64
            L.orc_sample_fermi.argtypes = [d, u64, u64, i64, vp]
            L.orc_simulate.argtypes = [vp, i32, vp, vp, vp, u64, u64, u64, vp, u64, vp, vp, vp, vp, i64,
                                       vp, u64, vp]
            L.orc_simulate.restype = u64
            L.orc_sizeof.argtypes = [C.c_int]
            L.orc_sizeof.restype = i64
            for k, dt in enumerate((TARGET_DTYPE, SECONDARY_DTYPE, RESIDUAL_DTYPE, COUNTERS_DTYPE,
                                    LIMITS_DTYPE, TRACE_DTYPE)):
                if L.orc_sizeof(k) != dt.itemsize:
                    raise RuntimeError(f"oracle record {k}: C size {L.orc_sizeof(k)} != {dt.itemsize}")
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# ------------------------------------------------------------------ component entry points
def philox4x64_10(counter, key) -> np.ndarray:
    c = np.ascontiguousarray(counter, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, np.uint64)
    lib().orc_philox4x64_10(_p(c), _p(k), _p(out))
    return out


def uniform(half: int) -> float:
    """The uniform of one 32-bit half of a Philox word."""
    return lib().orc_uniform(int(half))


def stream_draws(seed: int, event: int, n: int) -> np.ndarray:
    """The first n uniforms of an event's draw stream."""
    out = np.zeros(n, np.float64)
    lib().orc_stream_draws(seed, event, n, _p(out))
    return out


def semf_mass(Z: int, A: int) -> float:
    return lib().orc_semf_mass(Z, A)


def target(Z: int, A: int) -> np.ndarray:
    t = np.zeros(1, TARGET_DTYPE)
    if lib().orc_target_setup(Z, A, _p(t)) != 0:
        raise ValueError(f"unsupported target Z={Z} A={A}")
    return t[0]


def sigma(like: bool, p_gev: float) -> float:
    return lib().orc_sigma(int(like), p_gev)


def slope(like: bool, p_gev: float) -> float:
    return lib().orc_slope(int(like), p_gev)


def backward_a(p_gev: float) -> float:
    return lib().orc_backward_a(p_gev)


def g_hat(p1: float, E1: float, vF: float) -> float:
    """Majorant of sigma * v_rel * E1 (GeV mb) for a projectile with momentum p1, energy E1 (MeV)."""
    return lib().orc_g_hat(p1, E1, vF)


def cos_theta(B: float, pstar_gev: float, u: float) -> float:
    return lib().orc_cos_theta(B, pstar_gev, u)


def rotate(n, ct: float, phi: float) -> np.ndarray:
    n = np.ascontiguousarray(n, np.float64)
    d = np.zeros(3)
    lib().orc_rotate(_p(n), ct, float(np.sqrt((1 - ct) * (1 + ct))), phi, _p(d))
    return d


def collide(s1: int, p1, s2: int, p2, ut: float, uphi: float, uf: float):
    p1 = np.ascontiguousarray(p1, np.float64)
    p2 = np.ascontiguousarray(p2, np.float64)
    q1, q2 = np.zeros(3), np.zeros(3)
    lib().orc_collide(s1, _p(p1), s2, _p(p2), ut, uphi, uf, _p(q1), _p(q2))
    return q1, q2


def boundary_distance(tgt: np.ndarray, shell: int, r, d):
    t = np.array([tgt], TARGET_DTYPE)
    r = np.ascontiguousarray(r, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    direction = np.zeros(1, np.int32)
    s = lib().orc_boundary_distance(_p(t), shell, _p(r), _p(d), _p(direction))
    return s, int(direction[0])


def refract(n, p, m: float, dT: float, direction: int | None = None):
    """A boundary crossing (M11) with outward normal n; direction +1 (outward) or -1 (inward),
    by default the way p points along n."""
    n = np.ascontiguousarray(n, np.float64)
    p = np.array(p, np.float64)
    if direction is None:
        direction = 1 if float(np.dot(n, p)) >= 0.0 else -1
    ok = lib().orc_refract(_p(n), _p(p), m, dT, int(direction))
    return bool(ok), p


def width_integral(a: float, Y: float, b: float) -> float:
    return lib().orc_width_integral(a, Y, b)


def level_density(a: float, U: float, mode: int = 0) -> float:
    """The daughter's level density: mode 0 the Fermi gas (M20), 1 the composite (M26)."""
    return lib().orc_level_density(a, U, mode)


def width_integral_ct(a: float, Y: float, b: float):
    """Reading M26's width integral and its constant-temperature part."""
    part = np.zeros(1)
    total = lib().orc_width_integral_ct(a, Y, b, _p(part))
    return total, float(part[0])


def channel(Z: int, A: int, Estar: float, j: int, level_density: int = 0) -> dict:
    out = [np.zeros(1) for _ in range(6)]
    g = lib().orc_channel_ld(Z, A, Estar, j, level_density, *[_p(o) for o in out])
    V, b, Q, Md, a, x = (float(o[0]) for o in out)
    return dict(width=g, V=V, b=b, Q=Q, Md=Md, a=a, x=x)


def sample_U(a: float, x: float, b: float, n: int, seed: int = 0, event: int = 0):
    out = np.zeros(n)
    trials = lib().orc_sample_U(a, x, b, seed, event, n, _p(out))
    return out, trials


def sample_U_ct(a: float, Y: float, b: float, n: int, seed: int = 0, event: int = 0):
    """n draws of reading M26's emission sampler (daughter excitations U) and the trials taken."""
    out = np.zeros(n)
    trials = lib().orc_sample_U_ct(a, Y, b, seed, event, n, _p(out))
    return out, trials


def sample_fermi(pF: float, n: int, seed: int = 0, event: int = 0) -> np.ndarray:
    out = np.zeros((n, 3))
    lib().orc_sample_fermi(pF, seed, event, n, _p(out))
    return out


# ------------------------------------------------------------------ whole events
def make_targets(za_list):
    return np.array([target(Z, A) for (Z, A) in za_list], TARGET_DTYPE)


def simulate(targets, energies, tidx, seed: int, first_event_id: int = 0, limits=None,
             inject=None, trace: bool = False, trace_cap: int = 1 << 20, sec_per_event: int = 40,
             projectiles=None):
    """Runs events first_event_id + k on targets[tidx[k]] at energies[k] MeV, serially.

    targets: TARGET_DTYPE array (see make_targets) or list of (Z, A). projectiles: the
    incident nucleon of each event (1 proton, 0 neutron); None = all protons.
    Returns dict(secondaries, residuals, counters[, trace]). Secondaries are in event
    order, each event's in emission order.
    """
    L = lib()
    if not isinstance(targets, np.ndarray) or targets.dtype != TARGET_DTYPE:
        targets = make_targets(targets)
    targets = np.ascontiguousarray(targets)
    e = np.ascontiguousarray(energies, np.float64)
    ti = np.ascontiguousarray(tidx, np.int32)
    n = int(e.shape[0])
    assert ti.shape[0] == n
    pj = None if projectiles is None else np.ascontiguousarray(projectiles, np.int32)
    assert pj is None or pj.shape[0] == n
    lim = np.zeros(1, LIMITS_DTYPE)
    for k, v in {**DEFAULT_LIMITS, **(limits or {})}.items():
        lim[k] = v
    cnt = np.zeros(1, COUNTERS_DTYPE)
    res = np.zeros(n, RESIDUAL_DTYPE)
    inj = None if inject is None else np.ascontiguousarray(inject, np.float64)
    cap = max(16, n * sec_per_event)
    while True:
        sec = np.zeros(cap, SECONDARY_DTYPE)
        tr = np.zeros(trace_cap if trace else 0, TRACE_DTYPE)
        trc = np.zeros(1, np.uint64)
        got = L.orc_simulate(_p(targets), len(targets), _p(e), _p(ti), None if pj is None else _p(pj), n, seed,
                             first_event_id,
                             _p(sec), cap, _p(res), _p(cnt), _p(lim),
                             None if inj is None else _p(inj), 0 if inj is None else len(inj),
                             _p(tr) if trace else None, trace_cap if trace else 0, _p(trc))
        if got <= cap:
            break
        cap = int(got)
    out = dict(secondaries=sec[:got], residuals=res,
               counters={k: int(cnt[0][k]) for k in COUNTER_NAMES})
    if trace:
        out["trace"] = tr[: min(int(trc[0]), trace_cap)]
        out["trace_total"] = int(trc[0])
    return out


def simulate_parallel(targets, energies, tidx, seed: int, first_event_id: int = 0,
                      threads: int | None = None, chunk: int = 2048, limits=None, keep: bool = True,
                      projectiles=None):
    """simulate() over event chunks on a thread pool (the C call releases the GIL).

    Results are identical to simulate(): every event depends only on (seed, event id).
    Returns the same dict plus 'threads' (the number of worker threads used). With
    keep=False only the counters and the number of secondaries are returned (for timing).
    """
    if not isinstance(targets, np.ndarray) or targets.dtype != TARGET_DTYPE:
        targets = make_targets(targets)
    e = np.ascontiguousarray(energies, np.float64)
    ti = np.ascontiguousarray(tidx, np.int32)
    pj = None if projectiles is None else np.ascontiguousarray(projectiles, np.int32)
    n = e.shape[0]
    threads = threads or os.cpu_count() or 1
    starts = list(range(0, n, chunk))

    def run(s0):
        r = simulate(targets, e[s0:s0 + chunk], ti[s0:s0 + chunk], seed, first_event_id + s0,
                     limits=limits, projectiles=None if pj is None else pj[s0:s0 + chunk])
        r["secondaries"]["event"] += s0
        if not keep:
            r = dict(n_secondaries=len(r["secondaries"]), counters=r["counters"])
        return r

    lib()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(run, starts))
    if not keep:
        counters = {k: sum(p["counters"][k] for p in parts) for k in COUNTER_NAMES}
        return dict(n_secondaries=sum(p["n_secondaries"] for p in parts), counters=counters, threads=threads)
    sec = np.concatenate([p["secondaries"] for p in parts]) if parts else np.zeros(0, SECONDARY_DTYPE)
    res = np.concatenate([p["residuals"] for p in parts]) if parts else np.zeros(0, RESIDUAL_DTYPE)
    counters = {k: sum(p["counters"][k] for p in parts) for k in COUNTER_NAMES}
    return dict(secondaries=sec, residuals=res, counters=counters, threads=threads)
