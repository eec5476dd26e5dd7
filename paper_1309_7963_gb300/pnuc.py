"""Python binding of libpnuc (include/pnuc.h): argument marshalling only.

Every step of the simulation runs in the library's CUDA kernels. Device buffers are torch
tensors; streams are torch CUDA streams. There is no CPU fallback: constructing a Context
raises if the library cannot be loaded or no CUDA device is present.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None

SECONDARY_DTYPE = np.dtype([("event", "<u4"), ("species", "u1"), ("origin", "u1"), ("index", "<u2"),
                            ("T", "<f8"), ("ux", "<f4"), ("uy", "<f4"), ("uz", "<f4"), ("reserved", "<u4")])
RESIDUAL_DTYPE = np.dtype([("Z_cascade", "<u2"), ("A_cascade", "<u2"), ("Z_final", "<u2"), ("A_final", "<u2"),
                           ("n_cascade", "<u2"), ("n_evaporated", "<u2"), ("n_collisions", "<u2"),
                           ("n_attempts", "<u2"), ("flags", "<u4"), ("reserved", "<u4"),
                           ("Estar_cascade", "<f8"), ("Estar_final", "<f8"), ("P_cascade", "<f4", (3,)),
                           ("P_final", "<f4", (3,))])
assert SECONDARY_DTYPE.itemsize == 32 and RESIDUAL_DTYPE.itemsize == 64

COUNTER_NAMES = ("steps", "candidates", "kinematics", "pauli_blocked", "collisions", "crossings", "reflections",
                 "escapes", "captures", "attempts", "evap_steps", "evap_trials", "draws", "settled", "evap_passes",
                 "evap_exps", "evap_series", "cycles_transport", "cycles_collision", "cycles_evaporation",
                 "cycles_refill")
FLAGS = dict(bad_input=1, attempt_cap=2, step_cap=4, stack_overflow=8, bad_residual=16, no_excitation=32,
             evap_trial_cap=64, evap_step_cap=128, output_overflow=256)
# "fp32": FP32 bulk with FP64 evaporation widths; "fp32_scaled": the widths in FP32 as well, scaled by the
# largest channel's exponential; "fp64": the deterministic mode (per-event oracle parity)
PRECISION = {"fp32": 0, "fp64": 1, "fp32_scaled": 2}
METHOD = {"plain": 0, "persistent": 1, "sorted": 2}
STATUS = {0: "ok", 1: "invalid argument", 2: "out of range", 3: "capacity exceeded", 4: "CUDA error",
          5: "timeout", 6: "invalid state"}


class pnuc_config(C.Structure):
    _fields_ = [("device", C.c_int32), ("max_steps", C.c_int32), ("max_attempts", C.c_int32),
                ("max_evap_steps", C.c_int32), ("max_evap_trials", C.c_int32), ("level_density", C.c_int32)]


class pnuc_batch(C.Structure):
    _fields_ = [("energies", C.c_void_p), ("target_ids", C.c_void_p), ("n", C.c_uint64), ("seed", C.c_uint64),
                ("first_event_id", C.c_uint64), ("projectiles", C.c_void_p),
                ("event_ids", C.c_void_p)]


class pnuc_output(C.Structure):
    _fields_ = [("secondaries", C.c_void_p), ("capacity", C.c_uint64), ("count", C.c_void_p),
                ("residuals", C.c_void_p), ("counters", C.c_void_p)]


TRACE_DTYPE = np.dtype([("ticket", "<u8"), ("events", "<u8"), ("launch", "<u8"), ("stream", "<i4"),
                        ("group_requests", "<i4"), ("reruns", "<i4"), ("status", "<i4"), ("t_submit", "<f8"),
                        ("t_admit", "<f8"), ("t_launched", "<f8"), ("t_gpu_start", "<f8"), ("t_gpu_end", "<f8"),
                        ("t_complete", "<f8"), ("t_release", "<f8")])


class pnuc_tuning(C.Structure):
    _fields_ = [("block_size", C.c_int32), ("blocks_per_sm", C.c_int32), ("refill_threshold", C.c_int32),
                ("chunk", C.c_int32), ("kin_batch", C.c_int32)]


class pnuc_target_info(C.Structure):
    _fields_ = [("Z", C.c_int32), ("A", C.c_int32), ("R", C.c_double), ("EC", C.c_double), ("M", C.c_double),
                ("S_n", C.c_double), ("S_p", C.c_double), ("r", C.c_double * 16), ("rho", C.c_double * 15),
                ("vF", C.c_double * 15), ("pF", (C.c_double * 15) * 2), ("EF", (C.c_double * 15) * 2),
                ("V", (C.c_double * 15) * 2)]


class pnuc_peaks(C.Structure):
    _fields_ = [("fp32_fma", C.c_double), ("fp64_fma", C.c_double), ("mufu", C.c_double), ("int32_mad", C.c_double)]


class pnuc_tally_spec(C.Structure):
    _fields_ = [("n_T", C.c_int32), ("n_cos", C.c_int32), ("T_min", C.c_double), ("T_max", C.c_double),
                ("n_E", C.c_int32), ("Z_max", C.c_int32), ("E_min", C.c_double), ("E_max", C.c_double),
                ("A_max", C.c_int32), ("reserved", C.c_int32)]


class pnuc_server_config(C.Structure):
    _fields_ = [("precision", C.c_int32), ("streams", C.c_int32), ("arena_bytes", C.c_uint64),
                ("sec_per_event", C.c_uint32), ("max_pending", C.c_uint32), ("max_request_events", C.c_uint64),
                ("max_merge", C.c_uint32), ("merge_events", C.c_uint32),
                ("lane_events", C.c_uint32), ("max_inflight_events", C.c_uint32)]


class pnuc_server_stats(C.Structure):
    _fields_ = [("completed", C.c_uint64), ("failed", C.c_uint64), ("reruns", C.c_uint64), ("events", C.c_uint64),
                ("pending", C.c_uint64), ("latency_p50_ms", C.c_double), ("latency_p99_ms", C.c_double),
                ("latency_max_ms", C.c_double), ("queue_p50_ms", C.c_double), ("queue_p99_ms", C.c_double),
                ("elapsed_s", C.c_double), ("events_per_s", C.c_double), ("arena_peak_bytes", C.c_uint64),
                ("launches", C.c_uint64)]


class PnucError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"pnuc: {STATUS.get(status, status)}: {message}")
        self.status = status


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> C.CDLL:
    """Loads libpnuc.so (building it with nvcc if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"libpnuc not built: {_build.LIB} is missing")
    L = C.CDLL(_build.LIB)
    vp, u64, i32 = C.c_void_p, C.c_uint64, C.c_int32
    L.pnuc_default_config.argtypes = [C.POINTER(pnuc_config)]
    L.pnuc_default_config.restype = None
    L.pnuc_create.argtypes = [C.POINTER(pnuc_config), C.POINTER(vp)]
    L.pnuc_destroy.argtypes = [vp]
    L.pnuc_status_string.argtypes = [C.c_int]
    L.pnuc_status_string.restype = C.c_char_p
    L.pnuc_last_error.argtypes = [vp, C.c_char_p, C.c_size_t]
    L.pnuc_create_target.argtypes = [vp, i32, i32, C.POINTER(i32)]
    L.pnuc_target_table.argtypes = [vp, i32, C.POINTER(pnuc_target_info)]
    L.pnuc_simulate.argtypes = [vp, C.c_int, C.c_int, C.POINTER(pnuc_batch), C.POINTER(pnuc_output), vp]
    L.pnuc_simulate_host.argtypes = [vp, C.c_int, C.c_int, vp, vp, u64, u64, u64, vp, u64, C.POINTER(u64), vp, vp]
    L.pnuc_simulate_host_noalloc.argtypes = [vp, C.c_int, C.c_int, vp, vp, u64, u64, u64, vp, u64, C.POINTER(u64),
                                             vp, vp]
    L.pnuc_width_exp.argtypes = [vp, vp, vp, u64, vp]
    L.pnuc_get_tuning.argtypes = [vp, C.c_int, C.POINTER(pnuc_tuning)]
    L.pnuc_set_tuning.argtypes = [vp, C.c_int, C.POINTER(pnuc_tuning)]
    L.pnuc_measure_peaks.argtypes = [vp, C.POINTER(pnuc_peaks)]
    L.pnuc_kernel_timing.argtypes = [vp, C.c_int32]
    L.pnuc_kernel_times.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(u64)]
    L.pnuc_tally.argtypes = [vp, C.POINTER(pnuc_tally_spec), vp, u64, vp, vp, u64, vp, vp, vp]
    L.pnuc_tally_windows.argtypes = [vp, C.c_int32, C.c_double, C.c_double, C.POINTER(C.c_double),
                                     C.POINTER(C.c_double), C.c_int32, vp, u64, vp, vp]
    L.pnuc_autotune.argtypes = [vp, C.c_int, C.POINTER(pnuc_batch), C.POINTER(pnuc_output), C.c_int32,
                                C.POINTER(pnuc_tuning), C.POINTER(C.c_double), vp]
    L.pnuc_save_tuning.argtypes = [vp, C.c_char_p]
    L.pnuc_load_tuning.argtypes = [vp, C.c_char_p]
    L.pnuc_graph_create.argtypes = [vp, C.c_int, C.c_int, C.POINTER(pnuc_batch), C.POINTER(pnuc_output), C.POINTER(vp)]
    L.pnuc_graph_update.argtypes = [vp, C.POINTER(pnuc_batch), C.POINTER(pnuc_output)]
    L.pnuc_graph_launch.argtypes = [vp, vp]
    L.pnuc_graph_destroy.argtypes = [vp]
    L.pnuc_server_default_config.argtypes = [C.POINTER(pnuc_server_config)]
    L.pnuc_server_default_config.restype = None
    L.pnuc_server_create.argtypes = [vp, C.POINTER(pnuc_server_config), C.POINTER(vp)]
    L.pnuc_server_submit.argtypes = [vp, vp, vp, u64, u64, u64, C.POINTER(u64)]
    L.pnuc_server_submit_nucleons.argtypes = [vp, vp, vp, vp, u64, u64, u64, C.POINTER(u64)]
    L.pnuc_server_wait.argtypes = [vp, u64, C.c_int32, C.POINTER(u64)]
    L.pnuc_server_wait_any.argtypes = [vp, C.c_int32, C.POINTER(u64)]
    L.pnuc_server_fetch.argtypes = [vp, u64, vp, u64, vp]
    L.pnuc_server_view.argtypes = [vp, u64, C.POINTER(vp), C.POINTER(u64), C.POINTER(vp)]
    L.pnuc_server_release.argtypes = [vp, u64]
    L.pnuc_server_trace.argtypes = [vp, i32]
    L.pnuc_server_trace_read.argtypes = [vp, vp, u64, C.POINTER(u64)]
    L.pnuc_server_get_stats.argtypes = [vp, C.POINTER(pnuc_server_stats)]
    L.pnuc_server_reset_stats.argtypes = [vp]
    L.pnuc_server_destroy.argtypes = [vp]
    for name in ("pnuc_create", "pnuc_destroy", "pnuc_last_error", "pnuc_create_target", "pnuc_target_table",
                 "pnuc_simulate", "pnuc_simulate_host", "pnuc_simulate_host_noalloc", "pnuc_get_tuning",
                 "pnuc_set_tuning",
                 "pnuc_measure_peaks", "pnuc_autotune", "pnuc_save_tuning", "pnuc_load_tuning",
                 "pnuc_graph_create", "pnuc_graph_update", "pnuc_graph_launch", "pnuc_graph_destroy",
                 "pnuc_server_create", "pnuc_server_submit", "pnuc_server_submit_nucleons", "pnuc_server_wait",
                 "pnuc_server_wait_any",
                 "pnuc_server_fetch",
                 "pnuc_server_get_stats", "pnuc_server_reset_stats", "pnuc_server_destroy"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


@dataclass
class Result:
    """Device outputs of one batch (torch tensors) and their host decoders."""
    secondaries: "object"  # uint8 tensor (capacity, 32)
    count: "object"        # int64 tensor (1,)
    residuals: "object"    # uint8 tensor (n, 64)
    counters: "object" = None

    def n_secondaries(self) -> int:
        return int(self.count.item())

    def secondaries_np(self) -> np.ndarray:
        k = min(self.n_secondaries(), self.secondaries.shape[0])
        return self.secondaries[:k].cpu().numpy().reshape(-1).view(SECONDARY_DTYPE)

    def residuals_np(self) -> np.ndarray:
        return self.residuals.cpu().numpy().reshape(-1).view(RESIDUAL_DTYPE)

    def counters_dict(self) -> dict:
        if self.counters is None:
            return {}
        v = self.counters.cpu().numpy()
        return {k: int(v[i]) for i, k in enumerate(COUNTER_NAMES)}


class Context:
    """A libpnuc context on one CUDA device: target tables, scratch, tuning."""

    def __init__(self, device: int = 0, **limits):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("pnuc needs a CUDA device; none is available (there is no CPU fallback)")
        self._torch = torch
        self.lib = load()
        cfg = pnuc_config()
        self.lib.pnuc_default_config(C.byref(cfg))
        cfg.device = device
        for k, v in limits.items():
            setattr(cfg, k, int(v))
        h = C.c_void_p()
        st = self.lib.pnuc_create(C.byref(cfg), C.byref(h))
        if st != 0:
            raise PnucError(st, "pnuc_create failed")
        self.handle = h
        self.device = device
        self.targets: list[tuple[int, int]] = []

    def close(self):
        if getattr(self, "handle", None):
            self.lib.pnuc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != 0:
            buf = C.create_string_buffer(512)
            self.lib.pnuc_last_error(self.handle, buf, 512)
            raise PnucError(st, buf.value.decode())

    def create_target(self, Z: int, A: int) -> int:
        tid = C.c_int32()
        self._check(self.lib.pnuc_create_target(self.handle, Z, A, C.byref(tid)))
        if tid.value == len(self.targets):
            self.targets.append((Z, A))
        return tid.value

    def target_table(self, target_id: int) -> dict:
        info = pnuc_target_info()
        self._check(self.lib.pnuc_target_table(self.handle, target_id, C.byref(info)))
        arr = lambda x: np.ctypeslib.as_array(x).copy()
        return dict(Z=info.Z, A=info.A, R=info.R, EC=info.EC, M=info.M, S=np.array([info.S_n, info.S_p]),
                    r=arr(info.r), rho=arr(info.rho), vF=arr(info.vF), pF=arr(info.pF), EF=arr(info.EF),
                    V=arr(info.V))

    def get_tuning(self, precision: str = "fp32") -> dict:
        t = pnuc_tuning()
        self._check(self.lib.pnuc_get_tuning(self.handle, PRECISION[precision], C.byref(t)))
        return {name: getattr(t, name) for name, _ in pnuc_tuning._fields_}

    def set_tuning(self, precision: str = "fp32", **kw):
        cur = self.get_tuning(precision)
        cur.update(kw)
        t = pnuc_tuning(**cur)
        self._check(self.lib.pnuc_set_tuning(self.handle, PRECISION[precision], C.byref(t)))

    def width_exp(self, x):
        """pnuc_width_exp: the FP32 mode's double-precision width exponential of a float32 CUDA
        tensor (e^x for x in [1, 256), -1 elsewhere), as a float64 tensor."""
        torch = self._torch
        x = x.contiguous()
        assert x.dtype == torch.float32 and x.is_cuda
        out = torch.empty(x.shape, dtype=torch.float64, device=x.device)
        self._check(self.lib.pnuc_width_exp(self.handle, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()),
                                            x.numel(), C.c_void_p(torch.cuda.current_stream().cuda_stream)))
        return out

    def measure_peaks(self) -> dict:
        """Lane operations per second of the FP32 FMA, FP64 FMA, MUFU and INT32 MAD pipes."""
        p = pnuc_peaks()
        self._check(self.lib.pnuc_measure_peaks(self.handle, C.byref(p)))
        return dict(fp32_fma=p.fp32_fma, fp64_fma=p.fp64_fma, mufu=p.mufu, int32_mad=p.int32_mad)

    def kernel_timing(self, enable: bool) -> None:
        """Start (clearing the record) or stop recording per-kernel CUDA-event times."""
        self._check(self.lib.pnuc_kernel_timing(self.handle, 1 if enable else 0))

    def kernel_times(self) -> dict:
        """Summed milliseconds of the cascade (or plain) kernel and of the evaporation kernel
        over the recorded launches, and their number."""
        c, v, n = C.c_double(), C.c_double(), C.c_uint64()
        self._check(self.lib.pnuc_kernel_times(self.handle, C.byref(c), C.byref(v), C.byref(n)))
        return dict(cascade_ms=c.value, evaporation_ms=v.value, launches=n.value)

    def tally(self, result: "Result", energies, T_range=(0.0, 250.0), n_T=125, n_cos=1, E_range=(20.0, 250.0),
              n_E=1, Z_max=100, A_max=250, hists=None, stream=None, n_secondaries: int | None = None):
        """pnuc_tally: yield histograms of a batch's results (int64 tensors on the device,
        accumulated into `hists` if given): secondaries [2 origins][6 species][n_cos][n_T] over
        T_range (MeV), residual nuclei [n_E][Z_max + 1][A_max + 1] over incident E_range.
        n_secondaries: the batch's record count if known (else it is read from the device)."""
        torch = self._torch
        dev = torch.device("cuda", self.device)
        if hists is None:
            hists = (torch.zeros((2, 6, n_cos, n_T), dtype=torch.int64, device=dev),
                     torch.zeros((n_E, Z_max + 1, A_max + 1), dtype=torch.int64, device=dev))
        spec = pnuc_tally_spec(n_T, n_cos, T_range[0], T_range[1], n_E, Z_max, E_range[0], E_range[1], A_max, 0)
        n = int(energies.shape[0])
        s = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        n_sec = min(result.n_secondaries() if n_secondaries is None else n_secondaries,
                    int(result.secondaries.shape[0]))
        self._check(self.lib.pnuc_tally(self.handle, C.byref(spec), _ptr(result.secondaries), n_sec,
                                        _ptr(result.residuals), _ptr(energies), n, _ptr(hists[0]), _ptr(hists[1]),
                                        C.c_void_p(s)))
        return hists

    @staticmethod
    def angle_windows(angles_deg=(7.5, 30.0, 60.0, 150.0), width_deg: float = 1.0):
        """cos theta edges of windows theta in (a - w/2, a + w/2] around the given angles
        (degrees): cos_lo = cos(a + w/2), cos_hi = cos(a - w/2); a window that reaches 0
        degrees keeps uz = 1."""
        import math
        lo, hi = [], []
        for a in angles_deg:
            t0, t1 = max(a - 0.5 * width_deg, 0.0), min(a + 0.5 * width_deg, 180.0)
            lo.append(-1.0 if t1 >= 180.0 else math.cos(math.radians(t1)))
            hi.append(math.nextafter(1.0, 2.0) if t0 <= 0.0 else math.cos(math.radians(t0)))
        return lo, hi

    def tally_windows(self, result: "Result", angles_deg=(7.5, 30.0, 60.0, 150.0), width_deg: float = 1.0,
                      T_range=(0.0, 250.0), n_T=125, hist=None, stream=None, n_secondaries: int | None = None,
                      cos_edges=None):
        """pnuc_tally_windows: secondary spectra in angular windows (the paper's Fig. 2), an
        int64 tensor [2 origins][6 species][windows][n_T] on the device (accumulated into
        `hist` if given). The windows are angle_windows(angles_deg, width_deg) unless
        cos_edges = (cos_lo, cos_hi) gives them."""
        torch = self._torch
        lo, hi = cos_edges if cos_edges is not None else self.angle_windows(angles_deg, width_deg)
        k = len(lo)
        if hist is None:
            hist = torch.zeros((2, 6, k, n_T), dtype=torch.int64, device=torch.device("cuda", self.device))
        s = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        n_sec = min(result.n_secondaries() if n_secondaries is None else n_secondaries,
                    int(result.secondaries.shape[0]))
        D = C.c_double * max(k, 1)
        self._check(self.lib.pnuc_tally_windows(self.handle, n_T, T_range[0], T_range[1], D(*lo), D(*hi), k,
                                                _ptr(result.secondaries), n_sec, _ptr(hist), C.c_void_p(s)))
        return hist

    def _structs(self, energies, target_ids, seed, first_event_id, out, projectiles=None, event_ids=None):
        b = pnuc_batch(_ptr(energies), _ptr(target_ids), int(energies.shape[0]), seed, first_event_id,
                       _ptr(projectiles) if projectiles is not None else None,
                       _ptr(event_ids) if event_ids is not None else None)
        o = pnuc_output(_ptr(out.secondaries), out.secondaries.shape[0], _ptr(out.count), _ptr(out.residuals),
                        _ptr(out.counters))
        return b, o

    def autotune(self, energies, target_ids, seed: int, precision: str = "fp32", reps: int = 2,
                 out: "Result | None" = None, stream=None) -> tuple[dict, float]:
        """pnuc_autotune on device tensors; returns (best tuning, its mean launch time in ms)."""
        torch = self._torch
        out = out or self.alloc(int(energies.shape[0]))
        b, o = self._structs(energies, target_ids, seed, 0, out)
        t, ms = pnuc_tuning(), C.c_double()
        s = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        self._check(self.lib.pnuc_autotune(self.handle, PRECISION[precision], C.byref(b), C.byref(o), reps,
                                           C.byref(t), C.byref(ms), C.c_void_p(s)))
        return {name: getattr(t, name) for name, _ in pnuc_tuning._fields_}, ms.value

    def save_tuning(self, path: str):
        self._check(self.lib.pnuc_save_tuning(self.handle, os.fsencode(path)))

    def load_tuning(self, path: str):
        self._check(self.lib.pnuc_load_tuning(self.handle, os.fsencode(path)))

    def graph(self, energies, target_ids, seed: int, out: "Result", first_event_id: int = 0,
              precision: str = "fp32", method: str = "persistent", projectiles=None, event_ids=None) -> "Graph":
        """pnuc_graph_create: a CUDA-graph plan of one launch for fixed buffers (optional
        projectiles uint8 and event_ids int64 device tensors, as in simulate)."""
        return Graph(self, energies, target_ids, seed, out, first_event_id, precision, method, projectiles, event_ids)

    def alloc(self, n: int, capacity: int | None = None, counters: bool = False) -> Result:
        torch = self._torch
        dev = torch.device("cuda", self.device)
        cap = int(capacity if capacity is not None else max(64, 40 * n))
        return Result(secondaries=torch.empty((cap, 32), dtype=torch.uint8, device=dev),
                      count=torch.zeros(1, dtype=torch.int64, device=dev),
                      residuals=torch.empty((max(n, 1), 64), dtype=torch.uint8, device=dev),
                      counters=torch.zeros(len(COUNTER_NAMES), dtype=torch.int64, device=dev) if counters else None)

    def simulate(self, energies, target_ids, seed: int, first_event_id: int = 0, precision: str = "fp32",
                 method: str = "persistent", out: Result | None = None, capacity: int | None = None,
                 counters: bool = False, stream=None, projectiles=None, event_ids=None) -> Result:
        """Launches pnuc_simulate on device tensors (energies float64, target_ids int32,
        optional projectiles uint8: 1 proton, 0 neutron; None = protons; optional event_ids
        int64, the id of each event in place of first_event_id + i). Asynchronous on `stream`
        (default: torch's current stream)."""
        torch = self._torch
        n = int(energies.shape[0])
        if energies.dtype != torch.float64 or target_ids.dtype != torch.int32:
            raise TypeError("energies must be float64 and target_ids int32 CUDA tensors")
        if not (energies.is_cuda and target_ids.is_cuda) or target_ids.shape[0] != n:
            raise ValueError("energies and target_ids must be CUDA tensors of equal length")
        energies = energies.contiguous()
        target_ids = target_ids.contiguous()
        if out is None:
            out = self.alloc(n, capacity, counters)
        pj = None
        if projectiles is not None:
            if projectiles.dtype != torch.uint8 or not projectiles.is_cuda or projectiles.shape[0] != n:
                raise ValueError("projectiles must be a uint8 CUDA tensor of the batch's length")
            pj = projectiles.contiguous()
        ids = None
        if event_ids is not None:
            if event_ids.dtype != torch.int64 or not event_ids.is_cuda or event_ids.shape[0] != n:
                raise ValueError("event_ids must be an int64 CUDA tensor of the batch's length")
            ids = event_ids.contiguous()
        b = pnuc_batch(_ptr(energies), _ptr(target_ids), n, seed, first_event_id, _ptr(pj) if pj is not None else None,
                       _ptr(ids) if ids is not None else None)
        o = pnuc_output(_ptr(out.secondaries), out.secondaries.shape[0], _ptr(out.count), _ptr(out.residuals),
                        _ptr(out.counters))
        s = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        self._check(self.lib.pnuc_simulate(self.handle, PRECISION[precision], METHOD[method], C.byref(b),
                                           C.byref(o), C.c_void_p(s)))
        return out

    def simulate_host(self, energies: np.ndarray, target_ids: np.ndarray, seed: int, first_event_id: int = 0,
                      precision: str = "fp32", method: str = "persistent", capacity: int | None = None,
                      sec_out: np.ndarray | None = None, res_out: np.ndarray | None = None, stream=None):
        """pnuc_simulate_host: host (ideally pinned) numpy buffers in and out; synchronous.
        Returns (secondaries, residuals) as numpy structured arrays."""
        torch = self._torch
        e = np.ascontiguousarray(energies, np.float64)
        t = np.ascontiguousarray(target_ids, np.int32)
        n = e.shape[0]
        cap = int(capacity if capacity is not None else max(64, 40 * n))
        sec = sec_out if sec_out is not None else np.empty(cap, SECONDARY_DTYPE)
        res = res_out if res_out is not None else np.empty(n, RESIDUAL_DTYPE)
        cnt = C.c_uint64()
        s = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        self._check(self.lib.pnuc_simulate_host(self.handle, PRECISION[precision], METHOD[method],
                                                e.ctypes.data, t.ctypes.data, n, seed, first_event_id,
                                                sec.ctypes.data, sec.shape[0], C.byref(cnt), res.ctypes.data,
                                                C.c_void_p(s)))
        return sec[: cnt.value], res[:n]


class Graph:
    """A CUDA-graph launch plan (pnuc_graph_*); keeps its buffers alive."""

    def __init__(self, ctx: Context, energies, target_ids, seed, out, first_event_id, precision, method,
                 projectiles=None, event_ids=None):
        self.ctx, self.handle = ctx, C.c_void_p()
        self._keep = (energies, target_ids, out, projectiles, event_ids)
        b, o = ctx._structs(energies, target_ids, seed, first_event_id, out, projectiles, event_ids)
        ctx._check(ctx.lib.pnuc_graph_create(ctx.handle, PRECISION[precision], METHOD[method], C.byref(b), C.byref(o),
                                             C.byref(self.handle)))
        self.out = out

    def update(self, energies, target_ids, seed, out, first_event_id=0, projectiles=None, event_ids=None):
        b, o = self.ctx._structs(energies, target_ids, seed, first_event_id, out, projectiles, event_ids)
        self.ctx._check(self.ctx.lib.pnuc_graph_update(self.handle, C.byref(b), C.byref(o)))
        self._keep = (energies, target_ids, out, projectiles, event_ids)
        self.out = out

    def launch(self, stream=None):
        torch = self.ctx._torch
        s = (stream or torch.cuda.current_stream(self.ctx.device)).cuda_stream
        self.ctx._check(self.ctx.lib.pnuc_graph_launch(self.handle, C.c_void_p(s)))
        return self.out

    def close(self):
        if self.handle:
            self.ctx.lib.pnuc_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving loop (pnuc_server_*): continuous batching with memory-based admission."""

    TIMEOUT = 5

    def __init__(self, ctx: Context, precision: str = "fp32", **cfg):
        self.ctx, self.lib, self.handle = ctx, ctx.lib, C.c_void_p()
        c = pnuc_server_config()
        self.lib.pnuc_server_default_config(C.byref(c))
        c.precision = PRECISION[precision]
        for k, v in cfg.items():
            setattr(c, k, int(v))
        ctx._check(self.lib.pnuc_server_create(ctx.handle, C.byref(c), C.byref(self.handle)))
        self.n_events: dict[int, int] = {}

    def submit(self, energies, target_ids, seed: int, first_event_id: int = 0, projectiles=None) -> int:
        """Queues a request (optional projectiles: uint8 per event, 1 proton, 0 neutron); returns
        its ticket. Raises PnucError (status 3) when the queue is full."""
        e = np.ascontiguousarray(energies, np.float64)
        t = np.ascontiguousarray(target_ids, np.int32)
        tk = C.c_uint64()
        if projectiles is None:
            self.ctx._check(self.lib.pnuc_server_submit(self.handle, e.ctypes.data, t.ctypes.data, len(e), seed,
                                                        first_event_id, C.byref(tk)))
        else:
            pj = np.ascontiguousarray(projectiles, np.uint8)
            if pj.shape[0] != len(e):
                raise ValueError("projectiles must have one entry per event")
            self.ctx._check(self.lib.pnuc_server_submit_nucleons(self.handle, e.ctypes.data, t.ctypes.data,
                                                                 pj.ctypes.data, len(e), seed, first_event_id,
                                                                 C.byref(tk)))
        self.n_events[tk.value] = len(e)
        return tk.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        """Number of secondaries of the finished request, or None on timeout."""
        n = C.c_uint64()
        st = self.lib.pnuc_server_wait(self.handle, ticket, timeout_ms, C.byref(n))
        if st == self.TIMEOUT:
            return None
        self.ctx._check(st)
        return n.value

    def wait_any(self, timeout_ms: int = -1):
        """Ticket of the next request to have finished (completion order), or None on timeout."""
        tk = C.c_uint64()
        st = self.lib.pnuc_server_wait_any(self.handle, timeout_ms, C.byref(tk))
        if st == self.TIMEOUT:
            return None
        self.ctx._check(st)
        return tk.value

    def fetch(self, ticket: int, n_secondaries: int):
        sec = np.empty(max(n_secondaries, 1), SECONDARY_DTYPE)
        res = np.empty(self.n_events.pop(ticket), RESIDUAL_DTYPE)
        self.ctx._check(self.lib.pnuc_server_fetch(self.handle, ticket, sec.ctypes.data, len(sec), res.ctypes.data))
        return sec[:n_secondaries], res

    def view(self, ticket: int):
        """Zero-copy results of a finished request: (secondaries, residuals) as numpy arrays
        over the server's pinned host arena, valid until release(ticket)."""
        sp, rp, n = C.c_void_p(), C.c_void_p(), C.c_uint64()
        self.ctx._check(self.lib.pnuc_server_view(self.handle, ticket, C.byref(sp), C.byref(n), C.byref(rp)))
        n_res = self.n_events[ticket]

        def arr(ptr, count, dtype):
            if count == 0:
                return np.empty(0, dtype)
            buf = (C.c_ubyte * (count * dtype.itemsize)).from_address(ptr.value)
            return np.frombuffer(buf, dtype=dtype, count=count)
        return arr(sp, n.value, SECONDARY_DTYPE), arr(rp, n_res, RESIDUAL_DTYPE)

    def release(self, ticket: int):
        self.ctx._check(self.lib.pnuc_server_release(self.handle, ticket))
        self.n_events.pop(ticket, None)

    def trace(self, enable: bool) -> None:
        """pnuc_server_trace: start (clearing) or stop the per-request trace."""
        self.ctx._check(self.lib.pnuc_server_trace(self.handle, 1 if enable else 0))

    def trace_read(self) -> np.ndarray:
        """The trace entries (TRACE_DTYPE), in release order."""
        n = C.c_uint64(0)
        self.ctx._check(self.lib.pnuc_server_trace_read(self.handle, None, 0, C.byref(n)))
        out = np.zeros(n.value, TRACE_DTYPE)
        if n.value:
            self.ctx._check(self.lib.pnuc_server_trace_read(self.handle, C.c_void_p(out.ctypes.data), n.value,
                                                            C.byref(n)))
        return out

    def stats(self) -> dict:
        st = pnuc_server_stats()
        self.ctx._check(self.lib.pnuc_server_get_stats(self.handle, C.byref(st)))
        return {name: getattr(st, name) for name, _ in pnuc_server_stats._fields_}

    def reset_stats(self):
        self.ctx._check(self.lib.pnuc_server_reset_stats(self.handle))

    def close(self):
        if self.handle:
            self.lib.pnuc_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sort_secondaries(sec: np.ndarray) -> np.ndarray:
    """Secondaries ordered by (event, index): the output order of a launch is not fixed."""
    return sec[np.lexsort((sec["index"], sec["event"]))]
