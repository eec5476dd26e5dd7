"""Benchmark: proton-nucleus events/s on one GB300 (intranuclear cascade + evaporation).

Workload per GPU (one "step" = one launch of the whole hot path over one batch):
1e6 proton-16O + 1e6 proton-40Ca events at 200 MeV (one batch of 2e6 events, two targets),
FP32 bulk mode (FP64 NN collision boosts, energy/momentum bookkeeping and evaporation widths
with their exponentials), persistent kernel with warp-level lane refill. Beside it: the scaled
FP32 mode (evaporation widths in FP32 too), the plain kernel, the FP64 mode, and the other
configurations' workloads (4e6 mixed targets from a graph, 1e6 per heavy target). The same batch is also timed with the plain one-event-per-thread
kernel ("batched vs plain"). Inputs are synthetic (seeded) and resident in HBM when the timed
region starts; the e2e figure goes through the host-buffer C-ABI entry point with the
host<->device transfers inside the timed region (inputs copied in; outputs written by the
kernels into the caller's pinned host buffers).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) each rank simulates its own event-id range (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "p-nucleus events/s on 1 GB300, batched vs plain at oracle match; p50/p99 latency"
UNIT = "events/s"
N_EACH = 1_000_000
ENERGY = 200.0
# paper Table 1 rows (5), GTX680 fast-math, 2.6e6 events each at 200 MeV: p-16O 6.61 s, p-40Ca 9.77 s
PAPER_EVENTS_PER_S = 2 * 2.6e6 / (6.61 + 9.77)
WORKLOAD = "1e6 p-16O + 1e6 p-40Ca at 200 MeV, one batch of 2e6 events per step"


def workload_name(n_each: int) -> str:
    """The workload's name; a run with another --n-each says so."""
    if n_each == N_EACH:
        return WORKLOAD
    return f"{n_each:.3g} p-16O + {n_each:.3g} p-40Ca at 200 MeV, one batch of {2 * n_each:.3g} events per step"

# Algorithmic FP64 operations of the FP32-mode model per counted unit: the operations the
# model performs in FP64 there (the NN collision boosts, the event's energy/momentum
# bookkeeping, the evaporation Q-values, and in the FP32 mode the evaporation widths with
# their exponentials and the channel draw), each add, multiply, fused multiply-add, compare,
# divide, square root, reciprocal square root or exponential counting as one operation.
# Conversions between float and double are not arithmetic (the kernels do them on the integer
# pipes). The units are the kernels' own counters.
CASCADE_FP64_OPS = {
    # the FP32 mode's collision (collide_mixed): pair sums 3, E1 and E_t 3, s 4, 1/sqrt(s) 1,
    # sqrt(s) 1, D = 1/(E_t + sqrt(s)) 2, the CM direction 8, p* 1, K 3, CM energies 4, P.K and
    # D P.K 4, the boost factors 4, q1 and q2 6, T1 and T2 6; the Pauli tests 2, the cutoffs 4
    "kinematics": 56,
    "escapes": 5,  # energy and momentum sums of an escaping nucleon
}
EVAP_FP64_OPS_COMMON = {
    "settled": 11,     # E* from the energy balance (p0 with its square root, the sums)
    "evap_passes": 6,  # excitations X = E* - Q of the six channels (Q tabulated per parent)
    # the parent's mass + E*, the release, the daughter's mass, and the parent's energy and
    # momentum bookkeeping
    "evap_steps": 9,
}
EVAP_FP64_OPS = {
    "fp32": {**EVAP_FP64_OPS_COMMON,
             # widths in FP64 from FP32 factors: per open channel with x >= 1 the exponential
             # and w0 (e^x A1 + A0), 3; with x < 1 the series runs in FP32 and the width
             # w0 (F q + G h) takes 3; the sum of the six and its test 6 per pass, the channel
             # draw 13 per step
             "evap_exps": 3, "evap_series": 3},
    # the widths, the channel draw, U_d and the decay with its boost are FP32 arithmetic
    "fp32_scaled": dict(EVAP_FP64_OPS_COMMON),
}
EVAP_FP64_OPS["fp32"]["evap_passes"] += 6
EVAP_FP64_OPS["fp32"]["evap_steps"] += 13
KERNEL_FILES = ("pnuc_device.cuh", "pnuc_kernels.cuh", "kernel_fp32.cu", "pnuc_internal.h", "fpconv.h")
PRECISION_NOTE = {
    "fp32": "fp32 bulk (transport, free paths, cross sections, evaporation channel parameters, emission sampler "
            "and decay); fp64 NN collision boosts, energy/momentum bookkeeping with the Q-values, and the "
            "evaporation widths with their exponentials and the channel draw",
    "fp32_scaled": "as fp32, but the evaporation widths and the channel draw in fp32 (each width scaled by the "
                   "largest channel's exponential)",
}


def measured_hbm_gbs():
    """Copy bandwidth of this machine's GB300 (driver-measured), or None."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return None


def strip_c_comments(text: str) -> str:
    """C/C++ source with its comments removed and each run of whitespace made one space:
    what the compiler sees, so that an edit to comments or layout alone keeps the hash."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c == "/" and i + 1 < n and text[i + 1] == "/":
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif c == "/" and i + 1 < n and text[i + 1] == "*":
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        elif c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_sha1() -> str:
    """Hash of the event kernels' sources without comments or layout (a profile summary taken
    at other sources is not used)."""
    import hashlib
    h = hashlib.sha1()
    for f in KERNEL_FILES:
        h.update(strip_c_comments(open(os.path.join(ROOT, "paper_1309_7963_gb300", "csrc", f)).read()).encode())
    return h.hexdigest()


def profile_values() -> dict:
    """The last ncu captures of the FP32 cascade and evaporation kernels
    (profiles/persistent_kernels_traffic.txt): per kernel, DRAM bytes per event, issue-slot use,
    active threads per instruction and FP64-pipe use; empty if the kernel sources changed since."""
    path = os.path.join(ROOT, "profiles", "persistent_kernels_traffic.txt")
    if not os.path.exists(path):
        return {}
    kv = dict(line.strip().split(": ", 1) for line in open(path) if ": " in line and not line.startswith("#"))
    if kv.get("kernel_sha1", "") != kernel_sha1():
        return {}
    out = {}
    for k in ("cascade", "evaporation"):
        out[k] = {f: float(kv[f"{k}_{f}"]) for f in ("bytes_per_event", "issue_active_pct", "threads_per_inst",
                                                     "fp64_pipe_pct", "warp_inst_per_event") if f"{k}_{f}" in kv}
    return out


def fp64_ops_per_event(counters: dict, n_events: int, precision: str = "fp32") -> dict:
    cas = sum(counters[k] * v for k, v in CASCADE_FP64_OPS.items()) / n_events
    eva = sum(counters[k] * v for k, v in EVAP_FP64_OPS[precision].items()) / n_events
    return {"cascade": cas, "evaporation": eva}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-each", type=int, default=N_EACH)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-divergence", action="store_true")
    ap.add_argument("--no-others", action="store_true")
    return ap.parse_args()


def dist_env():
    from paper_1309_7963_gb300 import dist
    return dist.env()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.reader.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def serving_bench(ctx, seconds: float = 3.0) -> dict:
    """The serving loop under the synthetic transport driver: capacity from a saturating
    burst, then Poisson arrivals at 50%, 75% and 90% of it; p50/p99 from submit to results."""
    import time as _t

    from paper_1309_7963_gb300 import driver, inputs, pnuc
    tids = np.array([ctx.create_target(*za) for za in inputs.SERVING_TARGETS], np.int32)
    srv = pnuc.Server(ctx, precision="fp32", streams=16, arena_bytes=2 << 30)
    try:
        burst = inputs.serving_requests(256, rate_hz=1e9, seed=101)
        driver.run(srv, burst[:16], tids, seed=7)  # warm-up
        srv.reset_stats()
        rep = driver.run(srv, burst, tids, seed=7)
        capacity = rep["events_per_s"]
        mean_events = float(np.mean([len(r["energies"]) for r in burst]))
        runs = []
        for load in (0.5, 0.75, 0.9):
            rate = load * capacity / mean_events
            n_req = max(40, int(rate * seconds))
            reqs = inputs.serving_requests(n_req, rate_hz=rate, seed=200 + int(100 * load))
            srv.reset_stats()
            srv.trace(True)
            r = driver.run(srv, reqs, tids, seed=7)
            srv.trace(False)
            st = srv.stats()
            where = driver.attribute(srv.trace_read())
            runs.append({"load": load, "offered_events_per_s": rate * mean_events, "requests": r["requests"],
                         "events_per_s": r["events_per_s"], "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"],
                         "max_ms": r["max_ms"], "server_p50_ms": st["latency_p50_ms"],
                         "server_p99_ms": st["latency_p99_ms"], "queue_p99_ms": st["queue_p99_ms"],
                         "reruns": st["reruns"], "latency_phases": where})
        return {"capacity_events_per_s": capacity, "mean_request_events": mean_events,
                "config": "Poisson arrivals, 1e3-1e5 events log-uniform, 20-250 MeV, 12C/16O/40Ca/48Ti/56Fe, "
                          "16 streams, 2 GiB arenas, FP32; capacity from a burst of 256 requests; same-seed "
                          "requests merged up to 32 and 2^18 events per launch, 4 events per lane",
                "runs": runs}
    finally:
        srv.close()


def divergence_bound(ctx, n: int = 1_000_000, run: int = 32, reps: int = 3) -> dict:
    """The paper's divergence experiment (§3: every thread given the same random state ran
    p-12C events 4x (70 MeV) and 5x (200 MeV) faster): each workload is timed once with
    distinct event ids and once with runs of `run` lanes sharing one id (warp-uniform, so
    no lane of a warp diverges from the others; the runs still sample n / run different
    events, so the mix of event costs is kept). FP32 mode, plain kernel and persistent
    method; events/s and the ratio uniform / distinct."""
    import torch

    from paper_1309_7963_gb300 import inputs
    cases = [("p-12C 70 MeV", inputs.C12, 70.0), ("p-12C 200 MeV", inputs.C12, 200.0),
             ("p-16O 200 MeV", inputs.O16, 200.0), ("p-40Ca 200 MeV", inputs.CA40, 200.0)]
    out = {"run": run, "events": n, "cases": {}}
    res_cap = ctx.alloc(n, capacity=16 * n)
    stream = torch.cuda.current_stream()
    for name, target, energy in cases:
        tid = ctx.create_target(*target)
        e = torch.full((n,), energy, dtype=torch.float64, device="cuda")
        t = torch.full((n,), tid, dtype=torch.int32, device="cuda")
        first = 1 << 40
        ids = {"distinct": None, "uniform": first + torch.arange(n, device="cuda", dtype=torch.int64) // run}
        row = {}
        for method in ("plain", "persistent"):
            for kind, ev_ids in ids.items():
                ctx.simulate(e, t, seed=5, first_event_id=first, method=method, out=res_cap, event_ids=ev_ids)
                torch.cuda.synchronize()
                best = None
                for _ in range(reps):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    ctx.simulate(e, t, seed=5, first_event_id=first, method=method, out=res_cap, event_ids=ev_ids)
                    b.record(stream)
                    torch.cuda.synchronize()
                    ms = a.elapsed_time(b)
                    best = ms if best is None else min(best, ms)
                row[f"{method}_{kind}"] = n / (best * 1e-3)
            row[f"{method}_ratio"] = row[f"{method}_uniform"] / row[f"{method}_distinct"]
        out["cases"][name] = row
    return out


def other_workloads(ctx, flush, reps: int = 5, warm: int = 3) -> dict:
    """The other configurations' workloads, each timed with CUDA events on the launching
    stream (median of `reps` launches after `warm`, L2 flushed before each): 4e6 events on the
    mixed tissue targets at 20-250 MeV (one persistent launch with the autotuner's tuning,
    replayed from a CUDA graph) and 1e6 events on each heavy target at 100-250 MeV (persistent
    method), FP32 mode, each beside the plain kernel on the same batch."""
    import torch

    from paper_1309_7963_gb300 import inputs
    stream = torch.cuda.current_stream()

    def median_ms(fn, r=reps, wu=warm):
        for _ in range(wu):
            fn()
        torch.cuda.synchronize()
        ts = []
        for k in range(r):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    res = {}
    w = inputs.mixed(4_000_000, seed=0)
    tids = np.array([ctx.create_target(*za) for za in w.targets], np.int32)
    e = torch.tensor(w.energies, device="cuda")
    t = torch.tensor(tids[w.tidx], device="cuda")
    buf = ctx.alloc(w.n, capacity=8 * w.n)
    saved = ctx.get_tuning("fp32")
    try:
        best, _ = ctx.autotune(e, t, seed=w.seed, precision="fp32", reps=1)
        g = ctx.graph(e, t, seed=w.seed, out=buf, precision="fp32")
        ms = median_ms(g.launch)
        g.close()
    finally:
        ctx.set_tuning("fp32", **saved)
    pms = median_ms(lambda: ctx.simulate(e, t, seed=w.seed, precision="fp32", method="plain", out=buf), r=3, wu=1)
    res["mixed_4e6_graph_autotuned"] = {
        "workload": "4e6 events, 20-250 MeV, 60% 16O / 20% 12C / 10% 14N / 5% 40Ca / 5% 31P, one persistent "
                    "launch replayed from a CUDA graph with the autotuned tuning",
        "tuning": best, "ms": ms, "value": w.n / (ms * 1e-3), "plain_ms": pms, "plain_value": w.n / (pms * 1e-3),
        "batched_vs_plain": pms / ms}
    del buf, e, t
    for target in (inputs.TI48, inputs.FE56, inputs.PB208):
        w = inputs.heavy(target, 1_000_000, seed=3)
        tids = np.array([ctx.create_target(*za) for za in w.targets], np.int32)
        e = torch.tensor(w.energies, device="cuda")
        t = torch.tensor(tids[w.tidx], device="cuda")
        buf = ctx.alloc(w.n, capacity=24 * w.n)
        ms = median_ms(lambda: ctx.simulate(e, t, seed=w.seed, precision="fp32", method="persistent", out=buf))
        pms = median_ms(lambda: ctx.simulate(e, t, seed=w.seed, precision="fp32", method="plain", out=buf), r=3, wu=1)
        res[f"heavy_{target[1]}_1e6"] = {
            "workload": f"1e6 events on (Z, A) = {target}, 100-250 MeV, persistent method", "ms": ms,
            "value": w.n / (ms * 1e-3), "plain_ms": pms, "plain_value": w.n / (pms * 1e-3),
            "batched_vs_plain": pms / ms}
        del buf, e, t
    return res


def level_density_cost(w, first, flush, steps: int = 3) -> dict:
    """The bench batch with the constant-temperature level density below U_x (reading M26,
    pnuc_config.level_density = 1) against the default Fermi gas: events/s of the persistent
    method in the FP32 and FP64 modes, each in its own context, CUDA events, L2 flushed."""
    import torch

    from paper_1309_7963_gb300 import pnuc
    stream = torch.cuda.current_stream()
    out = {}
    for ld in (0, 1):
        c = pnuc.Context(torch.cuda.current_device(), level_density=ld)
        tids = np.array([c.create_target(*za) for za in w.targets], np.int32)
        e = torch.tensor(w.energies, dtype=torch.float64, device="cuda")
        t = torch.tensor(tids[w.tidx], dtype=torch.int32, device="cuda")
        buf = c.alloc(w.n, capacity=8 * w.n)
        for prec in ("fp32", "fp64"):
            c.simulate(e, t, seed=w.seed, first_event_id=first, precision=prec, out=buf)
            torch.cuda.synchronize()
            ms = []
            for k in range(steps):
                flush.fill_(float(k))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                c.simulate(e, t, seed=w.seed, first_event_id=first, precision=prec, out=buf)
                b.record(stream)
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            out[f"{'fermi_gas' if ld == 0 else 'constant_temperature'}_{prec}"] = w.n / (float(np.median(ms)) * 1e-3)
        del buf
        c.close()
    out["unit"] = UNIT
    return out


def cpu_baseline(n_each: int, threads: int | None = None) -> dict:
    """The CPU oracle, as it stands, on a bounded sample of the workload."""
    import oracle
    from paper_1309_7963_gb300 import inputs
    w = inputs.oxygen_calcium(n_each=n_each, energy=ENERGY)
    oracle.lib()
    t0 = time.perf_counter()
    r = oracle.simulate_parallel(w.targets, w.energies, w.tidx, seed=w.seed, threads=threads, keep=False)
    dt = time.perf_counter() - t0
    return {"value": w.n / dt, "unit": UNIT, "cores": r["threads"], "kind": "oracle",
            "sample": f"{n_each} p-16O + {n_each} p-40Ca events at 200 MeV (first ids of the workload), "
                      f"{dt:.2f} s on {r['threads']} host threads",
            "seconds": dt, "events": w.n}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    n_each = 100_000
    for _ in range(args.warmup):
        cpu_baseline(n_each // 10)
    vals = []
    for _ in range(args.steps):
        vals.append(cpu_baseline(n_each))
    v = float(np.median([x["value"] for x in vals]))
    cb = dict(vals[-1])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * 2 * n_each / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "step_sample": f"{2 * n_each} events per step"},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch

    from paper_1309_7963_gb300 import inputs, pnuc

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    ctx = pnuc.Context(local)
    w = inputs.oxygen_calcium(n_each=args.n_each, energy=ENERGY)
    tids = np.array([ctx.create_target(*za) for za in w.targets], np.int32)
    n = w.n
    from paper_1309_7963_gb300 import dist as pdist
    first = pdist.shard_first_event_id(rank, n)  # weak scaling: each rank its own event-id range
    e_dev = torch.tensor(w.energies, dtype=torch.float64, device="cuda")
    t_dev = torch.tensor(tids[w.tidx], dtype=torch.int32, device="cuda")
    cap = 8 * n
    out = ctx.alloc(n, capacity=cap)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def timed(method, steps, warmup, per_kernel=False, precision="fp32"):
        for _ in range(warmup):
            ctx.simulate(e_dev, t_dev, seed=w.seed, first_event_id=first, precision=precision, method=method, out=out)
        torch.cuda.synchronize()
        ctx.kernel_timing(per_kernel)  # CUDA events around each kernel, on the launching stream
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for k in range(steps):
            flush.fill_(float(k))  # L2 flush between steps
            ev[k][0].record(stream)
            ctx.simulate(e_dev, t_dev, seed=w.seed, first_event_id=first, precision=precision, method=method, out=out)
            ev[k][1].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        total_ms = t_start.elapsed_time(t_end)
        kern_ms = [a.elapsed_time(b) for a, b in ev]
        return total_ms, kern_ms

    clocks = ClockSampler(local)
    clocks.start()
    total_ms, kern_ms = timed("persistent", args.steps, args.warmup, per_kernel=True)
    ctx.kernel_timing(False)
    ktimes = ctx.kernel_times()
    total_ms = pdist.max_over_ranks(total_ms, device="cuda")
    n_sec = out.n_secondaries()
    res = out.residuals_np()
    value = world * n * args.steps / (total_ms * 1e-3)
    launch_ms = float(np.mean(kern_ms))

    # the same batch with the evaporation widths and the channel draw in FP32 (scaled widths)
    s_steps = max(2, args.steps // 2)
    s_total, _ = timed("persistent", s_steps, args.warmup, per_kernel=True, precision="fp32_scaled")
    ctx.kernel_timing(False)
    s_kt = ctx.kernel_times()
    s_total = pdist.max_over_ranks(s_total, device="cuda")
    scaled = {"value": world * n * s_steps / (s_total * 1e-3), "unit": UNIT, "ms_per_step": s_total / s_steps,
              "steps": s_steps, "precision": PRECISION_NOTE["fp32_scaled"],
              "cascade_ms": s_kt["cascade_ms"] / max(1, s_kt["launches"]),
              "evaporation_ms": s_kt["evaporation_ms"] / max(1, s_kt["launches"])}

    plain = None
    if not args.no_plain:
        p_total, p_kern = timed("plain", max(2, args.steps // 2), 1)
        plain = {"value": world * n * max(2, args.steps // 2) / (p_total * 1e-3), "unit": UNIT,
                 "ms_per_step": p_total / max(2, args.steps // 2)}

    # the FP64 deterministic mode (per-event oracle parity) on the same batch: batched vs plain
    fp64 = None
    if not args.no_plain:
        f_pers, _ = timed("persistent", 2, 1, precision="fp64")
        f_sort, _ = timed("sorted", 2, 1, precision="fp64")
        f_plain, _ = timed("plain", 2, 1, precision="fp64")
        fp64 = {"persistent": world * n * 2 / (f_pers * 1e-3), "sorted": world * n * 2 / (f_sort * 1e-3),
                "plain": world * n * 2 / (f_plain * 1e-3), "unit": UNIT,
                "batched_vs_plain": f_plain / min(f_pers, f_sort)}
    others = None if (args.no_others or world > 1) else other_workloads(ctx, flush)
    # the composite level density (reading M26, a context option) on the same batch
    level_ct = None
    if not (args.no_others or world > 1):
        level_ct = level_density_cost(w, first, flush)
    clk = clocks.stop()

    e2e = None
    if not args.no_e2e:
        # same metric through the host-buffer entry point: H2D of inputs, D2H of results inside
        e_h = torch.tensor(w.energies, dtype=torch.float64).pin_memory().numpy()
        t_h = torch.tensor(tids[w.tidx], dtype=torch.int32).pin_memory().numpy()
        sec_h = torch.empty((cap, 32), dtype=torch.uint8).pin_memory().numpy().reshape(-1).view(pnuc.SECONDARY_DTYPE)
        res_h = torch.empty((n, 64), dtype=torch.uint8).pin_memory().numpy().reshape(-1).view(pnuc.RESIDUAL_DTYPE)
        ctx.simulate_host(e_h, t_h, seed=w.seed, first_event_id=first, sec_out=sec_h, res_out=res_h)
        steps_e2e = max(2, args.steps // 2)
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(steps_e2e):
            sec, _ = ctx.simulate_host(e_h, t_h, seed=w.seed, first_event_id=first, sec_out=sec_h, res_out=res_h)
        dt = time.perf_counter() - t0
        e2e = {"value": world * n * steps_e2e / dt, "unit": UNIT, "h2d_bytes_per_step": int(e_h.nbytes + t_h.nbytes),
               "d2h_bytes_per_step": int(res_h.nbytes + len(sec) * 32 + 8),
               "path": "pnuc_simulate_host with pinned host buffers: inputs copied in, residuals and "
                       "secondaries written by the kernels into the pinned buffers (mapped host memory), "
                       "host wall clock per call"}

    # yield tallies of the last step's outputs (an HBM-streaming pass): L2 flushed before each
    tally = None
    if rank == 0:
        hbm_peak = measured_hbm_gbs()
        n_sec_out = min(out.n_secondaries(), cap)
        hs = (torch.zeros((2, 6, 1, 125), dtype=torch.int64, device="cuda"),
              torch.zeros((1, 31, 65), dtype=torch.int64, device="cuda"))
        tms = []
        for k in range(8):
            torch.cuda.synchronize()
            flush.fill_(float(k))  # the L2 flush also covers the host's launch of the tally
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.tally(out, e_dev, n_T=125, n_cos=1, n_E=1, E_range=(199.0, 201.0), Z_max=30, A_max=64, hists=hs,
                      n_secondaries=n_sec_out)
            b.record(stream)
            torch.cuda.synchronize()
            tms.append(a.elapsed_time(b))
        t_ms = float(np.median(tms[3:]))
        # the paper's Fig. 2 spectra: 1-degree windows at 7.5, 30, 60 and 150 degrees
        hw = torch.zeros((2, 6, 4, 125), dtype=torch.int64, device="cuda")
        twm = []
        for k in range(8):
            torch.cuda.synchronize()
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.tally_windows(out, hist=hw, n_secondaries=n_sec_out)
            b.record(stream)
            torch.cuda.synchronize()
            twm.append(a.elapsed_time(b))
        tw_ms = float(np.median(twm[3:]))
        del hw
        tbytes = 32 * n_sec_out + (32 + 8) * n
        # what DRAM delivers: HBM reads the residual records whole (64 bytes, of which the
        # kernel asks for the first 32), so 72 bytes per event instead of 40
        dbytes = 32 * n_sec_out + (64 + 8) * n
        tally = {"ms": t_ms, "algorithmic_bytes": tbytes, "GB_s": tbytes / (t_ms * 1e-3) / 1e9,
                 "hbm_peak_GB_s": hbm_peak, "frac": (tbytes / (t_ms * 1e-3) / 1e9) / hbm_peak if hbm_peak else None,
                 "dram_bytes": dbytes, "dram_GB_s": dbytes / (t_ms * 1e-3) / 1e9,
                 "fig2_windows": {"ms": tw_ms, "GB_s": 32 * n_sec_out / (tw_ms * 1e-3) / 1e9,
                                  "spec": "secondaries in 1-degree windows at 7.5, 30, 60, 150 degrees x 125 T bins"},
                 "spec": "secondaries 2 x 6 x 125 T bins (2 MeV, angle-integrated as in the paper's Fig. 1; "
                         "shared-memory counters), residuals 1 x 31 x 65 (Z, A) (shared-memory counters); "
                         "L2 flushed before each launch, the host's launch hidden behind the flush",
                 "secondaries": int(n_sec_out), "events": n}
        del hs

    # algorithmic work per event from the kernel's own counters (one counting launch)
    cnt = ctx.simulate(e_dev, t_dev, seed=w.seed, first_event_id=first, precision="fp32", method="persistent",
                       counters=True, capacity=cap)
    torch.cuda.synchronize()
    counters = cnt.counters_dict()
    del cnt
    ops_ev = fp64_ops_per_event(counters, n, "fp32")
    ops_ev_scaled = fp64_ops_per_event(counters, n, "fp32_scaled")
    peaks = ctx.measure_peaks()
    kernels = {}
    prof = profile_values()
    for name, ms_key in (("cascade", "cascade_ms"), ("evaporation", "evaporation_ms")):
        ms = ktimes[ms_key] / max(1, ktimes["launches"])
        achieved = ops_ev[name] * n / (ms * 1e-3)
        pk = prof.get(name, {})
        kernels[name] = {"ms_per_launch": ms, "fp64_ops_per_event": ops_ev[name], "achieved": achieved / 1e9,
                         "frac": achieved / peaks["fp64_fma"],
                         "traffic": pk["bytes_per_event"] * n if "bytes_per_event" in pk else None,
                         "ncu": {k: v for k, v in pk.items() if k != "bytes_per_event"} or None}
    # the issue-rate roofline: warp instructions per event (ncu capture of the same kernel
    # sources) x events per second of this run, against one warp instruction per cycle on
    # each of the 4 schedulers of every SM at the SM clock sampled during the timed region
    sm_hz = ((clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz") or 0) * 1e6
    issue_peak = 4 * torch.cuda.get_device_properties(local).multi_processor_count * sm_hz
    for name in kernels:
        ipe = prof.get(name, {}).get("warp_inst_per_event")
        if ipe and issue_peak > 0:
            rate = ipe * n / (kernels[name]["ms_per_launch"] * 1e-3)
            kernels[name]["issue"] = {"warp_inst_per_event": ipe, "achieved": rate / 1e9, "peak": issue_peak / 1e9,
                                      "unit": "G warp-inst/s", "frac": rate / issue_peak}
        else:
            kernels[name]["issue"] = None
    scaled["evaporation_fp64_ops_per_event"] = ops_ev_scaled["evaporation"]
    scaled["evaporation_fp64_frac"] = (ops_ev_scaled["evaporation"] * n / (scaled["evaporation_ms"] * 1e-3)
                                       / peaks["fp64_fma"]) if scaled["evaporation_ms"] > 0 else None
    top = max(kernels, key=lambda k: kernels[k]["ms_per_launch"])
    kt = kernels[top]
    roofline = {"bound": "alu", "pipe": "fp64", "kernel": f"{top} kernel (FP32 mode)", "achieved": kt["achieved"],
                "peak": peaks["fp64_fma"] / 1e9, "unit": "FP64 Gop/s", "frac": kt["frac"], "traffic": kt["traffic"],
                "traffic_note": "DRAM bytes per launch, scaled by events from an ncu capture of 8e5 events; "
                                "ncu: issue-slot use and active threads per instruction of the same capture",
                "peak_source": "pnuc_measure_peaks, FP64 FMA lane-ops/s measured in this run",
                "issue_rate": kt["issue"],
                "timed_launches": ktimes["launches"], "kernels": kernels, "peaks_lane_ops_per_s": peaks,
                "work_per_event": {k: v / n for k, v in counters.items() if not k.startswith("cycles")}}
    cyc = {k[7:]: counters[k] for k in counters if k.startswith("cycles_")}
    phase_split = {k: v / max(1, sum(cyc.values())) for k, v in cyc.items()}
    serving = None if (args.no_serving or world > 1) else serving_bench(ctx)
    divergence = None if (args.no_divergence or world > 1) else divergence_bound(ctx)
    if rank != 0:
        return
    cb = None
    if not args.no_cpu:
        cb = cpu_baseline(500_000)
        one = cpu_baseline(50_000, threads=1)
        cb["one_core"] = {"value": one["value"], "unit": UNIT, "cores": 1, "sample": one["sample"]}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / PAPER_EVENTS_PER_S, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": workload_name(n // 2), "events_per_step": n, "precision": PRECISION_NOTE["fp32"],
                   "method": "persistent (warp refill)", "tuning": ctx.get_tuning("fp32"),
                   "l2": "256 MiB buffer written between steps (inside the timed region)",
                   "parallelism": f"{world} rank(s), event-id ranges, no collective"},
        "launch_ms": launch_ms, "secondaries_per_step": n_sec,
        "flags_nonzero_fraction": float(np.mean(res["flags"] != 0)),
        "plain": plain, "batched_vs_plain": (value / plain["value"]) if plain else None, "fp64_mode": fp64,
        "fp32_scaled_mode": scaled, "other_workloads": others, "level_density_option": level_ct,
        "phase_split": phase_split,
        "p50_ms": serving["runs"][-1]["p50_ms"] if serving else None,
        "p99_ms": serving["runs"][-1]["p99_ms"] if serving else None,
        "latency_load": serving["runs"][-1]["load"] if serving else None,  # fraction of capacity
        "serving": serving,
        "e2e": e2e, "roofline": roofline, "cpu_baseline": cb, "clocks": clk, "gpu_launches": 2 * args.steps,
        "tally": tally, "divergence_bound": divergence,
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
