"""Synthetic proton-transport driver for the serving loop (pnuc_server): it submits
interaction requests at Poisson arrival times (inputs.serving_requests: 1e3-1e5 events,
log-uniform; 20-250 MeV; 12C, 16O, 40Ca, 48Ti, 56Fe), and a consumer thread waits for each
result, reads it in place (zero-copy views of the server's pinned arena) and releases it, as
a transport code would before it continues its histories."""
from __future__ import annotations

import gc
import threading
import time

import numpy as np

from . import inputs
from .pnuc import PnucError, Server


def run(server: Server, requests: list, target_ids: np.ndarray, seed: int, keep=None, time_limit_s: float = 120.0,
        pause_gc: bool = True):
    """Plays `requests` against `server` in real time. target_ids maps the workload's target
    index to the context's target id. keep(request, secondaries, residuals) is called for
    each result if given, with views valid only during the call (copy what you keep).
    Results are taken in the order they finish (pnuc_server_wait_any), as a transport code
    continues whichever histories are ready. Python's cyclic garbage collector is paused while
    the requests play (pause_gc): a full collection in a process that has loaded torch holds
    every thread for tens of milliseconds, which the trace showed as 30-36 ms client stalls.
    Returns client-side latencies (ms, submit to release) and throughput."""
    done = {}
    meta = {}  # ticket -> (request, submit time)
    lock = threading.Condition()
    finished = [False]
    t0 = time.perf_counter()

    def consumer():
        while True:
            with lock:
                if finished[0] and len(done) >= len(meta):
                    return
            tk = server.wait_any(20)
            if tk is None:
                continue
            with lock:  # the submitting thread records the ticket just after submit returns
                while tk not in meta:
                    lock.wait(0.001)
                req, t_sub = meta[tk]
            sec, res = server.view(tk)  # zero-copy: the results where they landed
            if keep is not None:
                keep(req, sec, res)
            server.release(tk)
            with lock:
                done[tk] = (t_sub, time.perf_counter(), req["energies"].shape[0])

    gc_was_on = gc.isenabled()
    if pause_gc:
        gc.disable()
    th = threading.Thread(target=consumer, daemon=True)
    th.start()
    for req in requests:
        delay = t0 + req["arrival"] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        if time.perf_counter() - t0 > time_limit_s:
            break
        while True:
            try:
                tk = server.submit(req["energies"], target_ids[req["tidx"]], seed, req["first_event_id"])
                break
            except PnucError as e:  # queue full: the driver backs off
                if e.status != 3:
                    raise
                time.sleep(0.001)
        with lock:
            meta[tk] = (req, time.perf_counter())
            lock.notify_all()
    with lock:
        finished[0] = True
        lock.notify_all()
    th.join()
    wall = time.perf_counter() - t0
    if pause_gc and gc_was_on:
        gc.enable()
    lat = np.array([(b - a) * 1e3 for a, b, _ in done.values()])
    events = sum(n for _, _, n in done.values())
    first = min(a for a, _, _ in done.values())
    last = max(b for _, b, _ in done.values())
    return dict(requests=len(done), events=events, wall_s=wall, events_per_s=events / (last - first),
                p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                max_ms=float(lat.max()))


PHASES = ("queue", "host_launch", "gpu_wait", "gpu_run", "detect", "client")


def phase_times(trace: np.ndarray) -> dict:
    """Per request (pnuc_server_trace entries), the milliseconds of each phase of its latency:
    queue (submit to admission), host_launch (admission to its launch enqueued), gpu_wait (to
    the GPU starting it), gpu_run (the launch on the GPU), detect (to the server seeing it
    complete), client (to the client's release)."""
    t = trace
    return {"queue": t["t_admit"] - t["t_submit"], "host_launch": t["t_launched"] - t["t_admit"],
            "gpu_wait": t["t_gpu_start"] - t["t_launched"], "gpu_run": t["t_gpu_end"] - t["t_gpu_start"],
            "detect": t["t_complete"] - t["t_gpu_end"], "client": t["t_release"] - t["t_complete"]}


def attribute(trace: np.ndarray, slow_ms: float = 20.0) -> dict:
    """Where the latency of the slow requests (submit to release above slow_ms) went: for each
    phase, how many slow requests it dominated and its mean over them; and each phase's p50 and
    p99 over all requests."""
    if len(trace) == 0:
        return {}
    ph = phase_times(trace)
    total = trace["t_release"] - trace["t_submit"]
    slow = total > slow_ms
    stack = np.stack([ph[k] for k in PHASES], 1)
    dom = np.argmax(stack, 1)
    out = {"requests": int(len(trace)), "slow_ms": slow_ms, "slow": int(slow.sum()),
           "dominant": {k: int(((dom == i) & slow).sum()) for i, k in enumerate(PHASES)},
           "mean_in_slow_ms": {k: float(ph[k][slow].mean()) if slow.any() else 0.0 for k in PHASES},
           "p50_ms": {k: float(np.percentile(ph[k], 50)) for k in PHASES},
           "p99_ms": {k: float(np.percentile(ph[k], 99)) for k in PHASES},
           "max_ms": {k: float(ph[k].max()) for k in PHASES}}
    return out


def make_requests(n_requests: int, rate_hz: float, seed: int = 0):
    return inputs.serving_requests(n_requests, rate_hz, seed=seed)
