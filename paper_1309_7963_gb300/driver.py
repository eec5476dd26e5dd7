"""Synthetic proton-transport driver for the serving loop (pnuc_server): it submits
interaction requests at Poisson arrival times (inputs.serving_requests: 1e3-1e5 events,
log-uniform; 20-250 MeV; 12C, 16O, 40Ca, 48Ti, 56Fe), and a consumer thread waits for each
result, reads it in place (zero-copy views of the server's pinned arena) and releases it, as
a transport code would before it continues its histories."""
from __future__ import annotations

import threading
import time

import numpy as np

from . import inputs
from .pnuc import PnucError, Server


def run(server: Server, requests: list, target_ids: np.ndarray, seed: int, keep=None, time_limit_s: float = 120.0):
    """Plays `requests` against `server` in real time. target_ids maps the workload's target
    index to the context's target id. keep(request, secondaries, residuals) is called for
    each result if given, with views valid only during the call (copy what you keep).
    Results are taken in the order they finish (pnuc_server_wait_any), as a transport code
    continues whichever histories are ready. Returns client-side latencies (ms, submit to
    release) and throughput."""
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
    lat = np.array([(b - a) * 1e3 for a, b, _ in done.values()])
    events = sum(n for _, _, n in done.values())
    first = min(a for a, _, _ in done.values())
    last = max(b for _, b, _ in done.values())
    return dict(requests=len(done), events=events, wall_s=wall, events_per_s=events / (last - first),
                p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                max_ms=float(lat.max()))


def make_requests(n_requests: int, rate_hz: float, seed: int = 0):
    return inputs.serving_requests(n_requests, rate_hz, seed=seed)
