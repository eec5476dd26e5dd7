"""Seeded synthetic workloads: incident energies and target indices for batches of events.

This module holds none of the model's arithmetic. It only draws the inputs (energies in
MeV, target index per event) that the paper's workloads describe (§4: 70 and 200 MeV
protons on ¹⁶O and ⁴⁰Ca; therapeutic nuclei; 20–250 MeV, §1), with numpy's Philox
generator on a key of its own so that the inputs never overlap the physics draws.
The CUDA path and the oracle both consume what it returns.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# (Z, A) of the target nuclei the workloads use
O16, C12, N14, CA40, P31, TI48, FE56, PB208 = (8, 16), (6, 12), (7, 14), (20, 40), (15, 31), (22, 48), (26, 56), (82, 208)
_INPUT_KEY_TAG = 0x494E505554  # keeps the input stream apart from the physics key (seed, 0)


@dataclass
class Workload:
    name: str
    targets: list          # list of (Z, A); tidx indexes it
    energies: np.ndarray   # float64, MeV
    tidx: np.ndarray       # int32
    seed: int              # physics seed (Philox key)
    first_event_id: int = 0

    @property
    def n(self) -> int:
        return int(self.energies.shape[0])

    def slice(self, start: int, stop: int) -> "Workload":
        return Workload(self.name, self.targets, self.energies[start:stop], self.tidx[start:stop],
                        self.seed, self.first_event_id + start)


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[seed, _INPUT_KEY_TAG + stream]))


def fixed(target, energy: float, n: int, seed: int = 0, first_event_id: int = 0, name=None) -> Workload:
    """n events at one energy on one target (the plain-method workloads)."""
    return Workload(name or f"p-{target} {energy} MeV", [tuple(target)], np.full(n, float(energy)),
                    np.zeros(n, np.int32), seed, first_event_id)


def plain_fp64(n: int = 10_000) -> Workload:
    """1e4 protons on ¹⁶O at exactly 200 MeV, Philox seed 0 (per-event parity workload)."""
    return fixed(O16, 200.0, n, seed=0, name="p-16O 200 MeV")


def oxygen_calcium(n_each: int = 1_000_000, energy: float = 200.0, seed: int = 0) -> Workload:
    """n_each p–¹⁶O then n_each p–⁴⁰Ca events at one energy (one batch, two targets)."""
    e = np.full(2 * n_each, float(energy))
    t = np.concatenate([np.zeros(n_each, np.int32), np.ones(n_each, np.int32)])
    return Workload(f"p-16O + p-40Ca {energy:g} MeV", [O16, CA40], e, t, seed)


def mixed(n: int = 4_000_000, seed: int = 0, emin=20.0, emax=250.0) -> Workload:
    """Energies uniform in [emin, emax]; targets 60% ¹⁶O, 20% ¹²C, 10% ¹⁴N, 5% ⁴⁰Ca, 5% ³¹P."""
    g = _rng(seed, 1)
    e = g.uniform(emin, emax, n)
    t = g.choice(5, size=n, p=[0.6, 0.2, 0.1, 0.05, 0.05]).astype(np.int32)
    return Workload("mixed tissue targets 20-250 MeV", [O16, C12, N14, CA40, P31], e, t, seed)


def heavy(target, n: int = 1_000_000, seed: int = 0, emin=100.0, emax=250.0) -> Workload:
    """Energies uniform in [emin, emax] on one heavy target (⁴⁸Ti, ⁵⁶Fe, ²⁰⁸Pb)."""
    g = _rng(seed, 2 + int(target[1]))
    return Workload(f"p-{target} {emin:g}-{emax:g} MeV", [tuple(target)], g.uniform(emin, emax, n),
                    np.zeros(n, np.int32), seed)


SERVING_TARGETS = [C12, O16, CA40, TI48, FE56]


def serving_requests(n_requests: int, rate_hz: float, seed: int = 0, min_batch=1_000, max_batch=100_000):
    """Synthetic proton-transport driver: Poisson arrivals (rate_hz), batch sizes
    log-uniform in [min_batch, max_batch], energies uniform 20–250 MeV, targets uniform over
    ¹²C, ¹⁶O, ⁴⁰Ca, ⁴⁸Ti, ⁵⁶Fe. Returns a list of dicts (arrival time in s, energies, tidx,
    request id). Event ids of request r are (r << 32) | index."""
    g = _rng(seed, 3)
    t = np.cumsum(g.exponential(1.0 / rate_hz, n_requests))
    sizes = np.exp(g.uniform(np.log(min_batch), np.log(max_batch), n_requests)).astype(np.int64)
    out = []
    for r in range(n_requests):
        k = int(sizes[r])
        out.append(dict(request=r, arrival=float(t[r]), energies=g.uniform(20.0, 250.0, k),
                        tidx=g.integers(0, len(SERVING_TARGETS), k).astype(np.int32),
                        first_event_id=r << 32))
    return out
