"""Multi-process launch helpers (one process per GPU under torchrun).

Events are independent and every event depends only on (seed, event id), so the work shards
by event-id range with no collective on the data path: rank r of a world of N simulates ids
[first + r*n, first + (r+1)*n). torch.distributed is used for a barrier around the timed
region, the maximum of the ranks' elapsed times, and (when a caller wants one result) a final
gather of the ranks' records on the host, after the simulation.
"""
from __future__ import annotations

import os


def env() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the torchrun environment (defaults: one process)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_first_event_id(rank: int, n_per_rank: int, first_event_id: int = 0) -> int:
    """First event id of a rank's shard (weak scaling: every rank simulates n_per_rank events)."""
    return first_event_id + rank * n_per_rank


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a float over all ranks (identity without an initialised process group)."""
    import torch
    import torch.distributed as td
    if not (td.is_available() and td.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def concat_shards(parts, n_per_rank: int):
    """One batch's records from its ranks' shards, in rank order: parts[r] = (secondaries,
    residuals) of rank r (numpy structured arrays with an "event" field counting from 0 in each
    shard); the secondaries' event indices are moved to their place in the whole batch."""
    import numpy as np
    secs, ress = [], []
    for r, (sec, res) in enumerate(parts):
        s = sec.copy()
        s["event"] = s["event"] + r * n_per_rank
        secs.append(s)
        ress.append(res)
    return np.concatenate(secs), np.concatenate(ress)


def gather_results(secondaries, residuals, n_per_rank: int, dst: int = 0):
    """Every rank's (secondaries, residuals) on rank dst as one batch (concat_shards); None on
    the other ranks and the inputs unchanged without a process group. Host arrays, after the
    simulation: the one collective of the multi-rank path."""
    import torch.distributed as td
    if not (td.is_available() and td.is_initialized()):
        return secondaries, residuals
    rank, world = td.get_rank(), td.get_world_size()
    parts = [None] * world if rank == dst else None
    td.gather_object((secondaries, residuals), parts, dst=dst)
    return concat_shards(parts, n_per_rank) if rank == dst else None
