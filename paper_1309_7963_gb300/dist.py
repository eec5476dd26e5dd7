"""Multi-process launch helpers (one process per GPU under torchrun).

Events are independent and every event depends only on (seed, event id), so the work shards
by event-id range with no collective on the data path: rank r of a world of N simulates ids
[first + r*n, first + (r+1)*n). torch.distributed is used only for a barrier around the
timed region and the maximum of the ranks' elapsed times.
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
