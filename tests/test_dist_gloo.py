"""The multi-rank path on CPU: two gloo ranks shard a workload by event-id range and
reproduce, event for event, the single-process result (computed here with the oracle, the
only CPU implementation); the final gather puts the whole batch's records on rank 0 with
event indices in the batch; the max-over-ranks timing helper takes the largest value."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1309_7963_gb300 import dist, inputs


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, n_per_rank, out_dir):
    import torch.distributed as td
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    td.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = dist.env()
    first = dist.shard_first_event_id(r, n_per_rank)
    full = inputs.mixed(w * n_per_rank, seed=17)
    part = full.slice(first, first + n_per_rank)
    out = oracle.simulate(part.targets, part.energies, part.tidx, seed=part.seed, first_event_id=part.first_event_id)
    res = out["residuals"]
    np.save(os.path.join(out_dir, f"rank{r}.npy"), res)
    got = dist.gather_results(out["secondaries"], res, n_per_rank)
    if r == 0:
        np.save(os.path.join(out_dir, "gathered_sec.npy"), got[0])
        np.save(os.path.join(out_dir, "gathered_res.npy"), got[1])
    else:
        assert got is None
    m = dist.max_over_ranks(10.0 + r)
    td.barrier()
    td.destroy_process_group()
    with open(os.path.join(out_dir, f"max{r}.txt"), "w") as f:
        f.write(repr(m))


def test_two_gloo_ranks_shard_by_event_id(tmp_path):
    world, n = 2, 300
    mp.spawn(worker, args=(world, free_port(), n, str(tmp_path)), nprocs=world, join=True)
    parts = [np.load(tmp_path / f"rank{r}.npy") for r in range(world)]
    full = inputs.mixed(world * n, seed=17)
    ref_out = oracle.simulate(full.targets, full.energies, full.tidx, seed=full.seed)
    ref = ref_out["residuals"]
    assert np.array_equal(np.concatenate(parts), ref)
    # the gather on rank 0: the whole batch's records, event indices in the batch
    order = lambda s: s[np.lexsort((s["index"], s["event"]))]
    assert np.array_equal(np.load(tmp_path / "gathered_res.npy"), ref)
    assert np.array_equal(order(np.load(tmp_path / "gathered_sec.npy")), order(ref_out["secondaries"]))
    for r in range(world):
        assert float((tmp_path / f"max{r}.txt").read_text()) == 10.0 + world - 1


def test_shard_ids_partition_the_range():
    ids = [range(dist.shard_first_event_id(r, 1000, 5), dist.shard_first_event_id(r, 1000, 5) + 1000)
           for r in range(4)]
    flat = [i for rng in ids for i in rng]
    assert flat == list(range(5, 5 + 4000))
    assert dist.max_over_ranks(3.5) == 3.5
