"""pnuc_simulate_host_noalloc: the host-buffer entry point for callers that cannot allocate
device memory while they run (their device memory belongs to another allocator, or their
footprint must not grow). It must give exactly what pnuc_simulate_host gives, call after
call on its shared static scratch, and refuse a batch that does not fit that scratch; outputs
in pinned host memory take no scratch, so larger batches fit."""
import ctypes as C

import numpy as np
import pytest

from paper_1309_7963_gb300 import inputs, pnuc

pytestmark = pytest.mark.gpu

PNUC_ERR_CAPACITY = 3


def pinned(n_bytes, dtype):
    import torch
    return torch.zeros(n_bytes, dtype=torch.uint8).pin_memory().numpy().view(dtype)


def noalloc(ctx, energies, tids, seed, first, cap, precision, method, pinned_out=False):
    """One call of the no-allocation entry point through the C ABI (outputs in pageable
    numpy arrays, or in pinned host memory, which the kernels write in place)."""
    e = np.ascontiguousarray(energies, np.float64)
    t = np.ascontiguousarray(tids, np.int32)
    if pinned_out:
        sec = pinned(32 * cap, pnuc.SECONDARY_DTYPE)
        res = pinned(64 * len(e), pnuc.RESIDUAL_DTYPE)
    else:
        sec = np.zeros(cap, pnuc.SECONDARY_DTYPE)
        res = np.zeros(len(e), pnuc.RESIDUAL_DTYPE)
    cnt = C.c_uint64()
    st = ctx.lib.pnuc_simulate_host_noalloc(ctx.handle, pnuc.PRECISION[precision], pnuc.METHOD[method], e.ctypes.data,
                                            t.ctypes.data, len(e), seed, first, sec.ctypes.data, cap, C.byref(cnt),
                                            res.ctypes.data, None)
    return st, sec[: min(cnt.value, cap)], res


def target_ids(ctx, w):
    ids = np.array([ctx.create_target(*za) for za in w.targets], np.int32)
    return ids[w.tidx]


def test_noalloc_equals_host_entry_point_on_consecutive_calls(ctx):
    cases = [(inputs.mixed(5000, seed=31), 31, 0, "fp32", "persistent"),
             (inputs.oxygen_calcium(n_each=3000, seed=32), 32, 777, "fp64", "plain")]
    for w, seed, first, precision, method in cases:
        tids = target_ids(ctx, w)
        cap = 8 * w.n
        st, sec, res = noalloc(ctx, w.energies, tids, seed, first, cap, precision, method)
        assert st == 0, ctx._check(st)
        ref_sec, ref_res = ctx.simulate_host(w.energies, tids, seed=seed, first_event_id=first, precision=precision,
                                             method=method, capacity=cap)
        assert len(sec) == len(ref_sec) > w.n
        assert np.array_equal(res, ref_res)
        assert np.array_equal(pnuc.sort_secondaries(sec), pnuc.sort_secondaries(ref_sec))


def test_noalloc_refuses_batches_beyond_its_scratch(ctx):
    w = inputs.mixed(30_000, seed=33)
    st, sec, res = noalloc(ctx, w.energies, target_ids(ctx, w), 33, 0, 8 * w.n, "fp32", "persistent")
    assert st == PNUC_ERR_CAPACITY and len(sec) == 0
    with pytest.raises(pnuc.PnucError, match="static scratch"):
        ctx._check(st)


def test_noalloc_with_pinned_outputs_takes_larger_batches(ctx):
    w = inputs.mixed(300_000, seed=34)
    tids = target_ids(ctx, w)
    st, sec, res = noalloc(ctx, w.energies, tids, 34, 5, 8 * w.n, "fp32", "persistent", pinned_out=True)
    assert st == 0, ctx._check(st)
    ref_sec, ref_res = ctx.simulate_host(w.energies, tids, seed=34, first_event_id=5, capacity=8 * w.n)
    assert np.array_equal(res, ref_res)
    assert np.array_equal(pnuc.sort_secondaries(sec), pnuc.sort_secondaries(ref_sec))
