"""pnuc_simulate_host with pageable host buffers (staged on the device, copied back) and
with pinned ones (secondaries written by the kernels in place): the results equal a device
launch of the same events; a reservation too small reports the full count."""
import numpy as np
import pytest

from paper_1309_7963_gb300 import inputs, pnuc

pytestmark = pytest.mark.gpu


def device_run(ctx, w, tids, precision="fp32"):
    import torch
    r = ctx.simulate(torch.tensor(w.energies, device="cuda"), torch.tensor(tids[w.tidx], device="cuda"),
                     seed=w.seed, first_event_id=w.first_event_id, precision=precision, capacity=8 * w.n)
    torch.cuda.synchronize()
    return pnuc.sort_secondaries(r.secondaries_np()), r.residuals_np()


def pinned(n_bytes, dtype):
    import torch
    return torch.empty(n_bytes, dtype=torch.uint8).pin_memory().numpy().view(dtype)


@pytest.mark.parametrize("where", ["pageable", "pinned"])
def test_host_entry_equals_a_device_launch(ctx, where):
    w = inputs.mixed(1_200_000, seed=6)
    n = w.n
    tids = np.array([ctx.create_target(*za) for za in w.targets], np.int32)
    ref_sec, ref_res = device_run(ctx, w, tids)
    kw = {}
    if where == "pinned":
        kw = dict(sec_out=pinned(8 * n * 32, pnuc.SECONDARY_DTYPE), res_out=pinned(n * 64, pnuc.RESIDUAL_DTYPE))
    sec, res = ctx.simulate_host(w.energies, tids[w.tidx], seed=w.seed, first_event_id=w.first_event_id,
                                 capacity=8 * n, **kw)
    assert np.array_equal(res, ref_res)
    assert np.array_equal(pnuc.sort_secondaries(sec), ref_sec)


@pytest.mark.parametrize("where", ["pageable", "pinned"])
def test_too_small_a_reservation_reports_the_count(ctx, where):
    w = inputs.oxygen_calcium(n_each=20_000)
    tids = np.array([ctx.create_target(*za) for za in w.targets], np.int32)
    ref_sec, ref_res = device_run(ctx, w, tids)
    total = len(ref_sec)
    kw = {}
    if where == "pinned":
        kw = dict(sec_out=pinned((total - 1) * 32, pnuc.SECONDARY_DTYPE), res_out=pinned(w.n * 64, pnuc.RESIDUAL_DTYPE))
    with pytest.raises(pnuc.PnucError) as e:
        ctx.simulate_host(w.energies, tids[w.tidx], seed=w.seed, first_event_id=w.first_event_id,
                          capacity=total - 1, **kw)
    assert e.value.status == 3
    sec, res = ctx.simulate_host(w.energies, tids[w.tidx], seed=w.seed, first_event_id=w.first_event_id,
                                 capacity=total)
    assert np.array_equal(res, ref_res) and np.array_equal(pnuc.sort_secondaries(sec), ref_sec)


def test_pinned_outputs_with_events_that_end_in_the_cascade(ctx):
    """Pinned host outputs with events that end in the cascade kernel (bad inputs: energies
    outside 20-250 MeV and target ids out of range) among events that evaporate: the records
    the kernels write in place equal a device launch of the same events."""
    w = inputs.mixed(50_000, seed=8)
    n = w.n
    tids = np.array([ctx.create_target(*za) for za in w.targets], np.int32)
    energies = np.array(w.energies, np.float64)
    targets = tids[w.tidx].astype(np.int32)
    energies[::97] = 10.0
    energies[1::101] = 300.0
    targets[2::89] = 99
    targets[3::113] = -1

    class W:
        pass
    ww = W()
    ww.energies, ww.seed, ww.first_event_id, ww.n = energies, w.seed, w.first_event_id, n
    ww.tidx = np.arange(n)
    ref_sec, ref_res = device_run(ctx, ww, targets)
    assert ((ref_res["flags"] & 1) != 0).sum() > 1000
    sec, res = ctx.simulate_host(energies, targets, seed=w.seed, first_event_id=w.first_event_id, capacity=8 * n,
                                 sec_out=pinned(8 * n * 32, pnuc.SECONDARY_DTYPE), res_out=pinned(n * 64, pnuc.RESIDUAL_DTYPE))
    assert np.array_equal(res, ref_res)
    assert np.array_equal(pnuc.sort_secondaries(sec), ref_sec)
