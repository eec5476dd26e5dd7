"""pnuc_tally against the reference tallies of oracle/tally.py: on the library's own records
the histograms are identical count for count (both the shared-memory and the global-atomic
path); in FP64 mode the library's tallies equal those of the oracle's events."""
import numpy as np
import pytest

import oracle
from oracle import tally as ref
from paper_1309_7963_gb300 import inputs, pnuc, yields

pytestmark = pytest.mark.gpu


def run(ctx, w, precision):
    import torch
    tids = np.array([ctx.create_target(*za) for za in w.targets], np.int32)
    e = torch.tensor(w.energies, device="cuda")
    t = torch.tensor(tids[w.tidx], device="cuda")
    r = ctx.simulate(e, t, seed=w.seed, precision=precision, method="persistent")
    torch.cuda.synchronize()
    return e, r


# counter paths: secondaries 1500 cells (two shared copies per 256-thread block), 12000 (one
# copy), 30000 (one 1024-thread block per SM), 60000 (global atomics); residuals 4030 cells
# (256-thread blocks), 46345 (1024-thread blocks), 583,073 (global atomics)
@pytest.mark.parametrize("n_cos,n_T,n_E,Z_max,A_max", [(1, 125, 2, 30, 64), (8, 125, 23, 30, 64),
                                                       (20, 125, 1, 30, 64), (40, 125, 23, 100, 250)])
def test_tally_equals_reference_on_the_same_records(ctx, n_cos, n_T, n_E, Z_max, A_max):
    import torch
    w = inputs.mixed(60_000, seed=8)
    e, r = run(ctx, w, "fp32")
    sh, rh = ctx.tally(r, e, n_T=n_T, n_cos=n_cos, n_E=n_E, Z_max=Z_max, A_max=A_max)
    torch.cuda.synchronize()
    sec, res = r.secondaries_np(), r.residuals_np()
    assert np.array_equal(sh.cpu().numpy(), ref.secondary_hist(sec["T"], sec["uz"], sec["species"], sec["origin"],
                                                                (0.0, 250.0), n_T, n_cos))
    assert np.array_equal(rh.cpu().numpy(), ref.residual_hist(res["Z_final"], res["A_final"], res["flags"], w.energies,
                                                               (20.0, 250.0), n_E, Z_max, A_max))
    # accumulation: a second call adds the same counts
    ctx.tally(r, e, n_T=n_T, n_cos=n_cos, n_E=n_E, Z_max=Z_max, A_max=A_max, hists=(sh, rh))
    assert np.array_equal(sh.cpu().numpy(), 2 * ref.secondary_hist(sec["T"], sec["uz"], sec["species"], sec["origin"],
                                                                    (0.0, 250.0), n_T, n_cos))


def test_fp64_tallies_equal_the_oracle_events(ctx):
    w = inputs.oxygen_calcium(n_each=5000)
    e, r = run(ctx, w, "fp64")
    sh, rh = ctx.tally(r, e, n_T=125, n_cos=20, n_E=1, E_range=(199.0, 201.0))
    orc = oracle.simulate_parallel(w.targets, w.energies, w.tidx, seed=w.seed)
    os_, ores = orc["secondaries"], orc["residuals"]
    want_s = ref.secondary_hist(os_["T"], os_["uz"].astype(np.float32), os_["species"], os_["origin"], (0.0, 250.0),
                                125, 20)
    want_r = ref.residual_hist(ores["Zf"], ores["Af"], ores["flags"], w.energies, (199.0, 201.0), 1, 100, 250)
    assert np.abs(sh.cpu().numpy() - want_s).sum() <= 2  # energies agree to 1e-9: a bin-edge flip is possible
    assert np.array_equal(rh.cpu().numpy(), want_r)


class Records:
    """records placed by the test (the layout of the library's output)"""

    def __init__(self, sec, res):
        import torch
        self.secondaries = torch.from_numpy(sec.view(np.uint8).reshape(len(sec), 32).copy()).cuda()
        self.residuals = torch.from_numpy(res.view(np.uint8).reshape(len(res), 64).copy()).cuda()

    def n_secondaries(self):
        return int(self.secondaries.shape[0])


def near_edges(rng, lo, hi, n, f32=False):
    """values on every bin edge of [lo, hi) in n bins and 1-3 ulps either side, plus random ones"""
    dt = np.float32 if f32 else np.float64
    e = np.repeat((lo + np.arange(-1, n + 2) * ((hi - lo) / n)).astype(dt), 13)
    k = np.tile(np.arange(-6, 7), len(e) // 13)
    x = e.copy()
    for i in range(len(x)):
        for _ in range(abs(int(k[i]))):
            x[i] = np.nextafter(x[i], dt(np.inf) if k[i] > 0 else dt(-np.inf))
    return np.concatenate([x, rng.uniform(lo - 1, hi + 1, 4000).astype(dt)])


@pytest.mark.parametrize("T_range,n_T,n_cos,E_range,n_E", [((0.0, 250.0), 125, 1, (199.0, 201.0), 1),
                                                           ((0.3, 217.7), 113, 7, (20.0, 250.0), 23),
                                                           ((-3.0, 41.0), 11, 40, (0.1, 0.7), 3)])
def test_bins_at_the_edges_equal_the_reference(ctx, T_range, n_T, n_cos, E_range, n_E):
    import torch
    rng = np.random.default_rng(n_T)
    T = near_edges(rng, *T_range, n_T)
    uz = rng.choice(near_edges(rng, -1.0, 1.0, n_cos, f32=True), len(T)).astype(np.float32)
    sec = np.zeros(len(T), pnuc.SECONDARY_DTYPE)
    sec["T"], sec["uz"] = T, uz
    sec["species"], sec["origin"] = rng.integers(0, 6, len(T)), rng.integers(0, 2, len(T))
    E = near_edges(rng, *E_range, n_E)
    res = np.zeros(len(E), pnuc.RESIDUAL_DTYPE)
    res["Z_final"], res["A_final"] = rng.integers(0, 9, len(E)), rng.integers(0, 17, len(E))
    res["flags"] = np.where(rng.random(len(E)) < 0.1, 1, 0)
    r = Records(sec, res)
    sh, rh = ctx.tally(r, torch.tensor(E, device="cuda"), T_range=T_range, n_T=n_T, n_cos=n_cos, E_range=E_range,
                       n_E=n_E, Z_max=8, A_max=16)
    assert np.array_equal(sh.cpu().numpy(), ref.secondary_hist(T, uz, sec["species"], sec["origin"], T_range, n_T,
                                                               n_cos))
    assert np.array_equal(rh.cpu().numpy(), ref.residual_hist(res["Z_final"], res["A_final"], res["flags"], E,
                                                               E_range, n_E, 8, 16))


def test_angle_windows_equal_the_reference(ctx):
    """the Fig. 2 windows (1 degree at 7.5, 30, 60 and 150 degrees) on the library's records,
    and 40 adjacent windows on records placed at and next to every edge"""
    import torch
    w = inputs.mixed(60_000, seed=9)
    e, r = run(ctx, w, "fp32")
    h = ctx.tally_windows(r, T_range=(0.0, 250.0), n_T=125)
    sec = r.secondaries_np()
    lo, hi = ctx.angle_windows()
    want = ref.secondary_window_hist(sec["T"], sec["uz"], sec["species"], sec["origin"], (0.0, 250.0), 125, lo, hi)
    assert want.sum() > 1000
    assert np.array_equal(h.cpu().numpy(), want)
    # adjacent windows of 0.05 in cos theta; uz on each edge's float and 1-3 floats either side
    lo2 = list(np.linspace(-1.0, 0.95, 40))
    hi2 = lo2[1:] + [1.0]
    rng = np.random.default_rng(2)
    uz = near_edges(rng, -1.0, 1.0, 40, f32=True)
    T = rng.uniform(0.0, 250.0, len(uz))
    rec = np.zeros(len(uz), pnuc.SECONDARY_DTYPE)
    rec["T"], rec["uz"] = T, uz
    rec["species"], rec["origin"] = rng.integers(0, 6, len(uz)), rng.integers(0, 2, len(uz))
    rr = Records(rec, np.zeros(1, pnuc.RESIDUAL_DTYPE))
    h2 = ctx.tally_windows(rr, n_T=50, cos_edges=(lo2, hi2))
    assert np.array_equal(h2.cpu().numpy(), ref.secondary_window_hist(T, uz, rec["species"], rec["origin"],
                                                                      (0.0, 250.0), 50, lo2, hi2))
    # accumulation, and bad window lists
    ctx.tally_windows(rr, n_T=50, cos_edges=(lo2, hi2), hist=h2)
    assert int(h2.sum()) == 2 * int(ref.secondary_window_hist(T, uz, rec["species"], rec["origin"], (0.0, 250.0), 50,
                                                               lo2, hi2).sum())
    for bad in (([0.1, 0.15], [0.2, 0.3]), ([0.3], [0.2]), ([0.0] * 65, [0.1] * 65), ([float("nan")], [0.5])):
        with pytest.raises(pnuc.PnucError):
            ctx.tally_windows(rr, cos_edges=bad)
    assert int(ctx.tally_windows(ctx.alloc(0)).sum()) == 0  # an empty batch
    torch.cuda.synchronize()


def test_positron_emitter_yields_and_edge_cases(ctx):
    import torch
    w = inputs.fixed(inputs.O16, 200.0, 50_000)
    e, r = run(ctx, w, "fp32")
    _, rh = ctx.tally(r, e, n_E=1, E_range=(150.0, 250.0))
    y = yields.emitter_yields(rh, (150.0, 250.0))
    assert y["events"][0] == (r.residuals_np()["flags"] & 3 == 0).sum()
    for name in ("15O", "11C", "13N"):
        assert 0.0 < y["yields"][name][0] < 1.0, name
    # empty batch and a bad spec
    empty = ctx.alloc(0)
    sh, rh = ctx.tally(empty, torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert int(sh.sum()) == 0 and int(rh.sum()) == 0
    with pytest.raises(pnuc.PnucError):
        ctx.tally(r, e, T_range=(10.0, 10.0))


def test_full_size_bench_batch_tallies_equal_the_reference(ctx):
    """the bench's workload (1e6 p-16O + 1e6 p-40Ca at 200 MeV, FP32 persistent, its tuning and
    output capacity) and the bench's tally specs: every count equal to the reference's"""
    import torch
    w = inputs.oxygen_calcium(n_each=1_000_000, energy=200.0)
    tids = np.array([ctx.create_target(*za) for za in w.targets], np.int32)
    e = torch.tensor(w.energies, device="cuda")
    t = torch.tensor(tids[w.tidx], device="cuda")
    r = ctx.simulate(e, t, seed=w.seed, precision="fp32", method="persistent", capacity=8 * w.n)
    sh, rh = ctx.tally(r, e, n_T=125, n_cos=1, n_E=1, E_range=(199.0, 201.0), Z_max=30, A_max=64)
    hw = ctx.tally_windows(r)
    torch.cuda.synchronize()
    sec, res = r.secondaries_np(), r.residuals_np()
    assert len(sec) > 9_000_000
    assert np.array_equal(sh.cpu().numpy(), ref.secondary_hist(sec["T"], sec["uz"], sec["species"], sec["origin"],
                                                                (0.0, 250.0), 125, 1))
    assert np.array_equal(rh.cpu().numpy(), ref.residual_hist(res["Z_final"], res["A_final"], res["flags"], w.energies,
                                                               (199.0, 201.0), 1, 30, 64))
    lo, hi = ctx.angle_windows()
    assert np.array_equal(hw.cpu().numpy(), ref.secondary_window_hist(sec["T"], sec["uz"], sec["species"],
                                                                       sec["origin"], (0.0, 250.0), 125, lo, hi))
