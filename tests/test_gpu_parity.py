"""GPU parity of the whole preparation + gridding path against the FP64 oracle, through the C ABI.

Bars (written here; FP32 accumulation against FP64 rounds each add to 2^-24 relative):
  * integer/index work bit-exact: per-record class bits (g, c, griddable), gridded entries
    (footprint origin, kernel pointer, plane, channel), run bounds, statistics;
  * FP32 accumulation vs FP64: grid rel-L2 <= 1e-5 and max-abs <= 1e-5 max|grid|; gamma and
    N_p within 1e-5 relative.
Sizes span several prep tiles, gridder segments and warps, with ragged tails.
"""
import dataclasses

import numpy as np
import pytest
import torch

import synth
from gpu_common import max_rel, rel_l2, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _entries_expected(o, wl):
    pl = o["pl"]
    rec = o["lrec"]
    k = pl.k[rec]
    return np.stack([pl.x0[rec], pl.y0[rec], pl.z[rec], k, pl.chan[rec]], 1), np.stack(
        [rec // wl.n_chan, o["llast"] // wl.n_chan], 1)


def _check(wl, compress, n_k=0, n_k_oracle=None):
    gp = run_gpu(wl, compress=compress, n_k=n_k)
    o = run_oracle(wl, compress=compress, n_k=n_k_oracle)
    pl = o["pl"]
    # per-record classification: bit0 g, bit1 c, bit2 griddable, bit3 take-conjugate
    cls = gp["rec_class"]
    assert np.array_equal((cls >> 3) & 1, (pl.psi < 0).astype(np.uint8))
    assert np.array_equal(cls & 1, o["g"].astype(np.uint8))
    assert np.array_equal((cls >> 1) & 1, o["c"].astype(np.uint8))
    assert np.array_equal((cls >> 2) & 1, pl.griddable.astype(np.uint8))
    # statistics (Sec. 4.3.4), exact
    st = gp["stats"]
    assert st["dropped"] == 0
    assert st["records"] == wl.rows * wl.n_chan
    assert st["griddable"] == int(pl.griddable.sum())
    assert st["gridded"] == o["stats"]["gridded"] and st["compressed"] == o["stats"]["compressed"]
    assert st["updates"] == o["stats"]["updates"] * wl.n_pol
    assert st["updates_saved"] == o["stats"]["updates_saved"] * wl.n_pol
    # gridded entries, channel-major
    e = gp["entries"]
    exp_e, exp_runs = _entries_expected(o, wl)
    got = np.stack([e[:, 0] & 0xFFFF, (e[:, 0] >> 16) & 0xFFFF, e[:, 2], e[:, 3] & 0xFFF, (e[:, 3] >> 16) & 0xFFFF], 1)
    assert got.shape == exp_e.shape
    assert np.array_equal(got, exp_e)
    assert np.array_equal(gp["runs"], exp_runs)
    S = pl.S[o["lrec"]]
    assert np.array_equal(e[:, 1] & 0xFFFF, (-pl.x0[o["lrec"]]) % S)
    assert np.array_equal((e[:, 1] >> 16) & 0xFFFF, (-pl.y0[o["lrec"]]) % S)
    # gamma, normaliser, grid
    assert max_rel(gp["gamma"], o["gamma"]) < TOL
    assert max_rel(gp["norm"], o["norm"]) < TOL
    assert rel_l2(gp["grid"], o["grid"]) < TOL
    assert max_rel(gp["grid"], o["grid"]) < TOL
    return gp, o


@pytest.mark.parametrize("compress", [False, True])
def test_w0_single_pol(compress):
    # w = 0, S = 7, beta = 8, N = 512, one channel: 496 baselines x 40 steps, 2% flags
    wl = synth.make("w0_small", n_times=40, flag_frac=0.02)
    gp, o = _check(wl, compress)
    if compress:
        assert gp["stats"]["compressed"] > 0


def test_wproj_quad_pol_two_channels():
    # w-projection slice: 300 baselines x 24 steps x 2 channels x 4 pols, 32 planes, S 9..65
    wl = synth.make("wproj_2k", n_times=24, n_chan=2, n_baselines=300, flag_frac=0.01)
    gp, o = _check(wl, True, n_k=256, n_k_oracle=256)
    assert len(set(o["pl"].k[o["pl"].griddable].tolist())) > 3


def test_degrid_geometry_dual_pol_like():
    # 4 channels, 16 planes; checks several channels with uneven coverage
    wl = synth.make("degrid_1k", n_times=30, n_baselines=200, flag_frac=0.05)
    _check(wl, True, n_k=128, n_k_oracle=128)


def test_empty_and_all_flagged():
    wl = synth.make("w0_small", n_times=3)
    wl.flag[:] = 1
    gp, o = _check(wl, True)
    assert gp["stats"]["griddable"] == 0 and np.all(gp["grid"] == 0)
    wl0 = synth.make("w0_small", n_times=1, n_baselines=0)
    assert wl0.rows == 0
    gp = run_gpu(wl0)
    assert gp["stats"]["records"] == 0 and np.all(gp["grid"] == 0)


def test_records_off_grid_are_dropped():
    wl = synth.make("w0_small", n_times=20)
    wl.uvw[::7, 0] *= 3.0      # push a seventh of the rows beyond the grid edge
    gp, o = _check(wl, True)
    assert gp["stats"]["griddable"] < wl.rows * wl.n_chan


def test_accumulates_over_batches():
    import paper_1403_4209_gb300 as wg
    wl = synth.make("w0_small", n_times=30)
    gp = run_gpu(wl)
    g, t, batch, wlst = gp["objects"]
    wg.vis_compress(g, t, batch, wlst)
    wg.grid_vis(g, t, wlst)
    torch.cuda.synchronize()
    assert rel_l2(g.data.cpu().numpy(), 2 * gp["grid"]) < 1e-6
    # per-tile partial sums of N_p are FP32 atomics: order-dependent at ~1e-7
    assert max_rel(g.normaliser().cpu().numpy(), 2 * gp["norm"]) < 1e-6


def test_plane_boundaries_bit_exact():
    # w exactly on each squared sqrt(w) midpoint b_m and one ulp either side (f = c0, so w' is w
    # in wavelengths): the plane index and griddability must match the oracle bit for bit
    from oracle.place import plane_bounds
    K, w_max = 7, 500.0
    b = plane_bounds(K, w_max)
    ws = np.concatenate([[0.0], b, np.nextafter(b, np.inf), np.nextafter(b, -np.inf), -b])
    rows = ws.size
    rng = np.random.default_rng(3)
    uvw = np.stack([rng.uniform(-20, 20, rows), rng.uniform(-20, 20, rows), ws], 1)
    wl = synth.Workload("plane_edges", uvw, np.array([synth.C0]), torch.ones((rows, 1, 1), dtype=torch.complex64),
                        torch.ones((rows, 1, 1)), torch.zeros((rows, 1, 1), dtype=torch.uint8), 256, 1.0, K,
                        w_max, 4, [9, 9, 11, 11, 13, 13, 15], 7, rows, 1)
    gp, o = _check(wl, False)
    pl = o["pl"]
    assert not pl.griddable[1 + K - 1] and pl.griddable[1 + 3 * K - 1]   # b_K excluded, just below it included


@pytest.mark.parametrize("K", [1, 7])
def test_nonfinite_and_signed_zero_coordinates_bit_exact(K):
    # NaN, +-inf, huge finite and signed-zero u, v, w: classification, take-conjugate bit,
    # statistics and grid must match the oracle (placement decisions are exact on both sides)
    import itertools
    from oracle.place import plane_bounds
    special = [np.nan, np.inf, -np.inf, 1e300, -1e300, 0.0, -0.0, 5.3, -7.9]
    wvals = [np.nan, np.inf, -np.inf, -0.0, 0.0, 120.0, -120.0, 1e300]
    uvw = np.array([(u, v, w) for u, v, w in itertools.product(special, special, wvals)], dtype=np.float64)
    rows = uvw.shape[0]
    w_max = 500.0
    sup = [9, 9, 11, 11, 13, 13, 15][:K]
    wl = synth.Workload("nonfinite", uvw, np.array([synth.C0]), torch.ones((rows, 1, 1), dtype=torch.complex64),
                        torch.ones((rows, 1, 1)), torch.zeros((rows, 1, 1), dtype=torch.uint8), 256, 1.0, K,
                        w_max if K > 1 else 0.0, 4, sup, 7, rows, 1)
    with np.errstate(invalid="ignore", over="ignore"):
        gp, o = _check(wl, False)
    assert o["pl"].griddable.any() and not o["pl"].griddable.all()


@pytest.mark.parametrize("du", [1.0, 0.7])
def test_cell_boundaries_bit_exact(du):
    # u', v' on the rounding boundaries of the oversampled lattice (t - 1/2 an integer, t = u' sc,
    # sc = beta / du with f = c0) and up to 3 ulps either side: the cell and sub-cell must match
    # the oracle bit for bit (the float estimate cannot decide these; the FP64 steps must)
    beta = 8
    sc = float(beta) / du
    base = (np.arange(-60, 60) + 0.5) / sc
    vals = [base]
    x = base.copy()
    y = base.copy()
    for _ in range(3):
        x = np.nextafter(x, np.inf)
        y = np.nextafter(y, -np.inf)
        vals += [x.copy(), y.copy()]
    u = np.concatenate(vals)
    rng = np.random.default_rng(11)
    v = rng.permutation(u)
    rows = u.size
    uvw = np.stack([u, v, rng.uniform(-5, 5, rows)], 1)
    wl = synth.Workload("cell_edges", uvw, np.array([synth.C0]), torch.ones((rows, 1, 1), dtype=torch.complex64),
                        torch.ones((rows, 1, 1)), torch.zeros((rows, 1, 1), dtype=torch.uint8), 64, du, 1, 0.0,
                        beta, [7], 7, rows, 1)
    gp, o = _check(wl, False)
    pl = o["pl"]
    assert pl.griddable.sum() > rows // 2
    # the entries carry the sub-cell through z: compare it with the oracle's directly
    g = np.nonzero(pl.griddable)[0]
    assert np.array_equal(np.sort(gp["entries"][:, 2]), np.sort(pl.z[g]))


@pytest.mark.parametrize("N,beta,pols,S", [(2048, 2, 4, 15), (2048, 4, 4, 63), (1024, 8, 2, 31), (4096, 8, 1, 127),
                                           (1024, 2, 1, 7)])
def test_sweep_configurations(N, beta, pols, S):
    # the configurations of bench.py's rate sweeps (the thesis's experiment batches 2-4): one
    # plane with a prescribed support, oversampling 2-8, 1-4 polarisations, grid side 1024-4096
    # at the uv extent of the 2048 grid (at 1024 the outer tracks leave the grid)
    base = synth.make("wproj_2k", n_times=40, n_chan=2, n_baselines=300, flag_frac=0.01)
    sel = {1: [0], 2: [0, 3], 4: [0, 1, 2, 3]}[pols]
    wl = dataclasses.replace(base, vis=base.vis[..., sel].contiguous(), weight=base.weight[..., sel].contiguous(),
                             flag=base.flag[..., sel].contiguous(), n_grid=N, du=base.du * 2048 / N,
                             oversample=beta, n_wplanes=1, supports=[S])
    gp, o = _check(wl, True)
    assert gp["stats"]["compressed"] > 0
