"""W-stacking on the GPU (WG_TABLE_WSTACK, WG_PREP_WSTACK, WG_IMAGE_WSTACK) against the FP64
oracle (oracle/wstack.py): the per-plane grids within the FP32 bar (1e-5 rel-L2), each channel's
N_p in its plane-0 grid channel, the stacked images within 1e-5 of their peak after multiplying
back taper x sinc squared, and degridding of the plane grids.  Workload: the w-projection
geometry sliced to 200 baselines x 30 steps x 2 channels, 4 pols, 2 % flags, on a 256² grid
with its own cell size, 8 planes holding the w = 0 kernel (support 9)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1403_4209_gb300 as wg
import synth
from gpu_common import rel_l2
from oracle.wstack import grid_stacked, image_stacked, stacking_table

pytestmark = pytest.mark.gpu

N, K = 256, 8


@pytest.fixture(scope="module")
def case():
    wl = synth.make("wproj_2k", n_times=30, n_chan=2, n_baselines=200, flag_frac=0.02)
    from synth import cell_and_wmax
    du, w_max = cell_and_wmax(wl.uvw, wl.freq, N, 9)
    sup = [9] * K
    t = wg.ConvTable.build(du, K, w_max, 8, 7, supports=sup, stacking=True)
    ot = stacking_table(du, K, w_max, 8, 7, supports=sup)
    dev = "cuda"
    g = wg.Grid(N, du, 4, wl.n_chan * K)
    b = wg.VisBatch(torch.as_tensor(wl.uvw, device=dev), torch.as_tensor(wl.freq, device=dev), wl.vis.to(dev),
                    wl.weight.to(dev), wl.flag.to(dev))
    w = wg.WorkList(wl.rows * wl.n_chan, wl.n_chan, 4)
    wg.vis_compress(g, t, b, w, wstack=True)
    wg.grid_vis(g, t, w)
    img = wg.grid_correct(g, t, mode=wg.IMAGE_WSTACK)
    torch.cuda.synchronize()
    pl = oracle.place(wl.uvw, wl.freq, du, N, ot, flag=wl.flag.numpy())
    return wl, du, t, ot, g, b, w, img.cpu().numpy(), pl


def test_table_planes_match_the_oracle(case):
    wl, du, t, ot, *_ = case
    data, zeta, sup, off = t.to_host()
    assert np.array_equal(sup, ot.supports)
    assert np.max(np.abs(data - ot.data)) <= 2e-7 * np.max(np.abs(ot.data))
    per = ot.data.size // K
    for k in range(1, K):
        assert np.array_equal(data[k * per:(k + 1) * per], data[:per])


def test_plane_grids_normaliser_and_image(case):
    wl, du, t, ot, g, b, w, img, pl = case
    vis, wt, f = wl.vis.numpy(), wl.weight.numpy(), wl.flag.numpy()
    G = grid_stacked(pl, ot, vis, wt, f, N)
    got = g.data.cpu().numpy()
    assert got.shape == G.shape and rel_l2(got, G) < 1e-5
    Np = oracle.normaliser(pl, ot, wt, f)
    gn = g.normaliser().cpu().numpy().reshape(wl.n_chan, K, 4)
    assert np.max(np.abs(gn[:, 0] - Np)) <= 1e-5 * np.max(Np) and np.all(gn[:, 1:] == 0)
    ref = image_stacked(G, Np, ot, 7, du)
    assert img.shape == ref.shape
    tap = oracle.taper_1d(N, 7) * oracle.correct.sinc_1d(N, 8)
    t2 = np.abs(tap[:, None] * tap[None, :])
    assert np.max(np.abs(img - ref) * t2) <= 1e-5 * np.max(np.abs(ref) * t2)


def test_degrid_reads_each_records_plane(case):
    wl, du, t, ot, g, b, w, img, pl = case
    out = wg.degrid_vis(g, t, b, w, mode=wg.DEGRID_ADJOINT).cpu().numpy().reshape(-1, 4)
    G = g.data.cpu().numpy().astype(np.complex128)
    import dataclasses
    pls = dataclasses.replace(pl, chan=(pl.chan.astype(np.int64) * K + np.where(pl.griddable, pl.k, 0)).astype(np.int32))
    exp = oracle.degrid(pls, ot, G, wl.weight.numpy(), wl.flag.numpy(), adjoint=True)
    assert np.max(np.abs(out - exp)) <= 1e-5 * np.max(np.abs(exp))


def test_stacking_needs_its_table(case):
    wl, du, t, ot, g, b, w, img, pl = case
    t2 = wg.ConvTable.build(du, K, t.w_max, 8, 7, supports=[9] * K)
    with pytest.raises(wg.WgError, match="INVALID_ARG"):
        wg.vis_compress(g, t2, b, w, wstack=True)
