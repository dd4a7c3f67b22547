"""Full-Stokes gridding and finalising on the GPU against the FP64 oracle: cross-hand swapping
of take-conjugate records (WG_PREP_CROSS_SWAP: grid, N_p and degridding) and the Stokes modes
of grid_correct for linear and circular feeds.  A polarised point source at the phase centre
must come back as (I, Q, U, V) within 2e-3; the grids and images agree with the oracle within
the FP32 bars (1e-5 rel-L2 for the grid; images within 1e-5 of the peak after multiplying back
taper x sinc squared)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1403_4209_gb300 as wg
import synth
from oracle.grid import degrid, grid_plain, normaliser
from gpu_common import rel_l2

pytestmark = pytest.mark.gpu

STOKES = (1.0, 0.3, -0.2, 0.15)
N = 512


@pytest.fixture(scope="module")
def geom():
    wl = synth.make("wproj_2k", n_times=60, n_chan=2, n_baselines=200, flag_frac=0.02)
    from synth import cell_and_wmax
    wl.n_grid = N
    wl.du, wl.w_max = cell_and_wmax(wl.uvw, wl.freq, N, max(wl.supports))
    ot = oracle.build_table(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support, supports=wl.supports)
    t = wg.ConvTable.build(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support, supports=wl.supports)
    pl = oracle.place(wl.uvw, wl.freq, wl.du, N, ot, flag=wl.flag.numpy())
    return wl, ot, t, pl


def _vis(rows, C, feeds):
    I, Q, U, V = STOKES
    c = [I + Q, U + 1j * V, U - 1j * V, I - Q] if feeds == "linear" else [I + V, Q + 1j * U, Q - 1j * U, I - V]
    return np.tile(np.array(c, np.complex64), (rows, C, 1))


def _run(wl, t, vis, swap, mode):
    dev = "cuda"
    g = wg.Grid(N, wl.du, 4, wl.n_chan)
    b = wg.VisBatch(torch.as_tensor(wl.uvw, device=dev), torch.as_tensor(wl.freq, device=dev),
                    torch.as_tensor(vis, device=dev), wl.weight.to(dev), wl.flag.to(dev))
    w = wg.WorkList(wl.rows * wl.n_chan, wl.n_chan, 4)
    wg.vis_compress(g, t, b, w, cross_swap=swap)
    wg.grid_vis(g, t, w)
    img = wg.grid_correct(g, t, mode=mode)
    torch.cuda.synchronize()
    return g, b, w, img.cpu().numpy()


@pytest.mark.parametrize("feeds,mode", [("linear", wg.IMAGE_STOKES_LINEAR), ("circular", wg.IMAGE_STOKES_CIRCULAR)])
def test_stokes_point_source_and_oracle(geom, feeds, mode):
    wl, ot, t, pl = geom
    vis = _vis(wl.rows, wl.n_chan, feeds)
    g, b, w, img = _run(wl, t, vis, True, mode)
    assert np.allclose(img[:, :, N // 2, N // 2], np.tile(STOKES, (wl.n_chan, 1)), atol=2e-3)
    wt, f = wl.weight.numpy(), wl.flag.numpy()
    G = grid_plain(pl, ot, vis, wt, f, N, cross_swap=True)
    assert rel_l2(g.data.cpu().numpy(), G) < 1e-5
    Np = normaliser(pl, ot, wt, f, cross_swap=True)
    assert np.max(np.abs(g.normaliser().cpu().numpy() - Np)) <= 1e-5 * np.max(Np)
    ref = oracle.grid_correct_stokes(G, Np, ot.beta, wl.taper_support, feeds)
    tap = oracle.taper_1d(N, wl.taper_support) * oracle.correct.sinc_1d(N, wl.oversample)
    t2 = np.abs(tap[:, None] * tap[None, :])
    assert np.max(np.abs(img - ref) * t2) <= 1e-5 * np.max(np.abs(ref) * t2)


def test_swapped_degrid_matches_oracle(geom):
    wl, ot, t, pl = geom
    rng = np.random.default_rng(9)
    vis = (rng.normal(size=(wl.rows, wl.n_chan, 4)) + 1j * rng.normal(size=(wl.rows, wl.n_chan, 4))).astype(np.complex64)
    g, b, w, _ = _run(wl, t, vis, True, wg.IMAGE_PER_POL)
    out = wg.degrid_vis(g, t, b, w, mode=wg.DEGRID_ADJOINT).cpu().numpy().reshape(-1, 4)
    G = g.data.cpu().numpy().astype(np.complex128)
    exp = degrid(pl, ot, G, wl.weight.numpy(), wl.flag.numpy(), adjoint=True, cross_swap=True)
    assert np.max(np.abs(out - exp)) <= 1e-5 * np.max(np.abs(exp))


def test_cross_swap_needs_four_polarisations(geom):
    wl, ot, t, pl = geom
    dev = "cuda"
    g = wg.Grid(N, wl.du, 2, 1)
    v = torch.zeros((wl.rows, 1, 2), dtype=torch.complex64, device=dev)
    b = wg.VisBatch(torch.as_tensor(wl.uvw, device=dev), torch.as_tensor(wl.freq[:1], device=dev), v,
                    torch.ones((wl.rows, 1, 2), device=dev), torch.zeros((wl.rows, 1, 2), dtype=torch.uint8, device=dev))
    w = wg.WorkList(wl.rows, 1, 2)
    with pytest.raises(wg.WgError, match="INVALID_ARG"):
        wg.vis_compress(g, t, b, w, cross_swap=True)
