"""GPU parity of conv_table_build, degrid_vis and grid_correct against the FP64 oracle.

Bars: table samples within FP32 rounding of the FP64 oracle (|d| <= 2e-7 max|C|), zeta within
1e-10, supports exact; degridded visibilities within 1e-5 relative (FP32 gather of S^2 terms);
the GPU adjoint identity Re<Gx, y> = Re<x, G^H y> to 1e-5; corrected images within 1e-5 of
max|image| on the inner half (FP32 FFT; the taper correction amplifies the edges).
Inputs to both sides come from the seeded generators only.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1403_4209_gb300 as wg
import synth
from gpu_common import max_rel, run_gpu

pytestmark = pytest.mark.gpu


def _cmp_table(gt, ot):
    data, zeta, sup, off = gt.to_host()
    assert np.array_equal(sup, ot.supports)
    assert np.array_equal(off, ot.offsets)
    assert np.max(np.abs(data - ot.data)) <= 2e-7 * np.max(np.abs(ot.data))
    assert np.max(np.abs(zeta - ot.zeta)) <= 1e-10 * np.max(np.abs(ot.zeta))


@pytest.mark.parametrize("K,w_max,beta,supports,n_k", [
    (1, 0.0, 8, [7], 64),                       # w = 0 kernel, S = 7, beta = 8
    (5, 300.0, 4, [9, 11, 15, 21, 27], 128),    # w-projection, prescribed supports
    (3, 80.0, 8, [11, 13, 19], 64),
])
def test_table_prescribed(K, w_max, beta, supports, n_k):
    du = 1.7
    gt = wg.ConvTable.build(du, K, w_max, beta, 7, supports=supports, n_k=n_k)
    ot = oracle.build_table(du, K, w_max, beta, 7, supports=supports, n_k=n_k)
    _cmp_table(gt, ot)


def test_table_threshold_supports():
    du = 1.7
    gt = wg.ConvTable.build(du, 6, 400.0, 4, 7, supports=None, n_k=128, threshold=1e-3)
    ot = oracle.build_table(du, 6, 400.0, 4, 7, supports=None, n_k=128, threshold=1e-3)
    _cmp_table(gt, ot)
    assert gt.supports[-1] > gt.supports[0]


def _random_grid(shape, seed):
    rng = np.random.default_rng(seed)
    return (rng.normal(size=shape) + 1j * rng.normal(size=shape)).astype(np.complex64)


@pytest.mark.parametrize("name,kw", [("w0_small", dict(n_times=24, flag_frac=0.03)),
                                     ("degrid_1k", dict(n_times=20, n_baselines=150, flag_frac=0.03))])
@pytest.mark.parametrize("mode", [wg.DEGRID_PREDICT, wg.DEGRID_ADJOINT])
def test_degrid_parity(name, kw, mode):
    wl = synth.make(name, **kw)
    gp = run_gpu(wl)
    g, t, batch, wlst = gp["objects"]
    y = _random_grid(tuple(g.data.shape), 5)
    g.data.copy_(torch.as_tensor(y))
    out = wg.degrid_vis(g, t, batch, wlst, mode=mode)
    torch.cuda.synchronize()
    ot = oracle.build_table(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support, supports=wl.supports)
    f = wl.flag.numpy()
    pl = oracle.place(wl.uvw, wl.freq, wl.du, wl.n_grid, ot, flag=f)
    ref = oracle.degrid(pl, ot, y.astype(np.complex128), wl.weight.numpy(), f, adjoint=(mode == wg.DEGRID_ADJOINT))
    got = out.cpu().numpy().reshape(-1, wl.n_pol)
    assert np.array_equal(got[~pl.griddable], np.zeros_like(got[~pl.griddable]))
    assert max_rel(got, ref) < 1e-5


def test_gpu_adjoint_identity():
    wl = synth.make("degrid_1k", n_times=16, n_baselines=120, flag_frac=0.05)
    gp = run_gpu(wl)                      # grid(x) for x = the synthetic visibilities
    g, t, batch, wlst = gp["objects"]
    Gx = gp["grid"].astype(np.complex128)
    y = _random_grid(tuple(g.data.shape), 9)
    g.data.copy_(torch.as_tensor(y))
    Ghy = wg.degrid_vis(g, t, batch, wlst, mode=wg.DEGRID_ADJOINT).cpu().numpy().astype(np.complex128)
    x = wl.vis.numpy().astype(np.complex128)
    lhs = np.real(np.vdot(Gx, y.astype(np.complex128)))
    rhs = np.real(np.vdot(x, Ghy))
    assert abs(lhs - rhs) <= 1e-5 * np.sqrt(np.vdot(Gx, Gx).real * np.vdot(y, y).real)


@pytest.mark.parametrize("P,mode", [(1, wg.IMAGE_PER_POL), (4, wg.IMAGE_PER_POL), (4, wg.IMAGE_STOKES_I)])
def test_grid_correct_parity(P, mode):
    N, C, du, beta = 256, 2, 1.3, 8
    t = wg.ConvTable.build(du, 1, 0.0, beta, 7, supports=[7])
    g = wg.Grid(N, du, P, C)
    y = _random_grid((C, N, N, P), 3) * 1e-3
    # a smooth bright component so the image is not noise-dominated
    yy, xx = np.mgrid[0:N, 0:N]
    y += (np.exp(-((xx - N / 2) ** 2 + (yy - N / 2) ** 2) / 200.0)[None, :, :, None]).astype(np.complex64)
    g.data.copy_(torch.as_tensor(y))
    rng = np.random.default_rng(2)
    norm = rng.uniform(50, 150, (C, P))
    g.normaliser().copy_(torch.as_tensor(norm))
    img = wg.grid_correct(g, t, mode=mode)
    torch.cuda.synchronize()
    ref = oracle.grid_correct(y.astype(np.complex128), norm, beta, 7, stokes_i=(mode == wg.IMAGE_STOKES_I))
    got = img.cpu().numpy()
    inner = (Ellipsis, slice(N // 4, 3 * N // 4), slice(N // 4, 3 * N // 4))
    assert np.max(np.abs(got[inner] - ref[inner])) <= 1e-5 * np.max(np.abs(ref[inner]))
    # the edges are divided by a taper down to ~2e-4: compare against the FP32 error scaled by it
    tap = oracle.taper_1d(N, 7) * oracle.correct.sinc_1d(N, beta)
    scale = 1.0 / np.abs(tap[:, None] * tap[None, :])
    err = np.abs(got - ref) / scale
    assert np.max(err) <= 1e-5 * np.max(np.abs(ref[inner]))
