"""Pins for the oracle's gridding, compression, normaliser, statistics, degridding,
correction and the end-to-end image (Sec. 4.3, 4.7, eq. "convgrid").

* worked counts printed in the thesis (tests/golden/worked_counts.txt);
* compression leaves the grid and N_p unchanged (Sec. 4.3.3), including a compressible
  record that follows a non-griddable one (reading O-2 of eq. "ci");
* the sequential compression (oracle.c) and the vectorised indicators agree;
* adjoint identity Re<G x, y> = Re<x, G^H y> in FP64;
* the centred inverse FFT equals a direct sum on a small grid;
* a unit point source at the phase centre gives a 1 Jy/beam peak (Sec. 4.3.2);
* a direct-Fourier dirty image with the w-term (measurement-equation sign) agrees with the
  w-projected, gridded and corrected image on the inner half of the field.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from oracle.table import Table

C0 = 299_792_458.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _records(rng, n, N, du, tab, w_choice=None):
    smax = int(tab.supports.max())
    lim = (N // 2 - smax // 2 - 2) * du
    u = rng.uniform(-lim, lim, n)
    v = rng.uniform(-lim, lim, n)
    if w_choice is None:
        w = np.zeros(n)
    else:
        w = w_choice
    return np.stack([u, v, w], 1)


def _rand_vis(rng, shape):
    return (rng.normal(size=shape) + 1j * rng.normal(size=shape)).astype(np.complex64)


def test_worked_counts_golden():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "worked_counts.txt")) if l.strip() and not l.startswith("#")]
    for S, P, upd, *_ in rows:
        S, P, upd = int(S), int(P), int(upd)
        N = S + 8
        tab = Table(1, np.array([S], np.int32), np.array([0], np.int64), np.ones(S * S, complex),
                    np.array([float(S * S)]), np.zeros(1), 0.0)
        uvw = np.zeros((1, 3))
        fl = np.zeros((1, 1, P), np.uint8)
        pl = oracle.place(uvw, np.array([C0]), 1.0, N, tab, flag=fl)
        g, c = oracle.classify(pl)
        st = oracle.stats(pl, g, c)
        assert st["updates"] * P == upd
        G = oracle.grid_plain(pl, tab, np.ones((1, 1, P), np.complex64), np.ones((1, 1, P), np.float32), fl, N)
        assert np.count_nonzero(G) == upd


def test_compression_invariance_on_tracks():
    wl = synth.make("w0_small", n_times=48, flag_frac=0.05)
    tab = oracle.build_table(wl.du, 1, 0.0, wl.oversample, 7, supports=wl.supports)
    vis, w, f = wl.vis.numpy(), wl.weight.numpy(), wl.flag.numpy()
    pl = oracle.place(wl.uvw, wl.freq, wl.du, wl.n_grid, tab, flag=f)
    G = oracle.grid_plain(pl, tab, vis, w, f, wl.n_grid)
    G2 = oracle.grid_compressed(pl, tab, vis, w, f, wl.n_grid)
    assert np.linalg.norm(G - G2) <= 1e-13 * np.linalg.norm(G)
    g, c = oracle.classify(pl)
    g2, c2, lrec, llast, gamma = oracle.compress(pl, vis, w, f)
    assert np.array_equal(g, g2) and np.array_equal(c, c2)
    st = oracle.stats(pl, g, c)
    assert st["gridded"] + st["compressed"] == int(pl.griddable.sum())
    assert st["compressed"] > 0.2 * st["gridded"]          # baseline tracks do compress
    assert st["updates"] == int((pl.S[g] ** 2).sum())


def test_compression_after_nongriddable_predecessor():
    # records 0,1,2 share footprint and kernel pointer; record 1 is fully flagged, so record
    # 2 must start a new gridded entry instead of joining a record that is not gridded.
    N, du = 64, 0.5
    tab = oracle.build_table(2.0, 1, 0.0, 4, 7, supports=[7], n_k=64)
    uvw = np.array([[1.0, 2.0, 0.0]] * 3 + [[1.0, 2.0, 0.0], [5.0, 2.0, 0.0]])
    fl = np.zeros((5, 1, 2), np.uint8)
    fl[1] = 1
    rng = np.random.default_rng(0)
    vis = _rand_vis(rng, (5, 1, 2))
    wt = rng.uniform(0.5, 2.0, (5, 1, 2)).astype(np.float32)
    pl = oracle.place(uvw, np.array([C0]), du, N, tab, flag=fl)
    g, c = oracle.classify(pl)
    assert list(g) == [True, False, True, False, True]
    assert list(c) == [False, False, False, True, False]
    G = oracle.grid_plain(pl, tab, vis, wt, fl, N)
    G2 = oracle.grid_compressed(pl, tab, vis, wt, fl, N)
    assert np.allclose(G, G2, rtol=0, atol=1e-13)
    gg, cc, lrec, llast, gamma = oracle.compress(pl, vis, wt, fl)
    assert list(lrec) == [0, 2, 4] and list(llast) == [0, 3, 4]
    assert np.allclose(gamma[1], wt[2, 0] * vis[2, 0] + wt[3, 0] * vis[3, 0], atol=1e-6)


def test_adjoint_identity_fp64():
    rng = np.random.default_rng(2)
    N, du = 48, 2.0
    tab = oracle.build_table(du, 5, 40.0, 8, 7, n_k=64)
    n, P = 300, 2
    uvw = _records(rng, n, N, du, tab, rng.uniform(-45.0, 45.0, 300))
    freq = np.array([C0, 1.1 * C0])
    fl = (rng.random((n, 2, P)) < 0.1).astype(np.uint8)
    wt = rng.uniform(0.1, 1.0, (n, 2, P)).astype(np.float32)
    x = _rand_vis(rng, (n, 2, P))
    pl = oracle.place(uvw, freq, du, N, tab, flag=fl)
    assert pl.griddable.sum() > 200 and (pl.psi < 0).sum() > 50
    Gx = oracle.grid_plain(pl, tab, x, wt, fl, N)
    y = rng.normal(size=Gx.shape) + 1j * rng.normal(size=Gx.shape)
    Ghy = oracle.degrid(pl, tab, y, wt, fl, adjoint=True)
    lhs = np.real(np.vdot(Gx, y))
    rhs = np.real(np.vdot(x.reshape(-1, P).astype(np.complex128), Ghy))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_inverse_fft_convention_direct_sum():
    rng = np.random.default_rng(4)
    N = 8
    G = rng.normal(size=(1, N, N, 1)) + 1j * rng.normal(size=(1, N, N, 1))
    img = oracle.correct.dirty_per_pol(G)[0, 0]
    ref = np.zeros((N, N))
    for my in range(N):
        for mx in range(N):
            s = 0j
            for y in range(N):
                for x in range(N):
                    s += G[0, y, x, 0] * np.exp(2j * np.pi * ((x - N // 2) * (mx - N // 2) + (y - N // 2) * (my - N // 2)) / N)
            ref[my, mx] = s.real
    assert np.max(np.abs(img - ref)) < 1e-12


def test_point_source_peak_is_one():
    wl = synth.make("w0_small", n_times=24)
    tab = oracle.build_table(wl.du, 1, 0.0, wl.oversample, 7, supports=wl.supports)
    f = wl.flag.numpy()
    pl = oracle.place(wl.uvw, wl.freq, wl.du, wl.n_grid, tab, flag=f)
    ones = np.ones(wl.vis.shape, np.complex64)
    G = oracle.grid_plain(pl, tab, ones, wl.weight.numpy(), f, wl.n_grid)
    Np = oracle.normaliser(pl, tab, wl.weight.numpy(), f)
    img = oracle.grid_correct(G, Np, tab.beta, 7)[0, 0]
    c = wl.n_grid // 2
    assert abs(img[c, c] - 1.0) < 1e-12 and img[c, c] >= img.max() - 1e-12


@pytest.mark.parametrize("K,w_max", [(1, 0.0), (17, 60.0)])
def test_end_to_end_against_direct_fourier(K, w_max):
    # records sit on the w-planes exactly (w sign random, exercising take-conjugate), so
    # the residual is the kernel's aliasing/truncation at beta = 64 (measured ~2e-3)
    rng = np.random.default_rng(7)
    N, du, beta, n = 64, 2.0, 64, 200
    tab = oracle.build_table(du, K, w_max, beta, 7, n_k=64)
    kk = rng.integers(0, K, n)
    w = rng.choice([-1.0, 1.0], n) * tab.w_planes[kk]
    uvw = _records(rng, n, N, du, tab, w)
    freq = np.array([C0])
    sky = synth.Sky(np.array([1.0, 0.6]), np.array([0.05, -0.08]), np.array([-0.07, 0.04]))
    vis = synth.visibilities(uvw, freq, sky, 1, 0.0, 1).numpy()
    wt = np.ones((n, 1, 1), np.float32)
    fl = np.zeros((n, 1, 1), np.uint8)
    pl = oracle.place(uvw, freq, du, N, tab, flag=fl)
    assert pl.griddable.all()
    G = oracle.grid_plain(pl, tab, vis, wt, fl, N)
    Np = oracle.normaliser(pl, tab, wt, fl)
    img = oracle.grid_correct(G, Np, beta, 7)[0, 0]
    ref = oracle.dirty_image(uvw, freq, vis, wt, fl, N, du)[0, 0]
    inner = slice(N // 4, 3 * N // 4)
    err = np.max(np.abs(img - ref)[inner, inner]) / np.max(np.abs(ref))
    assert err < 5e-3, err


@pytest.mark.parametrize("beta", [2, 8])
def test_sinc_is_transform_of_nearest_sample_rect(beta):
    # nearest-sample selection convolves the kernel with a rect of width du/beta
    # (eq. "coversampled"); its image-plane factor is the rect's normalised transform
    N, du = 32, 1.7
    t, wts = np.polynomial.legendre.leggauss(64)
    half = du / (2 * beta)
    d = half * t
    l = (np.arange(N) - N // 2) / (N * du)
    ft = (np.exp(2j * np.pi * d[None, :] * l[:, None]) * wts[None, :]).sum(1) * half / (2 * half)
    assert np.max(np.abs(oracle.correct.sinc_1d(N, beta) - ft.real)) < 1e-14
    assert np.max(np.abs(ft.imag)) < 1e-14
