"""Pins of the oracle's full-Stokes path: the cross-hand swap for take-conjugate records and the
Stokes conversion of the image finaliser (Algorithm "finalizer" step 2).

A polarised point source at the phase centre has constant visibilities given by the feed
relations (linear: XX = I+Q, YY = I-Q, XY = U+jV, YX = U-jV; circular: RR = I+V, LL = I-V,
RL = Q+jU, LR = Q-jU), so the normalised Stokes images at the centre must return (I, Q, U, V).
The geometry has records with w' < 0 (take-conjugate), which is where V needs the swap."""
import numpy as np
import pytest

import oracle
import synth
from oracle.grid import compress, degrid, grid_compressed, grid_plain, normaliser

STOKES = (1.0, 0.3, -0.2, 0.15)


@pytest.fixture(scope="module")
def geom():
    wl = synth.make("wproj_2k", n_times=60, n_chan=1, n_baselines=200)
    wl.n_grid = 512
    from synth import cell_and_wmax
    wl.du, wl.w_max = cell_and_wmax(wl.uvw, wl.freq, 512, max(wl.supports))
    ot = oracle.build_table(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support, supports=wl.supports)
    pl = oracle.place(wl.uvw, wl.freq, wl.du, 512, ot)
    assert (pl.psi < 0).any() and (pl.psi > 0).any() and pl.griddable.mean() > 0.9
    return wl, ot, pl


def _vis(rows, feeds, P=4):
    I, Q, U, V = STOKES
    if feeds == "linear":
        c = [I + Q, U + 1j * V, U - 1j * V, I - Q]
    else:
        c = [I + V, Q + 1j * U, Q - 1j * U, I - V]
    if P == 2:
        c = [c[0], c[3]]
    return np.tile(np.array(c, np.complex64), (rows, 1, 1)).reshape(rows, 1, P)


def _centre(wl, ot, pl, feeds, swap, P=4):
    rows = wl.uvw.shape[0]
    vis = _vis(rows, feeds, P)
    w = np.ones((rows, 1, P), np.float32)
    f = np.zeros((rows, 1, P), np.uint8)
    G = grid_plain(pl, ot, vis, w, f, 512, cross_swap=swap)
    Np = normaliser(pl, ot, w, f, cross_swap=swap)
    img = oracle.grid_correct_stokes(G, Np, ot.beta, wl.taper_support, feeds)
    return img[0, :, 256, 256]


@pytest.mark.parametrize("feeds", ["linear", "circular"])
def test_point_source_stokes_recovered_with_swap(geom, feeds):
    wl, ot, pl = geom
    got = _centre(wl, ot, pl, feeds, True)
    assert np.allclose(got, STOKES, atol=2e-3), got


def test_in_place_conjugation_loses_v(geom):
    wl, ot, pl = geom
    got = _centre(wl, ot, pl, "linear", False)
    assert np.allclose(got[:3], STOKES[:3], atol=2e-3)       # I, Q, U are unaffected
    assert abs(got[3] - STOKES[3]) > 0.2 * STOKES[3]           # V is not


@pytest.mark.parametrize("feeds,expect", [("linear", (STOKES[0], STOKES[1])), ("circular", (STOKES[0], STOKES[3]))])
def test_dual_polarisation_gives_two_stokes(geom, feeds, expect):
    wl, ot, pl = geom
    got = _centre(wl, ot, pl, feeds, True, P=2)
    assert got.shape == (2,) and np.allclose(got, expect, atol=2e-3)


def test_swap_keeps_compression_invariance_and_adjoint(geom):
    wl, ot, pl = geom
    rows = wl.uvw.shape[0]
    rng = np.random.default_rng(5)
    y = (rng.normal(size=(rows, 1, 4)) + 1j * rng.normal(size=(rows, 1, 4))).astype(np.complex64)
    w = np.ones((rows, 1, 4), np.float32)
    f = (rng.random((rows, 1, 4)) < 0.05).astype(np.uint8)
    G = grid_plain(pl, ot, y, w, f, 512, cross_swap=True)
    Gc = grid_compressed(pl, ot, y, w, f, 512, cross_swap=True)
    assert np.max(np.abs(Gc - G)) <= 1e-12 * np.abs(G).max()
    # adjoint under Re<.,.>: Re<G(y), X> = Re<y, G^H(X)>
    X = rng.normal(size=G.shape) + 1j * rng.normal(size=G.shape)
    lhs = np.real(np.vdot(G, X))
    rhs = np.real(np.vdot(y.reshape(-1, 4).astype(np.complex128),
                          degrid(pl, ot, X, w, f, adjoint=True, cross_swap=True)))
    assert abs(lhs - rhs) <= 1e-9 * abs(lhs)
