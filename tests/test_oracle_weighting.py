"""Pins of the oracle's uniform and robust weighting (definitions in oracle/weighting.py):
hand-computed weights for records sharing a cell, the uniform invariant (each occupied cell's
new weights sum to one), the natural and uniform limits of robust weighting, and the Hermitian
halves meeting in one cell."""
import numpy as np
import pytest

import oracle
import synth
from oracle.weighting import density, reweight


def _pl(uvw, du=1.0, N=64):
    tab = oracle.delta_table() if hasattr(oracle, "delta_table") else None
    return oracle.place(np.asarray(uvw, np.float64), np.array([synth.C0]), du, N, tab)


def test_hand_computed_cell_shares():
    # three records: two in the cell of u = 3 (weights 1 and 3), one alone at u = 10 (weight 2);
    # the delta table puts each record in the cell of its u (du = 1, f = c0: u' is u in wavelengths)
    uvw = np.array([[3.1, 0.0, 0.0], [2.9, 0.2, 0.0], [10.0, 0.0, 0.0]])
    pl = _pl(uvw)
    w = np.array([1.0, 3.0, 2.0]).reshape(3, 1, 1)
    f = np.zeros((3, 1, 1), np.uint8)
    uni = reweight(pl, w, f, 64, "uniform").ravel()
    assert np.allclose(uni, [0.25, 0.75, 1.0], rtol=1e-15)
    # robust: W = (4, 4, 2), sum W^2 over cells = 16 + 4 = 20, sum w = 6, f^2 = 25 / (20/6) at R = 0
    f2 = 25.0 / (20.0 / 6.0)
    rob = reweight(pl, w, f, 64, "robust", robust=0.0).ravel()
    assert np.allclose(rob, [1 / (1 + 4 * f2), 3 / (1 + 4 * f2), 2 / (1 + 2 * f2)], rtol=1e-15)


def test_conjugate_halves_share_a_cell():
    # (u, v, w) and (-u, -v, -w): the second is conjugated onto the first's position
    uvw = np.array([[5.2, -3.1, 1.0], [-5.2, 3.1, -1.0]])
    pl = _pl(uvw)
    assert pl.x[0] == pl.x[1] and pl.y[0] == pl.y[1] and pl.psi[1] < 0
    uni = reweight(pl, np.ones((2, 1, 1)), np.zeros((2, 1, 1), np.uint8), 64, "uniform").ravel()
    assert np.allclose(uni, [0.5, 0.5])


@pytest.fixture(scope="module")
def slice4():
    wl = synth.make("wproj_2k", n_times=80, n_chan=2, n_baselines=150, flag_frac=0.05)
    ot = oracle.build_table(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support, supports=wl.supports)
    pl = oracle.place(wl.uvw, wl.freq, wl.du, wl.n_grid, ot, flag=wl.flag.numpy())
    rng = np.random.default_rng(2)
    w = rng.uniform(0.5, 2.0, wl.weight.shape)
    return wl, pl, w


def test_uniform_weights_sum_to_one_per_cell(slice4):
    wl, pl, w = slice4
    f = wl.flag.numpy()
    uni = reweight(pl, w, f, wl.n_grid, "uniform")
    W1 = density(pl, uni.reshape(w.shape), f, wl.n_grid)
    occ = density(pl, w, f, wl.n_grid) > 0
    assert np.allclose(W1[occ], 1.0, rtol=1e-12)
    assert np.all(W1[~occ] == 0)


def test_robust_limits(slice4):
    wl, pl, w = slice4
    f = wl.flag.numpy()
    sel = pl.griddable
    nat = reweight(pl, w, f, wl.n_grid, "robust", robust=8.0)
    assert np.allclose(nat[sel], w.reshape(-1, 4)[sel], rtol=1e-10)
    uni = reweight(pl, w, f, wl.n_grid, "uniform")
    rob = reweight(pl, w, f, wl.n_grid, "robust", robust=-8.0)
    live = uni[sel] > 0                                          # (a flagged pol alone in its cell has W = 0)
    for p in range(4):
        r = rob[sel][live[:, p], p] / uni[sel][live[:, p], p]
        assert np.allclose(r, r[0], rtol=1e-6)                   # proportional to uniform per pol
