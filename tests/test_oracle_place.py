"""Pins for the oracle's placement and classification (Sec. 4.2.2 eqs. "choose"/"sat",
Sec. 4.3.3 position tuple, Sec. 4.3.4 eq. "conj", griddability of Sec. 4.3.2).

Expected cells come from exact rational arithmetic (fractions.Fraction) on inputs chosen so
that the FP64 products are exact, including the tie cases t = k + 1/2 which must round
down (delta-u in (-du/2, du/2]).  The delta kernel (S = 1, beta = 1, one plane) must put
every visibility in exactly that cell.
"""
from fractions import Fraction
import math

import numpy as np
import pytest

import oracle
from oracle.table import Table

C0 = 299_792_458.0


def _table(beta, supports, w_max=0.0):
    K = len(supports)
    sup = np.asarray(supports, np.int32)
    offs = np.concatenate([[0], np.cumsum(beta * beta * sup.astype(np.int64) ** 2)[:-1]])
    n = int((beta * beta * sup.astype(np.int64) ** 2).sum())
    return Table(beta, sup, offs.astype(np.int64), np.ones(n, complex), np.ones(K * beta * beta),
                 oracle.table.w_plane_values(K, w_max), w_max)


def _exact_cell(t: Fraction, beta: int):
    q = math.ceil(t - Fraction(1, 2))
    xc = math.ceil(Fraction(q, 1) / beta - Fraction(1, 2))
    return xc, q - beta * xc


@pytest.mark.parametrize("beta", [1, 2, 4, 8])
def test_exact_cell_and_suboffset(beta):
    rng = np.random.default_rng(beta)
    du = 0.5                       # power of two: sc = beta / du exact; f = c0 gives lam_inv = 1
    N = 256
    u = rng.integers(-4000, 4000, 500) / 64.0
    v = rng.integers(-4000, 4000, 500) / 64.0
    # add exact ties at half the oversampled step
    u[:50] = (2 * rng.integers(-200, 200, 50) + 1) * du / (2 * beta)
    w = rng.integers(0, 100, 500) / 8.0
    uvw = np.stack([u, v, w], 1)
    tab = _table(beta, [1])
    pl = oracle.place(uvw, np.array([C0]), du, N, tab)
    for i in range(500):
        xc, fu = _exact_cell(Fraction(u[i]) * beta / Fraction(du), beta)
        yc, fv = _exact_cell(Fraction(v[i]) * beta / Fraction(du), beta)
        assert (pl.x[i], pl.fu[i]) == (N // 2 + xc, fu)
        assert (pl.y[i], pl.fv[i]) == (N // 2 + yc, fv)
        assert -beta / 2 < fu <= beta / 2


def test_take_conjugate_flips_baseline():
    uvw = np.array([[3.25, -1.5, 2.0], [3.25, -1.5, -2.0], [-3.25, 1.5, 0.0]])
    tab = _table(4, [1])
    pl = oracle.place(uvw, np.array([C0]), 0.5, 64, tab)
    assert list(pl.psi) == [1, -1, 1]
    # these inputs sit exactly on the oversampled lattice: record 1 is gridded at (-u, -v),
    # the mirror of record 0, and record 2 (w = 0 keeps psi = +1) lands where record 1 does
    q = lambda x, f: 4 * (x - 32) + f  # noqa: E731
    assert q(pl.x[1], pl.fu[1]) == -q(pl.x[0], pl.fu[0]) == 4 * -6.5
    assert q(pl.y[1], pl.fv[1]) == -q(pl.y[0], pl.fv[0]) == 4 * 3.0
    assert (pl.x[2], pl.fu[2], pl.y[2], pl.fv[2]) == (pl.x[1], pl.fu[1], pl.y[1], pl.fv[1])
    assert pl.w[1] == 2.0 and pl.w[0] == 2.0


def test_nearest_plane_in_sqrt_w():
    K, w_max = 17, 900.0
    tab = _table(1, [1] * K, w_max)
    rng = np.random.default_rng(5)
    w = rng.uniform(0, 1.3 * w_max, 2000)
    uvw = np.stack([np.zeros_like(w), np.zeros_like(w), w], 1)
    pl = oracle.place(uvw, np.array([C0]), 1.0, 64, tab)
    planes = tab.w_planes
    for i in range(w.size):
        d = np.abs(np.sqrt(w[i]) - np.sqrt(planes))
        k = int(np.argmin(d))
        if np.sqrt(w[i]) > np.sqrt(w_max) + 0.5 * (np.sqrt(w_max) / (K - 1)):
            assert not pl.griddable[i]
        else:
            assert pl.k[i] == k and pl.griddable[i]


def test_footprint_edges_and_flags():
    N, S, beta, du = 32, 7, 1, 1.0
    tab = _table(beta, [S])
    h = (S - 1) // 2
    xs = np.array([h, h - 1, N - 1 - h, N - h])            # first/last fitting cell, and one beyond
    u = (xs - N // 2) * du
    uvw = np.stack([u, np.zeros(4), np.zeros(4)], 1)
    flag = np.zeros((4, 1, 2), np.uint8)
    pl = oracle.place(uvw, np.array([C0]), du, N, tab, flag=flag)
    assert list(pl.griddable) == [True, False, True, False]
    assert pl.x0[0] == 0 and pl.x0[2] + S - 1 == N - 1
    flag[0, 0, :] = 1          # all polarisations flagged -> not griddable
    flag[2, 0, 0] = 1          # one polarisation flagged -> still griddable
    pl = oracle.place(uvw, np.array([C0]), du, N, tab, flag=flag)
    assert list(pl.griddable) == [False, False, True, False]


def test_delta_kernel_places_exactly():
    rng = np.random.default_rng(11)
    N, du = 64, 0.5
    tab = oracle.delta_table()
    n = 400
    u = rng.integers(-900, 900, n) / 32.0
    v = rng.integers(-900, 900, n) / 32.0
    w = rng.integers(-50, 50, n) / 4.0
    uvw = np.stack([u, v, w], 1)
    vis = (rng.normal(size=(n, 1, 1)) + 1j * rng.normal(size=(n, 1, 1))).astype(np.complex64)
    wt = np.ones((n, 1, 1), np.float32)
    fl = np.zeros((n, 1, 1), np.uint8)
    pl = oracle.place(uvw, np.array([C0]), du, N, tab, flag=fl)
    G = oracle.grid_plain(pl, tab, vis, wt, fl, N)
    ref = np.zeros((N, N), complex)
    for i in range(n):
        s = -1 if w[i] < 0 else 1
        xc, _ = _exact_cell(Fraction(s * u[i]) / Fraction(du), 1)
        yc, _ = _exact_cell(Fraction(s * v[i]) / Fraction(du), 1)
        x, y = N // 2 + xc, N // 2 + yc
        if 0 <= x < N and 0 <= y < N:
            val = complex(vis[i, 0, 0])
            ref[y, x] += val.conjugate() if s < 0 else val
    assert np.array_equal(G[0, :, :, 0], ref)
