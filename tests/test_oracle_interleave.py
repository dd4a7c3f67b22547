"""Pins of the oracle's channel interleaving (Sec. 5.4 batch 1: channels interleaved and all
records gridded on one grid; compression then runs over the natural record order, across
channels).  Checked against the definitions, not against the oracle itself: a pure-Python
loop over eq. "ci" in interleaved order, compression invariance of the grid, the one-grid
definition as the sum of the channel grids, and a closed-form compression count."""
import numpy as np
import pytest

import oracle
import synth
from oracle.grid import compress, grid_compressed, grid_plain, normaliser, weighted_vis


@pytest.fixture(scope="module")
def case():
    wl = synth.make("mfs_2k", n_times=40, n_chan=3, n_baselines=60, flag_frac=0.05)
    ot = oracle.build_table(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support, supports=wl.supports)
    f = wl.flag.numpy()
    pl = oracle.place(wl.uvw, wl.freq, wl.du, wl.n_grid, ot, flag=f)
    return wl, ot, pl


def test_indicators_follow_eq_ci_in_interleaved_order(case):
    wl, ot, pl = case
    vis, w, f = wl.vis.numpy(), wl.weight.numpy(), wl.flag.numpy()
    g, c, lrec, llast, gamma = compress(pl, vis, w, f, interleave=True)
    n = pl.griddable.size
    eg = np.zeros(n, bool)
    ec = np.zeros(n, bool)
    heads, runs = [], []
    for i in range(n):                       # eq. "ci" over i = row*C + chan
        if not pl.griddable[i]:
            continue
        if i > 0 and pl.griddable[i - 1] and pl.x0[i] == pl.x0[i - 1] and pl.y0[i] == pl.y0[i - 1] \
                and pl.z[i] == pl.z[i - 1]:
            ec[i] = True
            runs[-1].append(i)
        else:
            eg[i] = True
            heads.append(i)
            runs.append([i])
    assert np.array_equal(g, eg) and np.array_equal(c, ec)
    assert np.array_equal(lrec, heads) and np.array_equal(llast, [r[-1] for r in runs])
    q = weighted_vis(pl, vis, w, f)
    for e in range(0, len(runs), 7):
        assert np.allclose(gamma[e], q[runs[e]].sum(0), rtol=1e-12, atol=1e-12)
    assert c.sum() > 0


def test_one_grid_is_the_sum_of_the_channel_grids_and_compression_keeps_it(case):
    wl, ot, pl = case
    vis, w, f = wl.vis.numpy(), wl.weight.numpy(), wl.flag.numpy()
    per_chan = grid_plain(pl, ot, vis, w, f, wl.n_grid)
    one = grid_plain(pl, ot, vis, w, f, wl.n_grid, interleave=True)
    assert one.shape == (1,) + per_chan.shape[1:]
    assert np.allclose(one[0], per_chan.sum(0), rtol=0, atol=1e-12 * np.abs(one).max())
    comp = grid_compressed(pl, ot, vis, w, f, wl.n_grid, interleave=True)
    assert np.max(np.abs(comp - one)) <= 1e-12 * np.abs(one).max()
    n1 = normaliser(pl, ot, w, f, interleave=True)
    assert np.allclose(n1[0], normaliser(pl, ot, w, f).sum(0), rtol=1e-14)


def test_identical_channels_compress_across_channels():
    # two channels at the same frequency place every record identically, so each (row, 1)
    # compresses into (row, 0), and (row, 0) into (row-1, 1) exactly when row and row-1 share
    # the footprint origin and kernel pointer
    wl = synth.make("w0_small", n_times=64)
    uvw = wl.uvw
    freq = np.array([wl.freq[0], wl.freq[0]])
    ot = oracle.build_table(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support, supports=wl.supports)
    pl = oracle.place(uvw, freq, wl.du, wl.n_grid, ot)
    rows = uvw.shape[0]
    vis = np.ones((rows, 2, 1), np.complex64)
    w = np.ones((rows, 2, 1), np.float32)
    f = np.zeros((rows, 2, 1), np.uint8)
    g, c, *_ = compress(pl, vis, w, f, interleave=True)
    gd = pl.griddable.reshape(rows, 2)[:, 0]
    x0, y0, z = (a.reshape(rows, 2)[:, 0] for a in (pl.x0, pl.y0, pl.z))
    same_prev = np.zeros(rows, bool)
    same_prev[1:] = gd[1:] & gd[:-1] & (x0[1:] == x0[:-1]) & (y0[1:] == y0[:-1]) & (z[1:] == z[:-1])
    assert c.reshape(rows, 2)[:, 1].sum() == gd.sum()
    assert np.array_equal(c.reshape(rows, 2)[:, 0], same_prev)
    assert g.sum() == gd.sum() - same_prev.sum()
