"""Pins of the oracle's w-stacking (eq. "stacking"): against the direct Fourier transform with
w-terms on tiny inputs (records on the w-planes, both signs of w), the same bar as the
w-projection end-to-end pin; dropping the plane phase correction must fail it; and with every
record at w = 0 the stacked image is the plain w = 0 image."""
import dataclasses

import numpy as np

import oracle
import synth
from oracle.wstack import grid_stacked, image_stacked, stacking_table
from test_oracle_grid import _records

C0 = 299_792_458.0


def _case(K, w_max, seed=7):
    rng = np.random.default_rng(seed)
    N, du, beta, n = 64, 2.0, 64, 200
    tab = stacking_table(du, K, w_max, beta, 7, n_k=64)
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
    ref = oracle.dirty_image(uvw, freq, vis, wt, fl, N, du)[0, 0]
    return N, du, tab, pl, vis, wt, fl, ref


def test_stacked_image_against_direct_fourier():
    N, du, tab, pl, vis, wt, fl, ref = _case(17, 60.0)
    G = grid_stacked(pl, tab, vis, wt, fl, N)
    assert G.shape[0] == 17
    img = image_stacked(G, oracle.normaliser(pl, tab, wt, fl), tab, 7, du)[0, 0]
    inner = slice(N // 4, 3 * N // 4)
    err = np.max(np.abs(img - ref)[inner, inner]) / np.max(np.abs(ref))
    assert err < 5e-3, err
    # without the per-plane phase correction the w-terms stay in the image
    tab0 = dataclasses.replace(tab, w_planes=np.zeros_like(tab.w_planes))
    bad = image_stacked(G, oracle.normaliser(pl, tab, wt, fl), tab0, 7, du)[0, 0]
    assert np.max(np.abs(bad - ref)[inner, inner]) / np.max(np.abs(ref)) > 10 * err


def test_all_records_at_w0_give_the_plain_image():
    N, du, tab, pl, vis, wt, fl, ref = _case(1, 0.0)
    G1 = grid_stacked(pl, tab, vis, wt, fl, N)
    img = image_stacked(G1, oracle.normaliser(pl, tab, wt, fl), tab, 7, du)
    G = oracle.grid_plain(pl, tab, vis, wt, fl, N)
    plain = oracle.grid_correct(G, oracle.normaliser(pl, tab, wt, fl), tab.beta, 7)
    assert np.max(np.abs(img - plain)) <= 1e-12 * np.max(np.abs(plain))


def test_stacking_table_planes_hold_the_w0_kernel():
    tab = stacking_table(2.0, 5, 60.0, 8, 7, supports=[7] * 5)
    w0 = oracle.build_table(2.0, 1, 0.0, 8, 7, supports=[7])
    for k in range(5):
        assert np.array_equal(tab.data[tab.offsets[k]:tab.offsets[k] + 64 * 49], w0.data)
    assert tab.w_planes[-1] == 60.0
