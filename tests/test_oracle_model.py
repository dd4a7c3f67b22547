"""Pins for the oracle's forward model A (sky image -> visibilities by degridding) and its
adjoint: the adjoint identity in FP64, the transpose pair of the image/grid transforms, and
central finite differences of chi^2 = sum |A x - v|^2 against 2 A^H (A x - v) on a 64 x 64
sub-problem with w-projection, flags and both signs of w."""
import numpy as np

import oracle
from oracle import model

C0 = 299_792_458.0


def _problem(seed=1, n=120, P=2, N=64, du=2.0, K=5, w_max=40.0):
    rng = np.random.default_rng(seed)
    tab = oracle.build_table(du, K, w_max, 8, 7, n_k=64)
    lim = (N // 2 - int(tab.supports.max()) // 2 - 2) * du
    uvw = np.stack([rng.uniform(-lim, lim, n), rng.uniform(-lim, lim, n), rng.uniform(-w_max, w_max, n)], 1)
    freq = np.array([C0, 1.05 * C0])
    fl = (rng.random((n, 2, P)) < 0.05).astype(np.uint8)
    fl[::17] = 1                                  # some records fully flagged
    pl = oracle.place(uvw, freq, du, N, tab, flag=fl)
    return rng, tab, pl, N, P


def test_image_grid_transpose_pair():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 2, 16, 16))
    g = rng.normal(size=(2, 16, 16, 2)) + 1j * rng.normal(size=(2, 16, 16, 2))
    lhs = np.real(np.vdot(model.image_to_grid(x, 8, 7), g))
    rhs = np.vdot(x, model.grid_to_image(g, 8, 7))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_forward_adjoint_identity():
    rng, tab, pl, N, P = _problem()
    assert pl.griddable.sum() > 150 and (~pl.griddable).sum() > 5
    x = rng.normal(size=(2, P, N, N))
    y = rng.normal(size=(pl.rows * 2, P)) + 1j * rng.normal(size=(pl.rows * 2, P))
    Ax = model.forward(pl, tab, x, 7)
    lhs = np.real(np.vdot(Ax, y))
    rhs = np.vdot(x, model.adjoint(pl, tab, y, N, 7))
    # 1/(taper sinc) reaches ~2.5e7 at the field corners: FP64 rounding of the sums is ~1e-11
    assert abs(lhs - rhs) <= 1e-9 * abs(lhs)


def test_chi2_gradient_finite_differences():
    rng, tab, pl, N, P = _problem(seed=2)
    x = rng.normal(size=(2, P, N, N)) * 1e-3
    v = rng.normal(size=(pl.rows * 2, P)) + 1j * rng.normal(size=(pl.rows * 2, P))
    f0, g = model.chi2_grad(pl, tab, x, v, 7)
    for _ in range(4):
        d = rng.normal(size=x.shape)
        h = 1e-4
        fp, _ = model.chi2_grad(pl, tab, x + h * d, v, 7)
        fm, _ = model.chi2_grad(pl, tab, x - h * d, v, 7)
        fd = (fp - fm) / (2 * h)
        an = float(np.sum(g * d))
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (fd, an)
