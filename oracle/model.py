"""Sky -> visibility forward model built from degridding, and its adjoint, FP64.  Test
infrastructure only.

A(x): a real sky image x [C][P][N][N] (one plane per channel and polarisation) is divided by the
grid-correction function taper x sinc (Sec. 4.7 steps 3-4), transformed with the centred
forward DFT (the inverse of the imaging transform of step 1; exponent -j2pi(ul + vm), the
measurement equation's sign), and degridded (the adjoint of eq. "gridding") to predict every
griddable record's visibilities (psi-conjugated back; 0 for records that are not griddable).

A^H(y): the adjoint of A under the real inner product Re<a, b>: the visibilities are gridded
with unit weights (psi-conjugated, all polarisations of every griddable record), inverse
transformed without normalisation, real part, divided by taper x sinc.  The gradient of
chi^2(x) = sum |A x - v|^2 is 2 A^H (A x - v).
"""
import numpy as np

from .correct import sinc_1d, taper_1d
from .grid import _grid_records, degrid


def _icorr(N, beta, taper_support):
    return 1.0 / (taper_1d(N, taper_support) * sinc_1d(N, beta))


def image_to_grid(image, beta, taper_support):
    """[C, P, N, N] real -> [C, N, N, P] complex: centred forward DFT of image / corr."""
    C, P, N, _ = image.shape
    ic = _icorr(N, beta, taper_support)
    x = image * (ic[None, None, :, None] * ic[None, None, None, :])
    G = np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(x, axes=(-2, -1)), axes=(-2, -1)), axes=(-2, -1))
    return np.ascontiguousarray(np.moveaxis(G, 1, 3))


def grid_to_image(grid, beta, taper_support):
    """[C, N, N, P] complex -> [C, P, N, N] real: Re of the centred inverse DFT (unnormalised),
    divided by corr (the transpose of image_to_grid)."""
    C, N, _, P = grid.shape
    g = np.moveaxis(grid, 3, 1)
    img = np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(g, axes=(-2, -1)), axes=(-2, -1)), axes=(-2, -1)) * (N * N)
    ic = _icorr(N, beta, taper_support)
    return img.real * (ic[None, None, :, None] * ic[None, None, None, :])


def forward(pl, table, image, taper_support):
    """A(x): predicted visibilities [rows*C, P] (complex128)."""
    G = image_to_grid(np.asarray(image, np.float64), table.beta, taper_support)
    return degrid(pl, table, G, adjoint=False)


def adjoint(pl, table, vis, n_grid, taper_support):
    """A^H(y): [C, P, N, N] real image."""
    P = vis.shape[-1]
    q = np.asarray(vis, np.complex128).reshape(-1, P)
    q = np.where((pl.psi < 0)[:, None], np.conj(q), q)
    sel = pl.griddable
    G = _grid_records(sel, pl.chan, pl.x0, pl.y0, pl.z, pl.S, q[sel], P, n_grid, pl.C, table)
    return grid_to_image(G, table.beta, taper_support)


def chi2_grad(pl, table, image, vis_obs, taper_support):
    """(chi^2, gradient) for chi^2(x) = sum |A x - v|^2."""
    r = forward(pl, table, image, taper_support) - np.asarray(vis_obs, np.complex128).reshape(-1, image.shape[1])
    r = np.where(pl.griddable[:, None], r, 0.0)
    return float(np.sum(np.abs(r) ** 2)), 2.0 * adjoint(pl, table, r, image.shape[-1], taper_support)
