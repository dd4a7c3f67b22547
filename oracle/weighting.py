"""Uniform and robust weighting, FP64.  Test infrastructure only.

The thesis names the schemes (Sec. 2.1, "Deconvolution and weighting schemes": uniform
weighting divides each weight by the density of measurements around it, natural weighting
keeps the inverse-variance weights, robust weighting after Briggs compromises between them)
and grids with natural weights only.  Written out from those published definitions:

  density   W_p(cell) = sum of eps_p (1 - f_p) over the griddable records in the grid cell
            (x, y) of their placement (one grid per channel; one grid when interleaved), per
            polarisation p; records of both Hermitian halves meet in one cell (psi trick);
  uniform   eps'_p = eps_p / W_p(cell)
  robust    eps'_p = eps_p / (1 + W_p(cell) f_p^2),  f_p^2 = (5 10^-R)^2 / (sum_cells W_p^2 /
            sum_records eps_p (1 - f_p)),  R the robustness (about -2: uniform, +2: natural)

Records that are not griddable keep their weights (they are never gridded).
"""
import numpy as np


def density(pl, weight, flag, n_grid, interleave=False):
    """W [C or 1][N][N][P] (FP64)."""
    P = np.asarray(weight).shape[-1]
    wf = np.asarray(weight, np.float64).reshape(-1, P) * (1.0 - np.asarray(flag, np.float64).reshape(-1, P))
    C = 1 if interleave else pl.C
    W = np.zeros((C, n_grid, n_grid, P))
    sel = pl.griddable
    ch = np.zeros_like(pl.chan) if interleave else pl.chan
    np.add.at(W, (ch[sel], pl.y[sel], pl.x[sel]), wf[sel])
    return W


def reweight(pl, weight, flag, n_grid, scheme, robust=0.0, interleave=False):
    """New weights [rows*C, P] (FP64) for scheme "uniform" or "robust"."""
    P = np.asarray(weight).shape[-1]
    w = np.asarray(weight, np.float64).reshape(-1, P)
    wf = w * (1.0 - np.asarray(flag, np.float64).reshape(-1, P))
    W = density(pl, weight, flag, n_grid, interleave)
    sel = pl.griddable
    ch = np.zeros_like(pl.chan) if interleave else pl.chan
    d = W[ch[sel], pl.y[sel], pl.x[sel]]                     # [n_sel, P]
    out = w.copy()
    if scheme == "uniform":
        out[sel] = np.where(d > 0, w[sel] / np.where(d > 0, d, 1.0), 0.0)
    elif scheme == "robust":
        f2 = (5.0 * 10.0 ** (-robust)) ** 2 / ((W ** 2).sum(axis=(0, 1, 2)) / wf[sel].sum(axis=0))
        out[sel] = w[sel] / (1.0 + d * f2[None, :])
    else:
        raise ValueError(scheme)
    return out
