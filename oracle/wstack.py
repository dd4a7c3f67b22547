"""W-stacking (thesis Sec. 2.2.2, eq. "stacking"), FP64.  Test infrastructure only.

The records are partitioned in w and each part is gridded onto its own constant-w grid with the
w = 0 kernel; after the inverse Fourier transform each plane is divided by its w-term g_w(l, m),
which for the -j2pi measurement-equation convention means multiplying by exp(+j2pi w_k (n-1)),
and the planes are added.  The partition is the w-projection one (the nearest plane k in
sqrt(w), Sec. 2.2.1), so placement and compression are unchanged; plane k's correction uses its
w_k = w_max (k/(K-1))^2, and pixels outside the unit disk (l^2 + m^2 >= 1) are set to zero.
The image is then the real part, divided by N_p and by taper x sinc as in Algorithm
"finalizer".
"""
import numpy as np

from .correct import dirty_complex, sinc_1d, taper_1d
from .grid import _grid_records, weighted_vis
from .table import build_table, exact_screen


def stacking_table(du, n_wplanes, w_max, beta, taper_support=7, supports=None, n_k=None):
    """K planes that all hold the w = 0 kernel (the w-projection plane values are kept)."""
    return build_table(du, n_wplanes, w_max, beta, taper_support, supports=supports, n_k=n_k,
                       screen=lambda w, l, m: exact_screen(0.0, l, m))


def grid_stacked(pl, table, vis, weight, flag, n_grid):
    """grid [C*K][N][N][P]: record (r, c) in plane k goes to grid c*K + k."""
    P = np.asarray(vis).shape[-1]
    q = weighted_vis(pl, vis, weight, flag)
    sel = pl.griddable
    K = table.K
    chan = pl.chan.astype(np.int64) * K + np.where(sel, pl.k, 0)
    return _grid_records(sel, chan, pl.x0, pl.y0, pl.z, pl.S, q[sel], P, n_grid, pl.C * K, table)


def nm1_grid(n_grid, du):
    """n - 1 = -r^2 / (1 + sqrt(1 - r^2)) at every pixel ([N][N], rows m), 0 outside the disk,
    with a mask of the pixels inside."""
    l = (np.arange(n_grid) - n_grid // 2) / (n_grid * du)
    L, M = np.meshgrid(l, l, indexing="xy")
    r2 = L * L + M * M
    inside = r2 < 1.0
    return np.where(inside, -r2 / (1.0 + np.sqrt(np.where(inside, 1.0 - r2, 1.0))), 0.0), inside


def image_stacked(grid, norm, table, taper_support, du):
    """[C*K][N][N][P] grids -> [C][P][N][N] images."""
    CK, N, _, P = grid.shape
    K = table.K
    C = CK // K
    nm1, inside = nm1_grid(N, du)
    z = dirty_complex(grid).reshape(C, K, P, N, N)
    screens = np.stack([np.where(inside, np.exp(2j * np.pi * table.w_planes[k] * nm1), 0.0) for k in range(K)])
    acc = (z * screens[None, :, None, :, :]).sum(axis=1)
    nz = np.where(norm != 0, norm, 1.0)
    img = acc.real * np.where(norm != 0, 1.0 / nz, 0.0)[:, :, None, None]
    t = taper_1d(N, taper_support) * sinc_1d(N, table.beta)
    return img / (t[None, None, :, None] * t[None, None, None, :])
