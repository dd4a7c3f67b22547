"""Gridding, compression, normaliser, statistics and degridding, FP64.  Test infrastructure only.

grid_plain       : eq. "gridding" (Sec. 4.3.2) record by record -- the definition.
compress         : the compression of Sec. 4.3.3 with eqs. "compress1"/"conjugatetake"
                   (sequential loop in oracle.c).
grid_compressed  : grids the compressed list; equals grid_plain up to rounding.
normaliser       : eq. "normalizer" (Sec. 4.3.2), N_p per channel.

cross_swap=True is full-Stokes gridding: a take-conjugate (psi = -1) quad-pol record feeds
polarisation 1 from polarisation 2 and 2 from 1, because conj(V_XY(u)) = V_YX(-u).  The thesis
conjugates each polarisation in place (eq. "conjugatetake"), exact for the parallel hands and
for U = (XY + YX)/2 but not for V.

interleave=True is channel interleaving (Sec. 5.4, batch 1: the channels of a record row are
interleaved and all records gridded onto one grid, as in multi-frequency synthesis): the grid
has one channel, a record's predecessor for compression is the previous record in natural
order row*C + chan, and N_p sums over all records.
stats            : the four statistics of Sec. 4.3.4.
degrid           : adjoint of the gridding map.  The vis -> grid map is only R-linear
                   (psi = -1 records are conjugated), so its adjoint under Re<a,b> is
                   conj-back of eps(1-f) * sum_ij conj(K) * grid for each record.
"""
import numpy as np

from .cloops import lib


def _p(a):
    return a.ctypes.data


def _swap_cross(a, pl, cross_swap):
    """Swaps polarisations 1 and 2 of the take-conjugate quad-pol records (cross_swap)."""
    if not cross_swap or a.shape[-1] != 4:
        return a
    b = a.copy()
    neg = pl.psi < 0
    b[neg, 1], b[neg, 2] = a[neg, 2], a[neg, 1]
    return b


def weighted_vis(pl, vis, weight, flag, cross_swap=False) -> np.ndarray:
    """q_{i,p} = eps (1-f) * vis, conjugated where psi = -1 (eq. "conjugatetake"); [rows*C, P]."""
    P = np.asarray(vis).shape[-1]
    v = np.asarray(vis, dtype=np.complex128).reshape(-1, P)
    wf = np.asarray(weight, np.float64).reshape(-1, P) * (1.0 - np.asarray(flag, np.float64).reshape(-1, P))
    q = _swap_cross(wf * v, pl, cross_swap)
    return np.where((pl.psi < 0)[:, None], np.conj(q), q)


def _grid_records(sel, chan, x0, y0, z, S, q, P, N, C, table):
    grid = np.zeros((C, N, N, P), dtype=np.complex128)
    tab = np.ascontiguousarray(table.data, dtype=np.complex128)
    a = [np.ascontiguousarray(v[sel], dtype=t) for v, t in
         ((chan, np.int32), (x0, np.int32), (y0, np.int32), (z, np.int64), (S, np.int32))]
    qq = np.ascontiguousarray(q, dtype=np.complex128)
    lib.or_grid(int(a[0].shape[0]), _p(a[0]), _p(a[1]), _p(a[2]), _p(a[3]), _p(a[4]), _p(qq),
                P, N, _p(tab), _p(grid))
    return grid


def _grid_chan(pl, interleave):
    """(grid channel of every record, number of grid channels)."""
    return (np.zeros_like(pl.chan), 1) if interleave else (pl.chan, pl.C)


def grid_plain(pl, table, vis, weight, flag, n_grid, interleave=False, cross_swap=False):
    """grid[c][y][x][p] = sum over griddable records of q_{i,p} * K_i (eq. "gridding")."""
    P = np.asarray(vis).shape[-1]
    q = weighted_vis(pl, vis, weight, flag, cross_swap)
    sel = pl.griddable
    chan, C = _grid_chan(pl, interleave)
    return _grid_records(sel, chan, pl.x0, pl.y0, pl.z, pl.S, q[sel], P, n_grid, C, table)


def compress(pl, vis, weight, flag, interleave=False, cross_swap=False):
    """Returns (g, c, list_rec, list_last, gamma) following the sequential compression."""
    rows, C = pl.rows, pl.C
    P = np.asarray(vis).shape[-1]
    n = rows * C
    gd = np.ascontiguousarray(pl.griddable, dtype=np.uint8)
    x0 = np.ascontiguousarray(pl.x0, dtype=np.int32)
    y0 = np.ascontiguousarray(pl.y0, dtype=np.int32)
    z = np.ascontiguousarray(pl.z, dtype=np.int64)
    psi = np.ascontiguousarray(pl.psi, dtype=np.int8)
    v = np.ascontiguousarray(np.asarray(vis).reshape(n, P).astype(np.complex64)).view(np.float32)
    w = np.ascontiguousarray(np.asarray(weight, dtype=np.float32).reshape(n, P))
    f = np.ascontiguousarray(np.asarray(flag, dtype=np.uint8).reshape(n, P))
    g = np.zeros(n, np.uint8)
    c = np.zeros(n, np.uint8)
    head = np.zeros(n, np.int64)
    lrec = np.zeros(n, np.int64)
    llast = np.zeros(n, np.int64)
    gamma = np.zeros((n, P), np.complex128)
    ne = lib.or_compress(rows, C, P, 1 if interleave else 0, 1 if cross_swap else 0, _p(gd), _p(x0), _p(y0), _p(z), _p(psi), _p(v), _p(w), _p(f),
                         _p(g), _p(c), _p(head), _p(lrec), _p(llast), _p(gamma))
    return (g.astype(bool), c.astype(bool), lrec[:ne].copy(), llast[:ne].copy(), gamma[:ne].copy())


def grid_compressed(pl, table, vis, weight, flag, n_grid, interleave=False, cross_swap=False):
    P = np.asarray(vis).shape[-1]
    g, c, lrec, llast, gamma = compress(pl, vis, weight, flag, interleave, cross_swap)
    chan, C = _grid_chan(pl, interleave)
    return _grid_records(lrec, chan, pl.x0, pl.y0, pl.z, pl.S, gamma, P, n_grid, C, table)


def normaliser(pl, table, weight, flag, interleave=False, cross_swap=False) -> np.ndarray:
    """N[c][p] = sum_i eps (g+c)(1-f) zeta_i  (eq. "normalizer"); (g+c) = griddable.
    Interleaved: one row, the sum over all records.  With cross_swap, the weights of the
    polarisation each record feeds."""
    rows, C = pl.rows, pl.C
    P = np.asarray(weight).shape[-1]
    wf = np.asarray(weight, np.float64).reshape(-1, P) * (1.0 - np.asarray(flag, np.float64).reshape(-1, P))
    wf = _swap_cross(wf, pl, cross_swap)
    zeta = np.where(pl.griddable, table.zeta[np.maximum(pl.zeta_idx, 0)], 0.0)
    contrib = wf * zeta[:, None]
    chan, C = _grid_chan(pl, interleave)
    out = np.zeros((C, P))
    np.add.at(out, chan, contrib)
    return out


def stats(pl, g, c):
    """Sec. 4.3.4: records gridded, records compressed, grid-point updates executed by the
    gridder and saved by compression (per polarisation; multiply by P for the metric)."""
    S2 = pl.S.astype(np.int64) ** 2
    return {"gridded": int(g.sum()), "compressed": int(c.sum()),
            "updates": int((S2 * g).sum()), "updates_saved": int((S2 * c).sum())}


def degrid(pl, table, grid, weight=None, flag=None, adjoint=False, interleave=False,
           cross_swap=False) -> np.ndarray:
    """Per record: m_p = sum_ij conj(K) grid_p over the footprint, conjugated back where
    psi = -1.  adjoint=True also applies eps (1 - f), giving the exact adjoint of the
    vis -> grid map.  Non-griddable records get 0.  Returns complex128 [rows*C, P]."""
    C, N, _, P = grid.shape
    sel = np.nonzero(pl.griddable)[0]
    chan, _ = _grid_chan(pl, interleave)
    a = [np.ascontiguousarray(v[sel], dtype=t) for v, t in
         ((chan, np.int32), (pl.x0, np.int32), (pl.y0, np.int32), (pl.z, np.int64), (pl.S, np.int32))]
    m = np.zeros((sel.shape[0], P), np.complex128)
    g = np.ascontiguousarray(grid, dtype=np.complex128)
    tab = np.ascontiguousarray(table.data, dtype=np.complex128)
    lib.or_degrid(int(sel.shape[0]), _p(a[0]), _p(a[1]), _p(a[2]), _p(a[3]), _p(a[4]), P, N,
                  _p(tab), _p(g), _p(m))
    m = np.where((pl.psi[sel] < 0)[:, None], np.conj(m), m)
    out = np.zeros((pl.rows * pl.C, P), np.complex128)
    out[sel] = m
    out = _swap_cross(out, pl, cross_swap)      # the adjoint of the swap is the swap
    if adjoint:
        wf = np.asarray(weight, np.float64).reshape(-1, P) * (1.0 - np.asarray(flag, np.float64).reshape(-1, P))
        out = out * wf
    return out
