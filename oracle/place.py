"""Record placement and classification, FP64.  Test infrastructure only.

Placement of record (row, chan) (thesis Sec. 4.2.2 eqs. "choose"/"sat"; Sec. 4.3.3
position tuple; Sec. 4.3.4 eq. "conj"), written as plain FP64 steps, each rounded once:

  lam_inv = f_c / c0                              (input I-2 of Sec. 4.3.2)
  sc      = lam_inv * (beta / du)                 (oversampled lattice units per metre)
  tu, tv  = u' * sc, v' * sc ;  w = w' * lam_inv
  psi     = +1 if w' >= 0 else -1 ; if psi = -1: tu, tv, w = -tu, -tv, -w
  q       = ceil(t - 0.5)           nearest sample at resolution du/beta, ties downward,
                                     so the residual lies in (-du/2, du/2] (eq. "sat")
  x_c     = ceil((q - beta/2) / beta)  (integer arithmetic), frac = q - beta x_c
            in (-beta/2, beta/2]
  x       = N/2 + x_c                (u = 0 in the middle of the grid, Sec. 4.3.3)
  k       = number of m in 1..K-1 with w >= b_m, where b_m = w_max * (t_m * t_m),
            t_m = (m - 0.5) / (K - 1): the squared midpoints between planes in sqrt(w), so k is
            the nearest plane in sqrt(w) (Sec. 2.2.1 / 4.2.1), ties upward; w >= b_K is beyond
            the last plane by more than half a spacing and not griddable
  S = S_k, h = (S-1)/2, footprint origin (x0, y0) = (x - h, y - h)
  z       = offset_k + ((frac_v - lo) * beta + (frac_u - lo)) * S^2,  lo = -((beta-1)//2)

A record is griddable iff k <= K-1, the whole S x S footprint lies inside [0, N)^2, and
at least one polarisation is unflagged (Sec. 4.3.2).
"""
import dataclasses

import numpy as np

C0 = 299_792_458.0


@dataclasses.dataclass
class Placement:
    rows: int
    C: int
    x: np.ndarray        # [rows*C] int64 cell column
    y: np.ndarray
    fu: np.ndarray       # sub-cell offsets in (-beta/2, beta/2]
    fv: np.ndarray
    k: np.ndarray        # w-plane index (may exceed K-1)
    psi: np.ndarray      # int8 take-conjugate sign
    w: np.ndarray        # |w| in wavelengths
    S: np.ndarray        # support (0 where k > K-1)
    x0: np.ndarray       # footprint origin
    y0: np.ndarray
    z: np.ndarray        # int64 kernel pointer (-1 where not griddable)
    zeta_idx: np.ndarray # index into C-3 (-1 where not griddable)
    griddable: np.ndarray  # bool
    chan: np.ndarray     # int32 channel of each record


def plane_bounds(K: int, w_max: float) -> np.ndarray:
    """b_m = w_max * (t * t), t = (m - 0.5) / (K - 1), for m = 1..K (FP64, each op rounded once)."""
    out = np.empty(K)
    for m in range(1, K + 1):
        t = (m - 0.5) / (K - 1)
        out[m - 1] = w_max * (t * t)
    return out


def _cell(q: np.ndarray, beta: int):
    qi = q.astype(np.int64)
    xc = (2 * qi + beta - 1) // (2 * beta)        # = ceil((q - beta/2) / beta)
    return xc, qi - beta * xc


def place(uvw_m: np.ndarray, freq_hz: np.ndarray, du: float, n_grid: int, table, flag=None) -> Placement:
    """Place every record (row, chan), record index i = row * C + chan."""
    uvw_m = np.asarray(uvw_m, dtype=np.float64)
    freq_hz = np.asarray(freq_hz, dtype=np.float64)
    rows, C = uvw_m.shape[0], freq_hz.shape[0]
    beta, K = table.beta, table.K
    lam_inv = freq_hz / C0
    sc = lam_inv * (float(beta) / du)
    up, vp, wp = (uvw_m[:, j][:, None] for j in range(3))
    tu = up * sc[None, :]
    tv = vp * sc[None, :]
    w = wp * lam_inv[None, :]
    neg = np.broadcast_to(wp < 0.0, tu.shape)
    psi = np.where(neg, -1, 1).astype(np.int8)
    tu = np.where(neg, -tu, tu)
    tv = np.where(neg, -tv, tv)
    w = np.where(neg, -w, w)
    qu = np.ceil(tu - 0.5)
    qv = np.ceil(tv - 0.5)
    sane = (np.abs(qu) < 2.0 ** 40) & (np.abs(qv) < 2.0 ** 40)
    qu = np.where(sane, qu, 0.0)
    qv = np.where(sane, qv, 0.0)
    xc, fu = _cell(qu, beta)
    yc, fv = _cell(qv, beta)
    x = n_grid // 2 + xc
    y = n_grid // 2 + yc
    if K == 1:
        k = np.zeros_like(x)
        inplane = sane
    else:
        if not table.w_max > 0.0:
            raise ValueError("w_max must be positive with more than one w-plane")
        b = plane_bounds(K, table.w_max)                     # b_1 .. b_K
        k = np.zeros(w.shape, dtype=np.int64)
        for m in range(1, K):
            k += (w >= b[m - 1])
        inplane = (w < b[K - 1]) & sane
    kc = np.where(inplane, k, 0)
    S = np.where(inplane, table.supports[kc], 0).astype(np.int64)
    h = (S - 1) // 2
    x0 = x - h
    y0 = y - h
    ingrid = inplane & (x0 >= 0) & (x0 + S - 1 <= n_grid - 1) & (y0 >= 0) & (y0 + S - 1 <= n_grid - 1)
    if flag is not None:
        f = np.asarray(flag).reshape(rows, C, -1)
        unflagged = (f == 0).any(axis=2)
    else:
        unflagged = np.ones((rows, C), dtype=bool)
    griddable = ingrid & unflagged
    lo = -((beta - 1) // 2)
    sub = (fv - lo) * beta + (fu - lo)
    z = np.where(griddable, table.offsets[kc] + sub * S * S, -1)
    zeta_idx = np.where(griddable, kc * beta * beta + sub, -1)
    chan = np.broadcast_to(np.arange(C, dtype=np.int32)[None, :], (rows, C))
    flat = lambda a: np.ascontiguousarray(np.asarray(a).reshape(-1))  # noqa: E731
    return Placement(rows, C, flat(x), flat(y), flat(fu), flat(fv), flat(k), flat(psi), flat(w),
                     flat(S), flat(x0), flat(y0), flat(z), flat(zeta_idx), flat(griddable), flat(chan))


def classify(pl: Placement):
    """Compression indicator c_i and gridding indicator g_i (eq. "ci", Sec. 4.3.2), as
    vectorised comparisons with the predecessor record (previous row, same channel).

    Reading of eq. "ci": the compared position is the whole footprint origin (x0, y0) and
    the kernel pointer z; the predecessor must itself be griddable."""
    rows, C = pl.rows, pl.C
    gd = pl.griddable.reshape(rows, C)
    x0, y0, z = (a.reshape(rows, C) for a in (pl.x0, pl.y0, pl.z))
    c = np.zeros((rows, C), dtype=bool)
    c[1:] = gd[1:] & gd[:-1] & (x0[1:] == x0[:-1]) & (y0[1:] == y0[:-1]) & (z[1:] == z[:-1])
    g = gd & ~c
    return g.reshape(-1), c.reshape(-1)
