"""Oversampled w-projection kernels, Algorithm "convgen" (thesis Sec. 4.2.3), FP64.
Test infrastructure only.

Per w-plane k (w_k = w_max (k/(K-1))^2, square-root spacing, Sec. 2.2.1 / 4.2.1):
  1. sample taper(l) taper(m) * gbar_w(l, m) on an N_k x N_k image patch spanning the
     field of view l, m in [-1/(2 du), 1/(2 du)), gbar_w = 1/g_w = exp(+j 2pi w (n-1))
     (Sec. 2.2.1, eqs. "localconv2" and "C_W");
  2. zero-pad to beta*N_k ("zero padding as interpolation", Sec. 4.2.1) and FFT, which
     samples C_w at du/beta (eq. "local:o");
  3. normalise all planes by one constant so that C_0(0,0) = 1 (Sec. 4.2.3);
  4. support: threshold mode takes the outermost sample with |C| > 1e-3 (Sec. 4.2.3);
     prescribed mode trims or zero-pads to a given support ("normal" mode, Sec. 4.2.1);
  5. trim and reorder: one S x S row-major sub-kernel per sub-cell offset, ordered by
     (dv, du) (output C-1, Sec. 4.2.2), plane offsets and supports (C-2);
  6. zeta = sum of the real parts of each sub-kernel (eq. "sum", output C-3).

Readings of passages the thesis leaves open: the patch sample at eta = -1 (which has no +1 partner) is zero
so that the w = 0 kernel is exactly real and symmetric; screen samples outside the unit
disk (l^2 + m^2 >= 1) are zero; n - 1 is evaluated as -r^2 / (1 + sqrt(1 - r^2)).
"""
import dataclasses
from typing import Callable, Optional, Sequence

import numpy as np

from .pswf import psi0, bandwidth


@dataclasses.dataclass
class Table:
    beta: int
    supports: np.ndarray      # [K] int32            (C-2, support)
    offsets: np.ndarray       # [K] int64            (C-2, first sample of plane k)
    data: np.ndarray          # [sum_k beta^2 S_k^2] complex128   (C-1)
    zeta: np.ndarray          # [K * beta^2] float64 (C-3)
    w_planes: np.ndarray      # [K] float64 wavelengths
    w_max: float
    threshold_supports: Optional[np.ndarray] = None

    @property
    def K(self):
        return int(self.supports.shape[0])

    @property
    def lo(self):
        """Smallest sub-cell offset index: offsets run over (-beta/2, beta/2]."""
        return -((self.beta - 1) // 2)

    def sub_kernel(self, k: int, fv: int, fu: int) -> np.ndarray:
        S = int(self.supports[k])
        b = self.beta
        idx = (fv - self.lo) * b + (fu - self.lo)
        o = int(self.offsets[k]) + idx * S * S
        return self.data[o:o + S * S].reshape(S, S)


def default_nk(s_max: int) -> int:
    """Image-plane patch size: max(64, next power of two >= 2 * S_max)."""
    n = 64
    while n < 2 * s_max:
        n *= 2
    return n


def w_plane_values(K: int, w_max: float) -> np.ndarray:
    if K == 1:
        return np.zeros(1)
    k = np.arange(K, dtype=np.float64)
    return w_max * (k / (K - 1)) ** 2


def exact_screen(w: float, l: np.ndarray, m: np.ndarray) -> np.ndarray:
    """gbar_w(l, m) = exp(+j 2 pi w (sqrt(1 - l^2 - m^2) - 1)), zero outside the unit disk."""
    r2 = l * l + m * m
    inside = r2 < 1.0
    nm1 = np.where(inside, -r2 / (1.0 + np.sqrt(np.where(inside, 1.0 - r2, 1.0))), 0.0)
    return np.where(inside, np.exp(2j * np.pi * w * nm1), 0.0)


def _patch(w, n_k, du, taper_1d, screen):
    """Step 1: the N_k x N_k image-plane patch taper(l) taper(m) gbar_w(l, m), and its taper row."""
    idx = np.arange(n_k)
    eta = 2.0 * (idx - n_k // 2) / n_k
    l = eta / (2.0 * du)
    t = taper_1d(l, eta)
    t = np.where(idx == 0, 0.0, t)                       # eta = -1 sample has no partner
    L, Mm = np.meshgrid(l, l, indexing="xy")             # [m][l]
    return (t[:, None] * t[None, :]) * screen(w, L, Mm)


def _oversampled_plane(w, n_k, beta, du, taper_1d, screen):
    """Step 2: the (beta*N_k)^2 oversampled C_w, centred (offset 0 at index M/2)."""
    M = beta * n_k
    padded = np.zeros((M, M), dtype=np.complex128)
    o = M // 2 - n_k // 2
    padded[o:o + n_k, o:o + n_k] = _patch(w, n_k, du, taper_1d, screen)
    return np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(padded)))


def _dc_norm(n_k, du, taper_1d, screen):
    """Step 3's constant: C_0(0,0), the DC value of the w = 0 patch's transform (its sum)."""
    return float(np.real(np.sum(_patch(0.0, n_k, du, taper_1d, screen))))


def threshold_support(C: np.ndarray, beta: int, threshold: float) -> int:
    M = C.shape[0]
    kv, ku = np.nonzero(np.abs(C) > threshold)
    if kv.size == 0:
        return 1
    R = int(max(np.max(np.abs(kv - M // 2)), np.max(np.abs(ku - M // 2))))
    return 2 * int(np.ceil(R / beta)) + 1


def _trim(C: np.ndarray, beta: int, S: int) -> np.ndarray:
    """Step 5: sub-kernel (fv, fu), sample [i][j] = C(beta (i - h) - fv, beta (j - h) - fu),
    h = (S-1)/2, rows <-> v, columns <-> u (eq. "choose"); out-of-range samples are 0."""
    M = C.shape[0]
    lo = -((beta - 1) // 2)
    f = np.arange(beta) + lo
    i = np.arange(S)
    off = beta * (i - (S - 1) // 2)
    ov = off[None, :] - f[:, None]               # [beta(f), S(i)]
    iv = ov + M // 2
    ok = (iv >= 0) & (iv < M)
    ivc = np.clip(iv, 0, M - 1)
    # out[fv][fu][i][j] = C[iv[fv][i]][iu[fu][j]]
    out = C[ivc[:, None, :, None], ivc[None, :, None, :]]
    mask = ok[:, None, :, None] & ok[None, :, None, :]
    return np.where(mask, out, 0.0)


def build_table(du: float, n_wplanes: int, w_max: float, beta: int, taper_support: int = 7,
                supports: Optional[Sequence[int]] = None, n_k: Optional[int] = None,
                threshold: float = 1e-3, taper: Optional[Callable] = None,
                screen: Optional[Callable] = None, planes: Optional[Sequence[int]] = None) -> Table:
    """Algorithm "convgen".  `taper(l, eta)` and `screen(w, l, m)` may be replaced (the
    pins substitute a Gaussian taper and the paraxial screen to reach a closed form).

    `planes` (prescribed supports only) builds the kernels of those planes alone: every plane
    is computed independently of the others (the normalisation constant comes from the w = 0
    patch), so the built planes are identical to a full build; the others keep their layout
    (supports, offsets) with zero samples, zero zeta and threshold support 0.  It bounds the
    host time and memory of large tables (64 planes of 4096^2 transforms) when a test's
    records touch only some planes."""
    K = n_wplanes
    c = bandwidth(taper_support)
    if taper is None:
        taper = lambda l, eta: psi0(c, eta)  # noqa: E731
    if screen is None:
        screen = exact_screen
    if planes is not None and supports is None:
        raise ValueError("a plane subset needs prescribed supports")
    todo = set(range(K)) if planes is None else {int(k) for k in planes}
    if any(k < 0 or k >= K for k in todo):
        raise ValueError("plane index out of range")
    w_planes = w_plane_values(K, w_max)
    if n_k is None:
        n_k = default_nk(max(supports) if supports is not None else 4 * taper_support)
    norm = _dc_norm(n_k, du, taper, screen)
    built, thr = {}, np.zeros(K, dtype=np.int32)
    for k in sorted(todo):
        C = _oversampled_plane(w_planes[k], n_k, beta, du, taper, screen) / norm
        thr[k] = threshold_support(C, beta, threshold)
        built[k] = C if supports is None else _trim(C, beta, int(supports[k]))
    sup = np.asarray(supports, dtype=np.int32) if supports is not None else thr.copy()
    if np.any(sup % 2 == 0) or np.any(sup < 1):
        raise ValueError("supports must be odd and positive")
    data, offsets, zeta = [], [], []
    off = 0
    for k in range(K):
        S = int(sup[k])
        if k in built:
            sub = built[k] if supports is not None else _trim(built[k], beta, S)   # [beta, beta, S, S]
        else:
            sub = np.zeros((beta, beta, S, S), dtype=np.complex128)
        offsets.append(off)
        data.append(sub.reshape(-1))
        zeta.append(sub.real.sum(axis=(2, 3)).reshape(-1))
        off += beta * beta * S * S
    return Table(beta, sup, np.asarray(offsets, np.int64), np.concatenate(data),
                 np.concatenate(zeta), w_planes, float(w_max), thr)


def delta_table() -> Table:
    """The delta kernel: one plane, beta = 1, support 1, sample value 1."""
    return Table(1, np.array([1], np.int32), np.array([0], np.int64),
                 np.array([1.0 + 0j]), np.array([1.0]), np.zeros(1), 0.0, None)
