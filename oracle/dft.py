"""Direct-Fourier dirty image including the w-term, FP64 (tiny inputs only).
Test infrastructure only.

I_D(l, m) = Re sum_i q_i exp(+j2pi(u_i l + v_i m + w_i (n - 1))) / sum_i eps_i (1 - f_i),
with q_i the weighted, flagged visibilities (eq. "weight") and (u, v, w) in wavelengths:
the inverse of the measurement equation (eq. "measurmentrewritten") that w-projection
gridding approximates (Sec. 2.2).  The weight sum is the direct-sum counterpart of N_p,
whose extra factor zeta is the kernel's own sum (eq. "normalizer").
"""
import numpy as np

C0 = 299_792_458.0


def dirty_image(uvw_m, freq_hz, vis, weight, flag, n_grid: int, du: float, pols=(0,),
                mask=None) -> np.ndarray:
    """mask: optional bool [rows, C] selecting the records to include (e.g. the griddable ones)."""
    uvw_m = np.asarray(uvw_m, np.float64)
    freq_hz = np.asarray(freq_hz, np.float64)
    rows, C = uvw_m.shape[0], freq_hz.shape[0]
    P = np.asarray(vis).shape[-1]
    v = np.asarray(vis, np.complex128).reshape(rows, C, P)
    wf = np.asarray(weight, np.float64).reshape(rows, C, P) * (1.0 - np.asarray(flag, np.float64).reshape(rows, C, P))
    k = np.arange(n_grid)
    l1 = (k - n_grid // 2) / (n_grid * du)
    L, M = np.meshgrid(l1, l1, indexing="xy")                 # [m][l]
    r2 = L * L + M * M
    nm1 = -r2 / (1.0 + np.sqrt(1.0 - r2))
    if mask is not None:
        wf = wf * np.asarray(mask, np.float64).reshape(rows, C, 1)
    out = np.zeros((C, len(pols), n_grid, n_grid))
    for c in range(C):
        lam_inv = freq_hz[c] / C0
        u, vv, w = (uvw_m[:, j] * lam_inv for j in range(3))
        for pi, p in enumerate(pols):
            acc = np.zeros((n_grid, n_grid), np.complex128)
            for i in range(rows):
                q = wf[i, c, p] * v[i, c, p]
                if q == 0:
                    continue
                acc += q * np.exp(2j * np.pi * (u[i] * L + vv[i] * M + w[i] * nm1))
            out[c, pi] = acc.real / wf[:, c, p].sum()
    return out
