"""Pins for the oracle's table build, Algorithm "convgen" (Sec. 4.2.3), outputs C-1..C-3.

* closed form: with a Gaussian taper and a paraxial, anisotropic, shifted screen the
  kernel is an analytic complex Gaussian; every sample of every sub-kernel must match it
  (this fixes FFT sign, centring, zero padding, oversampling, normalisation, sub-kernel
  order and the u/v and +/- orientation of the trim);
* brute force: with the exact w-screen and the PSWF taper, direct 2-D DFT sums at each
  sample offset on a small patch;
* w = 0 reduces to the PSWF (eigen-identity), C_0(0,0) = 1, symmetries, -w -> conj,
  zeta nearly independent of the sub-cell offset (Poisson summation).
"""
import numpy as np
import pytest

import oracle
from oracle.pswf import bandwidth
from oracle.table import default_nk, exact_screen


def _offsets(beta, S, fv, fu):
    i = np.arange(S)
    base = beta * (i - (S - 1) // 2)
    return base - fv, base - fu        # oversampled units, rows <-> v, cols <-> u


def test_closed_form_paraxial_gaussian():
    du, beta, K, w_max, S, n_k = 1.0, 4, 3, 12.0, 15, 64
    a = 112.0 * du * du                       # taper exp(-a l^2) ~ e^-28 at the patch edge
    su, sv = 0.3 * du, -0.45 * du             # uv shift breaks +/- symmetry

    def taper(l, eta):
        return np.exp(-a * l * l)

    def screen(w, L, M):                      # paraxial, anisotropic: exp(-j pi w (l^2 + 2 m^2))
        return np.exp(-1j * np.pi * w * (L * L + 2.0 * M * M)) * np.exp(2j * np.pi * (su * L + sv * M))

    tab = oracle.build_table(du, K, w_max, beta, supports=[S] * K, n_k=n_k, taper=taper, screen=screen)
    norm = (np.pi / a) * np.exp(-np.pi ** 2 * (su * su + sv * sv) / a)
    worst = 0.0
    for k in range(K):
        w = tab.w_planes[k]
        a1, a2 = a + 1j * np.pi * w, a + 2j * np.pi * w
        for fv in range(tab.lo, tab.lo + beta):
            for fu in range(tab.lo, tab.lo + beta):
                ov, ou = _offsets(beta, S, fv, fu)
                u = ou * du / beta
                v = ov * du / beta
                ref = (np.sqrt(np.pi / a2) * np.exp(-np.pi ** 2 * (v - sv) ** 2 / a2))[:, None] * \
                      (np.sqrt(np.pi / a1) * np.exp(-np.pi ** 2 * (u - su) ** 2 / a1))[None, :] / norm
                worst = max(worst, np.max(np.abs(tab.sub_kernel(k, fv, fu) - ref)))
    assert worst < 1e-10, worst


@pytest.mark.parametrize("w", [0.0, 3.0, 9.0])
def test_brute_force_dft_exact_screen(w):
    du, beta, n_k, S0, S = 0.05, 2, 16, 5, 9      # field of view 20 rad^-1... l up to 10: clipped by unit disk
    du = 0.8                                       # l in [-0.625, 0.625): inside the unit disk
    tab = oracle.build_table(du, 2, w, beta, S0, supports=[S, S], n_k=n_k)
    c = bandwidth(S0)
    idx = np.arange(n_k)
    eta = 2.0 * (idx - n_k // 2) / n_k
    l = eta / (2 * du)
    t = np.where(idx == 0, 0.0, oracle.psi0(c, eta))
    L, M = np.meshgrid(l, l, indexing="xy")
    f = t[:, None] * t[None, :]
    norm = f.sum()
    k = 1
    scr = exact_screen(tab.w_planes[k], L, M)
    for fv in (tab.lo, 0, tab.lo + beta - 1):
        for fu in (tab.lo, tab.lo + beta - 1):
            ov, ou = _offsets(beta, S, fv, fu)
            got = tab.sub_kernel(k, fv, fu)
            for i in range(S):
                for j in range(S):
                    u, v = ou[j] * du / beta, ov[i] * du / beta
                    ref = np.sum(f * scr * np.exp(-2j * np.pi * (u * L + v * M))) / norm
                    assert abs(got[i, j] - ref) < 1e-12


def test_brute_force_samples_at_full_size():
    # The w-projection workload's own table: 32 planes up to its w_max, supports 9..65,
    # beta = 8, 256^2 image patch zero-padded to 2048^2.  Sampled values of the outermost and
    # a middle plane against direct 2-D Fourier sums over the patch (65536 terms each), which
    # share none of the oracle's FFT, padding, shift, normalisation or trim steps.
    import synth
    wl = synth.make("wproj_2k", n_chan=1, n_times=2, n_baselines=4)   # the full workload's du and w_max
    n_k = default_nk(max(wl.supports))                 # the patch the workload's table is built on
    tab = oracle.build_table(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support, supports=wl.supports)
    beta, du = tab.beta, wl.du
    assert (n_k, beta, wl.n_wplanes) == (256, 8, 32)
    c = bandwidth(wl.taper_support)
    idx = np.arange(n_k)
    eta = 2.0 * (idx - n_k // 2) / n_k
    l = eta / (2 * du)
    t = np.where(idx == 0, 0.0, oracle.psi0(c, eta))
    L, M = np.meshgrid(l, l, indexing="xy")
    f = t[:, None] * t[None, :]
    norm = f.sum()
    checked = 0
    for k in (16, 31):
        S = int(tab.supports[k])
        h = (S - 1) // 2
        scr = f * exact_screen(tab.w_planes[k], L, M)
        for fv, fu in ((tab.lo, tab.lo + beta - 1), (0, 0), (2, -1)):
            ov, ou = _offsets(beta, S, fv, fu)
            got = tab.sub_kernel(k, fv, fu)
            for i, j in ((h, h), (h, 0), (0, h), (h // 2, h + 3), (S - 1, S - 2)):
                u, v = ou[j] * du / beta, ov[i] * du / beta
                ref = np.sum(scr * np.exp(-2j * np.pi * (u * L + v * M))) / norm
                assert abs(got[i, j] - ref) < 1e-12, (k, fv, fu, i, j, got[i, j], ref)
                checked += 1
    assert checked == 30
    assert abs(tab.sub_kernel(31, 0, 0)[32, 32]) > 1e-3          # a w-kernel, not a trivial one


def test_w0_kernel_is_pswf():
    du, beta, S0 = 2.0, 8, 7
    tab = oracle.build_table(du, 1, 0.0, beta, S0, supports=[9], n_k=64)
    c = bandwidth(S0)
    assert abs(tab.sub_kernel(0, 0, 0)[4, 4] - 1.0) < 1e-14        # C_0(0,0) = 1
    assert np.max(np.abs(tab.data.imag)) < 1e-14                  # real at w = 0
    for fv in range(tab.lo, tab.lo + beta):
        for fu in range(tab.lo, tab.lo + beta):
            ov, ou = _offsets(beta, 9, fv, fu)
            ev, eu = 2 * ov / beta / S0, 2 * ou / beta / S0
            mv, mu = np.abs(ev) < 1, np.abs(eu) < 1
            ref = np.outer(np.where(mv, oracle.psi0(c, np.clip(ev, -.99, .99)), 0),
                           np.where(mu, oracle.psi0(c, np.clip(eu, -.99, .99)), 0))
            m = np.outer(mv, mu)
            assert np.max(np.abs(tab.sub_kernel(0, fv, fu) - ref)[m]) < 1e-4


def _value_at(tab, k, ov, ou):
    """C_k at oversampled offsets (ov, ou) via the table layout."""
    b, S = tab.beta, int(tab.supports[k])
    h = (S - 1) // 2
    fv = (-ov) % b
    fv = fv if fv <= b // 2 else fv - b
    if fv < tab.lo:
        fv += b
    fu = (-ou) % b
    fu = fu if fu <= b // 2 else fu - b
    if fu < tab.lo:
        fu += b
    i = (ov + fv) // b + h
    j = (ou + fu) // b + h
    if not (0 <= i < S and 0 <= j < S):
        return None
    return tab.sub_kernel(k, fv, fu)[i, j]


def test_symmetries_and_negative_w():
    du, beta = 1.5, 4
    tp = oracle.build_table(du, 3, 40.0, beta, 7, supports=[11, 11, 11], n_k=64)
    tn = oracle.build_table(du, 3, -40.0, beta, 7, supports=[11, 11, 11], n_k=64)
    assert np.max(np.abs(tn.data - np.conj(tp.data))) < 1e-13
    rng = np.random.default_rng(3)
    for _ in range(300):
        k = int(rng.integers(0, 3))
        ov, ou = (int(x) for x in rng.integers(-18, 19, 2))
        a = _value_at(tp, k, ov, ou)
        for b in (_value_at(tp, k, ou, ov), _value_at(tp, k, -ov, -ou)):
            if a is not None and b is not None:
                assert abs(a - b) < 1e-13


def test_zeta_poisson_invariance_and_sum():
    tab = oracle.build_table(2.0, 1, 0.0, 8, 7, supports=[11], n_k=64)
    z = tab.zeta
    assert (z.max() - z.min()) / z.mean() < 2e-4
    for k in range(tab.K):
        for fv in range(tab.lo, tab.lo + 8):
            for fu in range(tab.lo, tab.lo + 8):
                idx = (fv - tab.lo) * 8 + (fu - tab.lo)
                assert abs(z[idx] - tab.sub_kernel(k, fv, fu).real.sum()) < 1e-12


def test_threshold_support_grows_with_w():
    du = 2.0
    tab = oracle.build_table(du, 6, 400.0, 4, 7, n_k=128)
    s = tab.supports
    assert s[0] == tab.threshold_supports[0]
    assert np.all(s % 2 == 1) and np.all(np.diff(s) >= 0) and s[-1] > s[0]
    # every sample outside the support is below the threshold for the centre sub-kernel
    assert np.all(np.abs(tab.sub_kernel(0, 0, 0)[[0, -1], :]) < 5e-2)
