"""Prolate spheroidal taper (thesis Sec. 2.3.3 "The tapering function"; Sec. 4.2.1 names
a prolate spheroidal tapering operator).  Test infrastructure only.

The thesis's operator reproduces casacore's approximation, whose parameters it does not
state.  The reading used here: the zeroth-order angular prolate spheroidal function
psi_0(c, eta), |eta| < 1, normalised so psi_0(c, 0) = 1, with bandwidth c = pi * S0 / 2
where S0 is the width in grid cells of the w = 0 kernel.  By the finite-Fourier-transform
eigen-identity of psi_0, a kernel C(u) = psi_0(c, 2u / (S0 du)) of width S0 cells has as
its image-plane taper c(l) proportional to psi_0(c, 2 du l) over the field of view.
scipy.special.pro_ang1 is the library primitive used for psi_0.
"""
import numpy as np
import scipy.special as sp


def bandwidth(taper_support: int) -> float:
    return np.pi * taper_support / 2.0


def psi0(c: float, eta) -> np.ndarray:
    """psi_0(c, eta) for |eta| <= 1, normalised to 1 at eta = 0.

    pro_ang1 is undefined at |eta| = 1 exactly; there the value is taken 1e-13 inside
    (psi_0 is smooth, so the difference is ~1e-15 relative)."""
    eta = np.asarray(eta, dtype=np.float64)
    e = np.clip(eta, -1.0 + 1e-13, 1.0 - 1e-13)
    v0 = sp.pro_ang1(0, 0, c, 0.0)[0]
    return sp.pro_ang1(0, 0, c, e)[0] / v0
