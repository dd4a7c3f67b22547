"""Pins for the oracle's prolate spheroidal taper (Sec. 2.3.3).

psi_0 is pinned by its defining property rather than by re-calling scipy: the finite
Fourier transform over [-1, 1] maps psi_0(c, .) to a multiple of itself (the eigen-identity
that makes the PSWF the optimal concentrated taper).  A wrong bandwidth convention, a
wrong order or a wrong normalisation breaks the constancy of the ratio below.
"""
import numpy as np
import pytest

import oracle
from oracle.pswf import bandwidth


@pytest.mark.parametrize("S0", [5, 7, 9])
def test_eigen_identity(S0):
    c = bandwidth(S0)
    t, wts = np.polynomial.legendre.leggauss(400)
    f = oracle.psi0(c, t)
    x = np.linspace(-0.95, 0.95, 39)
    ft = (np.exp(1j * c * x[:, None] * t[None, :]) * f[None, :] * wts[None, :]).sum(1)
    ratio = ft / oracle.psi0(c, x)
    assert np.max(np.abs(ft.imag)) < 1e-12
    lam = ratio.real.mean()
    assert np.max(np.abs(ratio.real - lam)) < 1e-9 * abs(lam)


def test_normalised_even_and_decaying():
    c = bandwidth(7)
    x = np.linspace(0, 0.99, 50)
    v = oracle.psi0(c, x)
    assert abs(oracle.psi0(c, 0.0) - 1.0) < 1e-14
    assert np.allclose(v, oracle.psi0(c, -x), rtol=0, atol=1e-15)
    assert np.all(np.diff(v) < 0)


def test_small_bandwidth_limit():
    # c -> 0: psi_0 tends to the Legendre polynomial P_0 = 1, with the first correction
    # of order c^2 (x^2 - 1/3) / 6 up to normalisation.
    c = 1e-3
    x = np.linspace(-0.9, 0.9, 7)
    assert np.max(np.abs(oracle.psi0(c, x) - 1.0)) < 1e-6
