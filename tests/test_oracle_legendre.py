"""Pins of the oracle's normalised associated Legendre functions (Sec. 3):
closed forms, scipy's lpmv (a library special case), discrete orthonormality on
Gaussian latitudes, and H = (1 - mu^2) dP/dmu against finite differences."""
import math

import numpy as np
import pytest

from oracle import legendre, quadrature as q


def test_closed_forms():
    mu = np.linspace(-0.99, 0.99, 37)
    P = legendre.assoc_legendre(3, mu)
    s = np.sqrt(1 - mu * mu)
    assert np.max(np.abs(P[0, 0] - np.sqrt(0.5))) < 1e-15
    assert np.max(np.abs(P[0, 1] - np.sqrt(1.5) * mu)) < 1e-15
    assert np.max(np.abs(P[1, 1] - np.sqrt(3) / 2 * s)) < 1e-15
    assert np.max(np.abs(P[0, 2] - np.sqrt(5 / 8) * (3 * mu * mu - 1))) < 1e-14
    assert np.max(np.abs(P[2, 2] - np.sqrt(15) / 4 * s * s)) < 1e-15
    assert np.all(P[1, 0] == 0) and np.all(P[3, 2] == 0)


def test_against_scipy_lpmv():
    sp = pytest.importorskip("scipy.special")
    mu = np.linspace(-0.97, 0.97, 23)
    R = 20
    P = legendre.assoc_legendre(R, mu)
    for m in range(R + 1):
        for n in range(m, R + 1):
            norm = math.sqrt((2 * n + 1) / 2 * math.factorial(n - m) / math.factorial(n + m))
            ref = (-1) ** m * sp.lpmv(m, n, mu) * norm   # remove the Condon-Shortley phase
            assert np.max(np.abs(P[m, n] - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("R,J", [(21, 32), (42, 64), (85, 128)])
def test_discrete_orthonormality(R, J):
    mu, w = q.gauss_legendre(J)
    P = legendre.assoc_legendre(R + 1, mu)
    for m in range(0, R + 2, max(1, R // 7)):
        G = (P[m, m:] * w) @ P[m, m:].T
        assert np.max(np.abs(G - np.eye(G.shape[0]))) < 1e-13


def test_H_against_finite_differences():
    R = 12
    mu = np.linspace(-0.9, 0.9, 19)
    h = 1e-5
    Pp = legendre.assoc_legendre(R + 1, mu + h)
    Pm = legendre.assoc_legendre(R + 1, mu - h)
    Pp2 = legendre.assoc_legendre(R + 1, mu + 2 * h)
    Pm2 = legendre.assoc_legendre(R + 1, mu - 2 * h)
    H = legendre.legendre_H(R, legendre.assoc_legendre(R + 1, mu))
    for m in range(R + 1):
        for n in range(m, R + 1):
            d = (8 * (Pp[m, n] - Pm[m, n]) - (Pp2[m, n] - Pm2[m, n])) / (12 * h)
            assert np.max(np.abs(H[m, n] - (1 - mu * mu) * d)) < 1e-8


def test_parity_symmetry():
    mu = np.linspace(0.05, 0.95, 10)
    R = 15
    Pn = legendre.assoc_legendre(R + 1, mu)
    Ps = legendre.assoc_legendre(R + 1, -mu)
    Hn, Hs = legendre.legendre_H(R, Pn), legendre.legendre_H(R, Ps)
    for m in range(R + 1):
        for n in range(m, R + 1):
            sgn = (-1) ** (n - m)
            assert np.max(np.abs(Ps[m, n] - sgn * Pn[m, n])) < 1e-13
            assert np.max(np.abs(Hs[m, n] + sgn * Hn[m, n])) < 1e-12
