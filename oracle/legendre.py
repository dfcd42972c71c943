"""Normalised associated Legendre functions (oracle; test infrastructure only).

Sec. 3, Eq. spectral_to_physical_space uses "normalized" associated Legendre
functions P^r_s.  Reading: orthonormal on [-1, 1] (integral of (P^m_n)^2 dmu
equals 1), no Condon-Shortley phase, P^{-m} = P^m.  With this choice Eq.
legendre_transform (Gaussian weights, 1/I in Eq. fourier_transform) is the
exact inverse of Eq. spectral_to_physical_space.

  P^m_m = sqrt((2m+1)/2 * prod_{k=1..m} (2k-1)/(2k)) (1 - mu^2)^{m/2}
  mu P^m_n = eps^m_{n+1} P^m_{n+1} + eps^m_n P^m_{n-1},
  eps^m_n = sqrt((n^2 - m^2) / (4 n^2 - 1))
  H^m_n = (1 - mu^2) dP^m_n/dmu = -n eps^m_{n+1} P^m_{n+1} + (n+1) eps^m_n P^m_{n-1}

Values below 1e-300 in magnitude are flushed to zero (near the poles at high
order they underflow anyway; their contributions are below any tolerance).
"""
from __future__ import annotations

import numpy as np

FLUSH = 1e-300


def eps(m: int, n: int) -> float:
    """eps^m_n = sqrt((n^2 - m^2) / (4 n^2 - 1)); zero for n <= m."""
    if n <= m:
        return 0.0
    return float(np.sqrt((n * n - m * m) / (4.0 * n * n - 1.0)))


def assoc_legendre(Rmax: int, mu: np.ndarray) -> np.ndarray:
    """P[m, n, j] = P^m_n(mu_j) for 0 <= m <= n <= Rmax (zero for n < m)."""
    mu = np.asarray(mu, dtype=np.float64)
    s = np.sqrt(1.0 - mu * mu)
    P = np.zeros((Rmax + 1, Rmax + 1, mu.size))
    prod = 1.0
    for m in range(Rmax + 1):
        if m > 0:
            prod *= (2.0 * m - 1.0) / (2.0 * m)
        with np.errstate(under="ignore"):
            pmm = np.sqrt((2.0 * m + 1.0) / 2.0 * prod) * s ** m
        pmm = np.where(np.abs(pmm) < FLUSH, 0.0, pmm)
        P[m, m] = pmm
        p_nm1 = np.zeros_like(mu)  # P^m_{m-1} = 0
        p_n = pmm
        for n in range(m, Rmax):
            e_np1, e_n = eps(m, n + 1), eps(m, n)
            with np.errstate(under="ignore"):
                p_np1 = (mu * p_n - e_n * p_nm1) / e_np1
            p_np1 = np.where(np.abs(p_np1) < FLUSH, 0.0, p_np1)
            P[m, n + 1] = p_np1
            p_nm1, p_n = p_n, p_np1
    return P


def legendre_H(R: int, P: np.ndarray) -> np.ndarray:
    """H[m, n, j] = (1 - mu_j^2) dP^m_n/dmu (mu_j) for n <= R, from P tabulated
    up to degree R + 1 (P.shape[0] >= R + 2)."""
    if P.shape[0] < R + 2:
        raise ValueError("H needs P up to degree R + 1")
    H = np.zeros((R + 1, R + 1, P.shape[2]))
    for m in range(R + 1):
        for n in range(m, R + 1):
            e_np1, e_n = eps(m, n + 1), eps(m, n)
            p_nm1 = P[m, n - 1] if n - 1 >= m else 0.0
            H[m, n] = -n * e_np1 * P[m, n + 1] + (n + 1.0) * e_n * p_nm1
    return H
