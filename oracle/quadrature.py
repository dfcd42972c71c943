"""Quadrature rules and SDC matrices (oracle; test infrastructure only).

Sec. 3 (Gaussian latitudes for Eq. legendre_transform), Sec. 4.2 (Gauss-Lobatto
nodes, Eq. weights for q_{m+1,j}, forward-Euler weights q~E, LU-trick weights
q~I), Sec. 4.3.3 (Lagrange matrices Pi^c_f, Pi^f_c).
"""
from __future__ import annotations

import numpy as np


def _legendre_pj(J: int, x: np.ndarray):
    """P_J(x) and P_{J-1}(x) by the Bonnet three-term recurrence."""
    p_prev = np.ones_like(x)
    p = x.copy()
    if J == 0:
        return p_prev, np.zeros_like(x)
    for k in range(2, J + 1):
        p_prev, p = p, ((2 * k - 1) * x * p - (k - 1) * p_prev) / k
    return p, p_prev


def gauss_legendre(J: int) -> tuple[np.ndarray, np.ndarray]:
    """Gaussian latitudes mu_j = roots of P_J and weights w_j, ordered north
    (mu near +1) to south.  Sec. 3: mu_j are the roots of the degree-J
    Legendre polynomial, w_j the Gaussian weights; w_j = 2 / ((1 - mu^2) P_J'^2).
    Newton iteration from cos(pi (j + 3/4) / (J + 1/2))."""
    j = np.arange(J, dtype=np.float64)
    x = np.cos(np.pi * (j + 0.75) / (J + 0.5))
    for _ in range(100):
        p, pm = _legendre_pj(J, x)
        dp = J * (x * p - pm) / (x * x - 1.0)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    p, pm = _legendre_pj(J, x)
    dp = J * (x * p - pm) / (x * x - 1.0)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    return x, w


def lobatto_nodes(n: int) -> np.ndarray:
    """n Gauss-Lobatto nodes on [0, 1] (Sec. 4.2, Eq.
    time_discretization_sdc_nodes): both end points plus the roots of
    P'_{n-1}, mapped from [-1, 1]."""
    if n < 2:
        raise ValueError("need at least 2 Lobatto nodes")
    inner = np.polynomial.legendre.Legendre.basis(n - 1).deriv().roots() if n > 2 else np.zeros(0)
    inner = np.sort(np.real(inner))
    x = np.concatenate([[-1.0], inner, [1.0]])
    return (x + 1.0) / 2.0


def lagrange_basis(t: np.ndarray, j: int, s: np.ndarray) -> np.ndarray:
    """L^j(s) = prod_{k != j} (s - t_k) / (t_j - t_k)."""
    out = np.ones_like(np.asarray(s, dtype=np.float64))
    for k in range(len(t)):
        if k != j:
            out = out * (s - t[k]) / (t[j] - t[k])
    return out


def collocation_matrix(t: np.ndarray) -> np.ndarray:
    """Q with q_{m,j} = integral_0^{t_m} L^j(s) ds on the unit interval
    (Sec. 4.2, Eq. weights, divided by Delta t).  Each integral is exact: a
    Gauss-Legendre rule with len(t) points integrates the degree len(t)-1
    polynomial L^j exactly."""
    n = len(t)
    xq, wq = gauss_legendre(n)
    Q = np.zeros((n, n))
    for m in range(n):
        for j in range(n):
            s = t[m] * (xq + 1.0) / 2.0
            Q[m, j] = t[m] / 2.0 * np.sum(wq * lagrange_basis(t, j, s))
    return Q


def explicit_euler_matrix(t: np.ndarray) -> np.ndarray:
    """q~E: forward Euler over the sub-intervals (Sec. 4.2):
    q~E_{m+1,j} = (t_{j+1} - t_j) for j <= m, zero otherwise."""
    n = len(t)
    QE = np.zeros((n, n))
    for m in range(n - 1):
        for j in range(m + 1):
            QE[m + 1, j] = t[j + 1] - t[j]
    return QE


def lu_implicit_matrix(Q: np.ndarray) -> np.ndarray:
    """q~I from the LU decomposition of Q (Sec. 4.2, the approach of Weiser 2015).

    Reading: the first Lobatto row of Q is zero, so the factorisation is taken
    on the node block 1..M.  With (Q[1:,1:])^T = L U (Doolittle: L unit lower
    triangular, no pivoting), q~I[1:,1:] = U^T, which is lower triangular as a
    forward sweep needs; row and column 0 are zero."""
    A = Q[1:, 1:].T.copy()
    k = A.shape[0]
    L = np.eye(k)
    U = np.zeros((k, k))
    for i in range(k):
        for c in range(i, k):
            U[i, c] = A[i, c] - L[i, :i] @ U[:i, c]
        for r in range(i + 1, k):
            L[r, i] = (A[r, i] - L[r, :i] @ U[:i, i]) / U[i, i]
    QI = np.zeros_like(Q)
    QI[1:, 1:] = U.T
    return QI


def lagrange_matrix(t_from: np.ndarray, t_to: np.ndarray) -> np.ndarray:
    """Pi with Pi[i, j] = L^j_from(t_to[i]) (Sec. 4.3.3: Pi^c_f when t_from are
    the fine nodes and t_to the coarse nodes; Pi^f_c the other way round)."""
    return np.array([[lagrange_basis(t_from, j, ti) for j in range(len(t_from))] for ti in t_to])
