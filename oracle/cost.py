"""Cost model of Sec. 4.5 (oracle; test infrastructure only).

Eq. computational_cost_mlsdc, Eq. computational_cost_sdc, Eq. theoretical_speedup,
with the paper's assumptions C^s = C^fi = C^fe on a level and costs scaling
with the coefficient count K_l = 3 R_l (R_l + 1) / 2.
"""
from __future__ import annotations


def coarse_cost_ratio(alpha: float, Rf: int) -> float:
    """C_c / C_f = K_c / K_f = alpha^2 (R_f + 1/alpha) / (R_f + 1)."""
    return alpha * alpha * (Rf + 1.0 / alpha) / (Rf + 1.0)


def cost_mlsdc(Mf: int, Mc: int, N_ML: int, alpha: float, Rf: int, Cf: float = 1.0) -> float:
    Cc = coarse_cost_ratio(alpha, Rf) * Cf
    return N_ML * Mf * 3 * Cf + N_ML * Mc * 3 * Cc + N_ML * Mc * 2 * Cc


def cost_sdc(Mf: int, N_S: int, Cf: float = 1.0) -> float:
    return N_S * Mf * 3 * Cf


def theoretical_speedup(Mf: int, Mc: int, N_ML: int, alpha: float, Rf: int, N_S: int) -> float:
    """S^theo = C^SDC(M_f+1, N_S) / C^MLSDC(M_f+1, M_c+1, N_ML, alpha)."""
    return cost_sdc(Mf, N_S) / cost_mlsdc(Mf, Mc, N_ML, alpha, Rf)
