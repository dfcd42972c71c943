"""IMEX SDC and two-level MLSDC (oracle; test infrastructure only).

Sec. 4.2, Eq. update_equation_sdcq_discrete_form: one sweep updates nodes
m = 0..M-1 in order,
  Theta^{m+1,(k+1)} = Theta^n
      + dt sum_{j<=m}   q~E_{m+1,j} [F_E(Theta^{j,(k+1)}) - F_E(Theta^{j,(k)})]
      + dt sum_{j<=m+1} q~I_{m+1,j} [F_I(Theta^{j,(k+1)}) - F_I(Theta^{j,(k)})]
      + dt sum_{j=0..M} q_{m+1,j} F(Theta^{j,(k)})   [+ tau^{m+1} on a coarse level,
                                                       Eq. modified_update_equation_sdcq_discrete_form]
The j = m+1 implicit term holds the unknown, so the node value solves
Eq. implicit_systems: Theta - dt q~I_{m+1,m+1} F_I(Theta) = b.  Readings: the
sums include j = 0 (node 0 never changes, so its differences vanish);
F_I and F_E at the new node are re-evaluated after the solve.

Sec. 4.3, Algorithm 1 (two space-time levels): A) fine sweep; B) restrict the
fine nodes to the coarse level (time injection Pi^c_f then spectral truncation
D^c_f) and evaluate F there, saving copies; C) FAS correction
tau_c = A_c(R Theta_f) - R A_f(Theta_f) (Eq. tau_term_level_l+1, tau_f = 0),
A(Theta) = Theta - dt (Q x I) F(Theta) (Eq. collocation_problem), then coarse
sweep(s); D) add the interpolated (zero-pad then Pi^f_c) coarse corrections of
Theta, F_I and F_E to the fine nodes 1..M_f, with no re-evaluation.
Initialisation (Sec. 4.3.2): Theta^n copied to every fine node.
Readings: tau uses the fine F produced by step A; the coarse node 0 value is
the restriction of Theta^n, evaluated once per step; the step's result is the
last fine node after step D of the last iteration; the number of coarse sweeps
per SweepCoarse call is a parameter (the paper uses one).
"""
from __future__ import annotations

import numpy as np

from . import quadrature


class Level:
    """A problem (F_E, F_I, implicit solve) on a set of Gauss-Lobatto nodes."""

    def __init__(self, problem, n_nodes: int):
        self.prob = problem
        self.t = quadrature.lobatto_nodes(n_nodes)
        self.M = n_nodes - 1
        self.Q = quadrature.collocation_matrix(self.t)
        self.QE = quadrature.explicit_euler_matrix(self.t)
        self.QI = quadrature.lu_implicit_matrix(self.Q)


def sweep(lev: Level, dt: float, Theta, FI, FE, tau=None):
    """One IMEX SDC sweep (Eq. update_equation_sdcq_discrete_form / Eq.
    modified_update_equation_sdcq_discrete_form when tau is given).
    Theta, FI, FE: lists of M+1 node arrays at sweep k; returns sweep k+1."""
    M, Q, QE, QI, prob = lev.M, lev.Q, lev.QE, lev.QI, lev.prob
    Tn = list(Theta)
    FIn = list(FI)
    FEn = list(FE)
    for m in range(M):
        b = Theta[0].copy()
        for j in range(m + 1):
            b = b + dt * QE[m + 1, j] * (FEn[j] - FE[j])
        for j in range(m + 1):
            b = b + dt * QI[m + 1, j] * (FIn[j] - FI[j])
        b = b - dt * QI[m + 1, m + 1] * FI[m + 1]
        for j in range(M + 1):
            b = b + dt * Q[m + 1, j] * (FI[j] + FE[j])
        if tau is not None:
            b = b + tau[m + 1]
        Tn[m + 1] = prob.implicit_solve(b, dt * QI[m + 1, m + 1])
        FIn[m + 1] = prob.implicit_rhs(Tn[m + 1])
        FEn[m + 1] = prob.explicit_rhs(Tn[m + 1])
    return Tn, FIn, FEn


def spread(lev: Level, u0):
    """k = 0 initialisation: Theta^n at every node, F evaluated once."""
    fi = lev.prob.implicit_rhs(u0)
    fe = lev.prob.explicit_rhs(u0)
    n = lev.M + 1
    return [u0.copy() for _ in range(n)], [fi] * n, [fe] * n


def sdc_step(lev: Level, u0, dt: float, n_sweeps: int, tape=None):
    """SDC(M+1, N_S): spread then N_S sweeps; returns the last node.
    With a `tape` dict, the node values of every sweep are recorded (the
    points where F_E was evaluated, for the adjoint)."""
    Theta, FI, FE = spread(lev, u0)
    if tape is not None:
        tape["sweeps"] = []
    for _ in range(n_sweeps):
        Theta, FI, FE = sweep(lev, dt, Theta, FI, FE)
        if tape is not None:
            tape["sweeps"].append(Theta)
    return Theta[-1]


def collocation_operator(lev: Level, dt: float, Theta, FI, FE):
    """A(Theta) = Theta - dt (Q x I) F(Theta) at every node (Eq. collocation_problem)."""
    n = lev.M + 1
    return [Theta[m] - dt * sum(lev.Q[m, j] * (FI[j] + FE[j]) for j in range(n)) for m in range(n)]


def mlsdc_step(fine: Level, coarse: Level, u0, dt: float, n_iter: int, n_coarse_sweeps: int = 1,
               return_nodes: bool = False, tape=None):
    """One time step of two-level MLSDC (Algorithm 1, repeated n_iter times).
    With a `tape` dict, the node values at which F_E was evaluated are
    recorded per iteration (fine sweep, restriction, coarse sweeps)."""
    pf, pc = fine.prob, coarse.prob
    Pi_cf = quadrature.lagrange_matrix(fine.t, coarse.t)   # fine -> coarse (time)
    Pi_fc = quadrature.lagrange_matrix(coarse.t, fine.t)   # coarse -> fine (time)
    Mf, Mc = fine.M, coarse.M

    def restrict_node(vals, i):
        return pf.restrict(sum(Pi_cf[i, j] * vals[j] for j in range(Mf + 1)), pc)

    def interpolate_node(dvals, m):
        return pf.interpolate(sum(Pi_fc[m, i] * dvals[i] for i in range(Mc + 1)), pc)

    Th_f, FI_f, FE_f = spread(fine, u0)
    u0c = restrict_node(Th_f, 0)
    Th_c = [u0c] * (Mc + 1)
    FI_c = [pc.implicit_rhs(u0c)] * (Mc + 1)
    FE_c = [pc.explicit_rhs(u0c)] * (Mc + 1)
    if tape is not None:
        tape.update(u0c=u0c, iters=[])
    for _ in range(n_iter):
        # A) fine sweep
        Th_f, FI_f, FE_f = sweep(fine, dt, Th_f, FI_f, FE_f)
        # B) restrict, re-evaluate, save the restriction
        Th_c, FI_c, FE_c = list(Th_c), list(FI_c), list(FE_c)
        for m in range(1, Mc + 1):
            Th_c[m] = restrict_node(Th_f, m)
            FI_c[m] = pc.implicit_rhs(Th_c[m])
            FE_c[m] = pc.explicit_rhs(Th_c[m])
        Th_s, FI_s, FE_s = list(Th_c), list(FI_c), list(FE_c)
        # C) FAS correction and coarse sweep(s)
        A_c = collocation_operator(coarse, dt, Th_c, FI_c, FE_c)
        A_f = collocation_operator(fine, dt, Th_f, FI_f, FE_f)
        tau = [A_c[i] - restrict_node(A_f, i) for i in range(Mc + 1)]
        coarse_nodes = []
        for _s in range(n_coarse_sweeps):
            Th_c, FI_c, FE_c = sweep(coarse, dt, Th_c, FI_c, FE_c, tau)
            coarse_nodes.append(Th_c)
        if tape is not None:
            tape["iters"].append({"fine": Th_f, "restricted": Th_s, "coarse": coarse_nodes})
        # D) return to the fine level (no function evaluations)
        dT = [Th_c[i] - Th_s[i] for i in range(Mc + 1)]
        dI = [FI_c[i] - FI_s[i] for i in range(Mc + 1)]
        dE = [FE_c[i] - FE_s[i] for i in range(Mc + 1)]
        Th_f, FI_f, FE_f = list(Th_f), list(FI_f), list(FE_f)
        for m in range(1, Mf + 1):
            Th_f[m] = Th_f[m] + interpolate_node(dT, m)
            FI_f[m] = FI_f[m] + interpolate_node(dI, m)
            FE_f[m] = FE_f[m] + interpolate_node(dE, m)
    if return_nodes:
        return Th_f, FI_f, FE_f
    return Th_f[-1]


def mlsdc_step_levels(levels: list, u0, dt: float, n_iter: int, n_coarse_sweeps: int = 1,
                      return_nodes: bool = False):
    """One time step of MLSDC on L >= 2 space-time levels (levels[0] finest).

    The paper treats two levels (Algorithm 1) and leaves more for future work;
    it calls the iteration a V-cycle from the fine level to the coarse level and
    back, and writes the FAS term for a general pair of levels (Eq.
    tau_term_level_l+1: tau_{l+1} = A_{l+1}(R Theta_l) - R A_l(Theta_l) + R tau_l).
    Reading for L levels:
      A) one sweep on level 0;
      down, for l = 0..L-2: restrict level l's nodes 1..M_{l+1} to level l+1,
         evaluate F there and save copies (step B), form tau_{l+1} with the
         restricted tau_l, and do n_coarse_sweeps sweeps on level l+1 (step C);
      up, for l = L-2..0: add the interpolated corrections of level l+1 (its
         values minus the saved copies) to level l's nodes 1..M_l (step D),
         then, on an intermediate level (l > 0), one sweep with tau_l.
    Initialisation as in Algorithm 1: Theta^n on every fine node; node 0 of
    each coarser level is the restriction of the level above's node 0,
    evaluated once.  With two levels this is mlsdc_step."""
    L = len(levels)
    probs = [lv.prob for lv in levels]
    down = [quadrature.lagrange_matrix(levels[l].t, levels[l + 1].t) for l in range(L - 1)]
    up = [quadrature.lagrange_matrix(levels[l + 1].t, levels[l].t) for l in range(L - 1)]

    def restrict(l, vals, i):
        return probs[l].restrict(sum(down[l][i, j] * vals[j] for j in range(levels[l].M + 1)), probs[l + 1])

    def interpolate(l, dvals, m):
        return probs[l].interpolate(sum(up[l][m, i] * dvals[i] for i in range(levels[l + 1].M + 1)), probs[l + 1])

    Th, FI, FE = [None] * L, [None] * L, [None] * L
    Th[0], FI[0], FE[0] = spread(levels[0], u0)
    for l in range(1, L):
        u0l = restrict(l - 1, Th[l - 1], 0)
        n = levels[l].M + 1
        Th[l] = [u0l] * n
        FI[l] = [probs[l].implicit_rhs(u0l)] * n
        FE[l] = [probs[l].explicit_rhs(u0l)] * n
    tau = [None] * L
    saved = [None] * L
    for _ in range(n_iter):
        Th[0], FI[0], FE[0] = sweep(levels[0], dt, Th[0], FI[0], FE[0])
        for l in range(L - 1):
            c = l + 1
            Th[c], FI[c], FE[c] = list(Th[c]), list(FI[c]), list(FE[c])
            for m in range(1, levels[c].M + 1):
                Th[c][m] = restrict(l, Th[l], m)
                FI[c][m] = probs[c].implicit_rhs(Th[c][m])
                FE[c][m] = probs[c].explicit_rhs(Th[c][m])
            saved[c] = (list(Th[c]), list(FI[c]), list(FE[c]))
            A_c = collocation_operator(levels[c], dt, Th[c], FI[c], FE[c])
            A_f = collocation_operator(levels[l], dt, Th[l], FI[l], FE[l])
            tau[c] = [A_c[i] - restrict(l, A_f, i) for i in range(levels[c].M + 1)]
            if tau[l] is not None:
                tau[c] = [tau[c][i] + restrict(l, tau[l], i) for i in range(levels[c].M + 1)]
            for _s in range(n_coarse_sweeps):
                Th[c], FI[c], FE[c] = sweep(levels[c], dt, Th[c], FI[c], FE[c], tau[c])
        for l in range(L - 2, -1, -1):
            c = l + 1
            Ts, Is, Es = saved[c]
            dT = [Th[c][i] - Ts[i] for i in range(levels[c].M + 1)]
            dI = [FI[c][i] - Is[i] for i in range(levels[c].M + 1)]
            dE = [FE[c][i] - Es[i] for i in range(levels[c].M + 1)]
            Th[l], FI[l], FE[l] = list(Th[l]), list(FI[l]), list(FE[l])
            for m in range(1, levels[l].M + 1):
                Th[l][m] = Th[l][m] + interpolate(l, dT, m)
                FI[l][m] = FI[l][m] + interpolate(l, dI, m)
                FE[l][m] = FE[l][m] + interpolate(l, dE, m)
            if l > 0:
                Th[l], FI[l], FE[l] = sweep(levels[l], dt, Th[l], FI[l], FE[l], tau[l])
    if return_nodes:
        return Th[0], FI[0], FE[0]
    return Th[0][-1]
