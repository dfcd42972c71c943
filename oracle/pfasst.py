"""Two-level PFASST: MLSDC over P time slices at once (oracle; test
infrastructure only).

The paper (Sec. 1 and its conclusions) names the parallel full approximation
scheme in space and time, PFASST, as the time-parallel extension of its
two-level MLSDC; it does not print the algorithm.  This is the published
two-level PFASST iteration (Emmett and Minion) restated on top of this
oracle's Algorithm 1 steps A-D (sdc.mlsdc_step), with slice p covering
[t0 + p dt, t0 + (p+1) dt].  Readings (stated because the paper gives none):

Predictor.  Every slice's fine nodes start as u0 spread.  The coarse level is
run serially over the slices: slice 0 starts from R(u0), slice p from slice
p-1's coarse end value, each spread and swept n_predictor_sweeps times (no
tau; by default n_coarse_sweeps; with 0 every slice starts from u0).
For p >= 1 the fine nodes then become the spread of u0 plus the zero-padded
coarse correction of the slice's initial value, v_p = u0 + (D^c_f)^T
(Th_c[p][0] - R(u0)), with F_I and F_E evaluated there.  Slice 0's fine nodes
stay u0 (its coarse predictor values are overwritten by the first
restriction), so slice 0 is exactly MLSDC.

Iteration k (per slice, in slice order, which is the pipeline's data flow):
  A) for p >= 1 and k >= 2: fine node 0 = slice p-1's fine end value at the
     end of iteration k-1 ("sent" forward a whole iteration earlier), F
     re-evaluated there; then one fine sweep;
  B) restrict fine nodes 0..M_c (node 0 included: its restriction is what the
     slice's fine initial value says), evaluate F, save copies;
  C) tau_c = A_c(R Theta_f) - R A_f(Theta_f) (Eq. tau_term_level_l+1); for
     p >= 1, coarse node 0 = slice p-1's coarse end value of this iteration
     (the blocking "receive"), F re-evaluated there; n_c coarse sweeps with tau;
  D) add the interpolated corrections (coarse value minus saved copy, at
     nodes 0..M_c) to fine nodes 1..M_f, for Theta, F_I and F_E.
The result after n_iter iterations is each slice's last fine node.

With P = 1 every step reduces to sdc.mlsdc_step.  At a fixed point every
slice holds the fine collocation solution started from the previous slice's
end value: the serial sequence of P collocation steps.
"""
from __future__ import annotations

from . import quadrature
from .sdc import Level, collocation_operator, spread, sweep


def pfasst(fine: Level, coarse: Level, u0, dt: float, P: int, n_iter: int, n_coarse_sweeps: int = 1,
           return_slices: bool = False, n_predictor_sweeps: int | None = None):
    pf, pc = fine.prob, coarse.prob
    Pi_cf = quadrature.lagrange_matrix(fine.t, coarse.t)
    Pi_fc = quadrature.lagrange_matrix(coarse.t, fine.t)
    Mf, Mc = fine.M, coarse.M

    def restrict_node(vals, i):
        return pf.restrict(sum(Pi_cf[i, j] * vals[j] for j in range(Mf + 1)), pc)

    def interpolate_node(dvals, m):
        return pf.interpolate(sum(Pi_fc[m, i] * dvals[i] for i in range(Mc + 1)), pc)

    def with_node0(lev, Th, FI, FE, u):
        Th, FI, FE = list(Th), list(FI), list(FE)
        Th[0] = u
        FI[0] = lev.prob.implicit_rhs(u)
        FE[0] = lev.prob.explicit_rhs(u)
        return Th, FI, FE

    # predictor
    fine_nodes = [spread(fine, u0) for _ in range(P)]
    Ru0 = pf.restrict(u0, pc)
    coarse_nodes = []
    cu = Ru0
    for p in range(P):
        Th_c, FI_c, FE_c = spread(coarse, cu)
        for _ in range(n_coarse_sweeps if n_predictor_sweeps is None else n_predictor_sweeps):
            Th_c, FI_c, FE_c = sweep(coarse, dt, Th_c, FI_c, FE_c)
        coarse_nodes.append((Th_c, FI_c, FE_c))
        cu = Th_c[-1]
    for p in range(1, P):
        fine_nodes[p] = spread(fine, u0 + pf.interpolate(coarse_nodes[p][0][0] - Ru0, pc))

    end_prev = None
    for k in range(n_iter):
        end_now = []
        coarse_end = None
        for p in range(P):
            Th_f, FI_f, FE_f = fine_nodes[p]
            # A) new fine initial value (from the previous iteration), fine sweep
            if p >= 1 and k >= 1:
                Th_f, FI_f, FE_f = with_node0(fine, Th_f, FI_f, FE_f, end_prev[p - 1])
            Th_f, FI_f, FE_f = sweep(fine, dt, Th_f, FI_f, FE_f)
            # B) restrict nodes 0..M_c, evaluate, save
            Th_c = [restrict_node(Th_f, i) for i in range(Mc + 1)]
            FI_c = [pc.implicit_rhs(t) for t in Th_c]
            FE_c = [pc.explicit_rhs(t) for t in Th_c]
            Th_s, FI_s, FE_s = list(Th_c), list(FI_c), list(FE_c)
            # C) FAS correction, coarse initial value from slice p-1, coarse sweeps
            A_c = collocation_operator(coarse, dt, Th_c, FI_c, FE_c)
            A_f = collocation_operator(fine, dt, Th_f, FI_f, FE_f)
            tau = [A_c[i] - restrict_node(A_f, i) for i in range(Mc + 1)]
            if p >= 1:
                Th_c, FI_c, FE_c = with_node0(coarse, Th_c, FI_c, FE_c, coarse_end)
            for _ in range(n_coarse_sweeps):
                Th_c, FI_c, FE_c = sweep(coarse, dt, Th_c, FI_c, FE_c, tau)
            coarse_end = Th_c[-1]
            # D) interpolate the corrections to fine nodes 1..M_f
            dT = [Th_c[i] - Th_s[i] for i in range(Mc + 1)]
            dI = [FI_c[i] - FI_s[i] for i in range(Mc + 1)]
            dE = [FE_c[i] - FE_s[i] for i in range(Mc + 1)]
            Th_f, FI_f, FE_f = list(Th_f), list(FI_f), list(FE_f)
            for m in range(1, Mf + 1):
                Th_f[m] = Th_f[m] + interpolate_node(dT, m)
                FI_f[m] = FI_f[m] + interpolate_node(dI, m)
                FE_f[m] = FE_f[m] + interpolate_node(dE, m)
            fine_nodes[p] = (Th_f, FI_f, FE_f)
            end_now.append(Th_f[-1])
        end_prev = end_now
    ends = [fine_nodes[p][0][-1] for p in range(P)]
    return ends if return_slices else ends[-1]
