"""Tangent-linear and adjoint of the SDC / MLSDC time step (oracle; test
infrastructure only).

The adjoint objective (reverse mode of Sec. 2 - Sec. 4.3 with respect to the
initial state Theta^0) is the geopotential misfit after n steps,
  J = 1/2 ||Phi'(T) - Phi_t||^2 = 1/2 (1/I) sum_{iota,j} w_j (Phi - Phi_t)^2,
with ||.|| the Parseval norm of Sec. 3 (|xi^0_n|^2 + 2 |xi^m_n|^2, m >= 1).

Inner product.  Every state is a complex array of stored coefficients; it is
treated as the real vector of its (Re, Im) parts, so
  <x, y> = sum Re(conj(x) y).
The fields are real (Sec. 3), so Im xi^0_n is not a degree of freedom: every
output of the method has it zero and no output depends on it; gradients are
returned with it zero.  Grid fields use the plain sum over points, Fourier
coefficients [J, R+1] the same complex inner product.  The transpose T^t of
a real-linear map T is defined by <y, T x> = <T^t y, x>.

Only F_E is nonlinear.  Everything else in a step (the node update, F_I,
the implicit solve, the restriction, the FAS correction, the interpolation)
is linear with constant coefficients, so the adjoint walks the step
backwards applying each operation's transpose, with F_E replaced by the
transpose of its Jacobian at the point where it was evaluated (recorded by
the forward step's tape).

The tangent-linear step is the forward algorithm itself run on (x, dx)
pairs, with F_E(x, dx) = (F_E(x), F_E'(x) dx) (Tangent below), so it shares
every line of the forward step's schedule.
"""
from __future__ import annotations

import numpy as np

from . import quadrature
from .sht import Grid, norm2, spec_mn, truncate, zero_m0_imag, zero_pad
from .sdc import Level, mlsdc_step, sdc_step


def inner(x: np.ndarray, y: np.ndarray) -> float:
    """<x, y> = sum Re(conj(x) y) over all entries (real arrays: plain sum)."""
    return float(np.sum(np.real(np.conj(x) * y)))


# ---------------------------------------------------------------------------
# transposes of the transform building blocks (Sec. 3)


def fourier_synthesis_t(g: Grid, f: np.ndarray) -> np.ndarray:
    """Transpose of Grid.fourier_synthesis, f = Re F_0 + sum_{m>=1} 2 Re(F_m e^{i m lambda}):
    F_m = c_m sum_iota f e^{-i m lambda_iota}, c_0 = 1, c_m = 2."""
    F = (f @ g._e_fwd).astype(np.complex128)
    F[..., 1:] *= 2.0
    F[..., 0] = F[..., 0].real
    return F


def fourier_analysis_t(g: Grid, F: np.ndarray) -> np.ndarray:
    """Transpose of Grid.fourier_analysis, F_m = (1/I) sum_iota f e^{-i m lambda}:
    f_iota = (1/I) Re sum_{m=0..R} F_m e^{i m lambda_iota} (each m once)."""
    return np.real(F @ g._e_inv) / g.I


def legendre_synthesis_t(g: Grid, F: np.ndarray, table: np.ndarray) -> np.ndarray:
    """Transpose of F^m_j = sum_n spec^m_n T^m_n(mu_j) (real table): spec^m_n = sum_j T^m_n(mu_j) F^m_j."""
    return g.legendre_analysis(F, table, np.ones(g.J))


def legendre_analysis_t(g: Grid, spec: np.ndarray, table: np.ndarray, weight: np.ndarray) -> np.ndarray:
    """Transpose of spec^m_n = sum_j F^m_j T^m_n(mu_j) w_j: F^m_j = w_j sum_n T^m_n(mu_j) spec^m_n."""
    return g.legendre_synthesis(spec, table) * weight[:, None]


def times_im_t(g: Grid, x: np.ndarray) -> np.ndarray:
    """Transpose of x -> i m x (real-linear): y -> -i m y."""
    return -1j * g.m * x


def synthesis_t(g: Grid, f: np.ndarray) -> np.ndarray:
    return zero_m0_imag(g, legendre_synthesis_t(g, fourier_synthesis_t(g, f), g.P))


def analysis_t(g: Grid, s: np.ndarray) -> np.ndarray:
    s = zero_m0_imag(g, s)
    return fourier_analysis_t(g, legendre_analysis_t(g, s, g.P, g.w))


def vector_synthesis_t(g: Grid, Ub: np.ndarray, Vb: np.ndarray, a: float):
    """Transpose of (psi, chi) -> (U, V) (Grid.vector_synthesis)."""
    Um = fourier_synthesis_t(g, Ub)
    Vm = fourier_synthesis_t(g, Vb)
    # U_m = (synth(i m chi, P) - synth(psi, H)) / a ; V_m = (synth(i m psi, P) + synth(chi, H)) / a
    psi = (-legendre_synthesis_t(g, Um, g.H) + times_im_t(g, legendre_synthesis_t(g, Vm, g.P))) / a
    chi = (times_im_t(g, legendre_synthesis_t(g, Um, g.P)) + legendre_synthesis_t(g, Vm, g.H)) / a
    return zero_m0_imag(g, psi), zero_m0_imag(g, chi)


def vector_analysis_t(g: Grid, divb: np.ndarray, curlb: np.ndarray, a: float):
    """Transpose of (X, Y) -> (div, curl) (Grid.vector_analysis)."""
    wt = g.w / (1.0 - g.mu ** 2)
    divb = zero_m0_imag(g, divb) / a
    curlb = zero_m0_imag(g, curlb) / a
    # div = (i m ana(Xm, P) - ana(Ym, H)) / a ; curl = (i m ana(Ym, P) + ana(Xm, H)) / a
    Xm = legendre_analysis_t(g, times_im_t(g, divb), g.P, wt) + legendre_analysis_t(g, curlb, g.H, wt)
    Ym = -legendre_analysis_t(g, divb, g.H, wt) + legendre_analysis_t(g, times_im_t(g, curlb), g.P, wt)
    return fourier_analysis_t(g, Xm), fourier_analysis_t(g, Ym)


# ---------------------------------------------------------------------------
# F_E: Jacobian-vector and vector-Jacobian products (Sec. 2, Sec. 4.1)


def _grid_state(swe, x):
    g, p = swe.grid, swe.p
    phi, zeta, delta = x
    zeta_g = g.synthesis(zeta)
    phi_g = g.synthesis(phi)
    U, V = g.vector_synthesis(swe.inverse_laplacian(zeta), swe.inverse_laplacian(delta), p.a)
    f = 2.0 * p.omega * g.mu[:, None]
    return zeta_g, phi_g, U, V, f


def explicit_rhs_tl(swe, x: np.ndarray, dx: np.ndarray) -> np.ndarray:
    """F_E'(x) dx: the products A..E of SWE.explicit_rhs linearised."""
    g, p = swe.grid, swe.p
    zeta_g, phi_g, U, V, f = _grid_state(swe, x)
    dphi, dzeta, ddelta = dx
    dzg = g.synthesis(dzeta)
    dpg = g.synthesis(dphi)
    dU, dV = g.vector_synthesis(swe.inverse_laplacian(dzeta), swe.inverse_laplacian(ddelta), p.a)
    dA = dzg * U + (zeta_g + f) * dU
    dB = dzg * V + (zeta_g + f) * dV
    dC = dpg * U + phi_g * dU
    dD = dpg * V + phi_g * dV
    dE = (U * dU + V * dV) / (1.0 - g.mu[:, None] ** 2)
    div_CD, _ = g.vector_analysis(dC, dD, p.a)
    div_AB, curl_AB = g.vector_analysis(dA, dB, p.a)
    E_s = g.analysis(dE)
    return zero_m0_imag(g, np.stack([-div_CD, -div_AB, curl_AB - swe.L * E_s]))


def explicit_rhs_ad(swe, x: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """F_E'(x)^t lam, the transposes of SWE.explicit_rhs's steps in reverse order."""
    g, p = swe.grid, swe.p
    zeta_g, phi_g, U, V, f = _grid_state(swe, x)
    lam = zero_m0_imag(g, lam)
    # out = [-div_CD, -div_AB, curl_AB - L E_s]
    Cb, Db = vector_analysis_t(g, -lam[0], np.zeros_like(lam[0]), p.a)
    Ab, Bb = vector_analysis_t(g, -lam[1], lam[2], p.a)
    Eb = analysis_t(g, -swe.L * lam[2])
    # A = (zeta+f) U, B = (zeta+f) V, C = phi U, D = phi V, E = (U^2+V^2) / (2 (1-mu^2))
    rc = 1.0 / (1.0 - g.mu[:, None] ** 2)
    zgb = Ab * U + Bb * V
    pgb = Cb * U + Db * V
    Ub = Ab * (zeta_g + f) + Cb * phi_g + Eb * U * rc
    Vb = Bb * (zeta_g + f) + Db * phi_g + Eb * V * rc
    psib, chib = vector_synthesis_t(g, Ub, Vb, p.a)
    # psi = lap^-1 zeta, chi = lap^-1 delta (diagonal, real)
    zeta_b = synthesis_t(g, zgb) + swe.inverse_laplacian(psib)
    phi_b = synthesis_t(g, pgb)
    delta_b = swe.inverse_laplacian(chib)
    return zero_m0_imag(g, np.stack([phi_b, zeta_b, delta_b]))


def implicit_rhs_t(swe, lam: np.ndarray) -> np.ndarray:
    """Transpose of F_I = [ -Phibar delta + nu L Phi', nu L zeta, -L Phi' + nu L delta ]."""
    p, L = swe.p, swe.L
    lp, lz, ld = lam
    return np.stack([p.nu * L * lp - L * ld, p.nu * L * lz, -p.phibar * lp + p.nu * L * ld])


def implicit_solve_t(swe, lam: np.ndarray, alpha: float) -> np.ndarray:
    """Transpose of x = (I - alpha F_I)^-1 b: solve (I - alpha F_I^t) y = lam.
    Per coefficient, with c = 1 - alpha nu L:
      (I - alpha F_I^t) = [[c, 0, alpha L], [0, c, 0], [alpha Phibar, 0, c]]."""
    p, L = swe.p, swe.L
    c = 1.0 - alpha * p.nu * L
    lp, lz, ld = lam
    yz = lz / c
    yp = (c * lp - alpha * L * ld) / (c * c - alpha * alpha * p.phibar * L)
    yd = (ld - alpha * p.phibar * yp) / c
    return np.stack([yp, yz, yd])


class Tangent:
    """A problem on (x, dx) pairs [2][3][N_c]: linear operators act on both
    parts, F_E returns (F_E(x), F_E'(x) dx).  Running the forward SDC / MLSDC
    code on it gives the tangent-linear step."""

    def __init__(self, swe):
        self.swe = swe
        self.R = swe.R

    def explicit_rhs(self, u):
        return np.stack([self.swe.explicit_rhs(u[0]), explicit_rhs_tl(self.swe, u[0], u[1])])

    def implicit_rhs(self, u):
        return np.stack([self.swe.implicit_rhs(u[0]), self.swe.implicit_rhs(u[1])])

    def implicit_solve(self, b, alpha):
        return np.stack([self.swe.implicit_solve(b[0], alpha), self.swe.implicit_solve(b[1], alpha)])

    def restrict(self, u, coarse):
        return truncate(u, self.R, coarse.R)

    def interpolate(self, u, coarse):
        return zero_pad(u, coarse.R, self.R)


def sdc_step_tl(lev: Level, u0, du0, dt, n_sweeps):
    tl = Level(Tangent(lev.prob), lev.M + 1)
    return sdc_step(tl, np.stack([u0, du0]), dt, n_sweeps)[1]


def mlsdc_step_tl(fine: Level, coarse: Level, u0, du0, dt, n_iter, n_coarse_sweeps):
    tf = Level(Tangent(fine.prob), fine.M + 1)
    tc = Level(Tangent(coarse.prob), coarse.M + 1)
    return mlsdc_step(tf, tc, np.stack([u0, du0]), dt, n_iter, n_coarse_sweeps)[1]


# ---------------------------------------------------------------------------
# transposes of the time-stepping operations (Sec. 4.2, Sec. 4.3, Algorithm 1)


def _zeros(n, like):
    return [np.zeros_like(like) for _ in range(n)]


def sweep_ad(lev: Level, dt: float, Tn, Tb, FIb, FEb, with_tau: bool):
    """Transpose of sdc.sweep.  Tn: the sweep's output nodes (F_E was
    evaluated at Tn[1..M]); Tb, FIb, FEb: adjoints of its outputs.  Returns
    the adjoints of its inputs (Theta, F_I, F_E, tau)."""
    M, Q, QE, QI, prob = lev.M, lev.Q, lev.QE, lev.QI, lev.prob
    Tnb, FInb, FEnb = list(Tb), list(FIb), list(FEb)
    Thb, FIob, FEob = _zeros(M + 1, Tb[0]), _zeros(M + 1, Tb[0]), _zeros(M + 1, Tb[0])
    taub = _zeros(M + 1, Tb[0]) if with_tau else None
    for m in reversed(range(M)):
        # FEn[m+1] = F_E(Tn[m+1]) ; FIn[m+1] = F_I(Tn[m+1])
        g = Tnb[m + 1] + explicit_rhs_ad(prob, Tn[m + 1], FEnb[m + 1]) + implicit_rhs_t(prob, FInb[m + 1])
        FEnb[m + 1] = np.zeros_like(g)
        FInb[m + 1] = np.zeros_like(g)
        Tnb[m + 1] = np.zeros_like(g)
        # Tn[m+1] = solve(b, dt qI_{m+1,m+1})
        bb = implicit_solve_t(prob, g, dt * QI[m + 1, m + 1])
        # b = Theta[0] + sum_{j<=m} dt qE (FEn_j - FE_j) + dt qI (FIn_j - FI_j)
        #     - dt qI_{m+1,m+1} FI_{m+1} + sum_j dt q (FI_j + FE_j) [+ tau_{m+1}]
        Thb[0] = Thb[0] + bb
        for j in range(m + 1):
            FEnb[j] = FEnb[j] + dt * QE[m + 1, j] * bb
            FEob[j] = FEob[j] - dt * QE[m + 1, j] * bb
            FInb[j] = FInb[j] + dt * QI[m + 1, j] * bb
            FIob[j] = FIob[j] - dt * QI[m + 1, j] * bb
        FIob[m + 1] = FIob[m + 1] - dt * QI[m + 1, m + 1] * bb
        for j in range(M + 1):
            FIob[j] = FIob[j] + dt * Q[m + 1, j] * bb
            FEob[j] = FEob[j] + dt * Q[m + 1, j] * bb
        if with_tau:
            taub[m + 1] = taub[m + 1] + bb
    # node 0 of the outputs is node 0 of the inputs
    Thb[0] = Thb[0] + Tnb[0]
    FIob[0] = FIob[0] + FInb[0]
    FEob[0] = FEob[0] + FEnb[0]
    return Thb, FIob, FEob, taub


def spread_ad(lev: Level, u0, Thb, FIb, FEb):
    """Transpose of sdc.spread: Theta^n copied to every node, F once at u0."""
    prob = lev.prob
    return sum(Thb) + implicit_rhs_t(prob, sum(FIb)) + explicit_rhs_ad(prob, u0, sum(FEb))


def sdc_step_ad(lev: Level, u0, dt, n_sweeps, lam):
    """Transpose of the tangent-linear SDC step at u0, applied to lam."""
    tape = {}
    sdc_step(lev, u0, dt, n_sweeps, tape=tape)
    M = lev.M
    Thb, FIb, FEb = _zeros(M + 1, u0), _zeros(M + 1, u0), _zeros(M + 1, u0)
    Thb[M] = lam.copy()
    for k in reversed(range(n_sweeps)):
        Thb, FIb, FEb, _ = sweep_ad(lev, dt, tape["sweeps"][k], Thb, FIb, FEb, False)
    return zero_m0_imag(lev.prob.grid, spread_ad(lev, u0, Thb, FIb, FEb))


def mlsdc_step_ad(fine: Level, coarse: Level, u0, dt, n_iter, n_coarse_sweeps, lam):
    """Transpose of the tangent-linear MLSDC step at u0 (Algorithm 1,
    n_iter iterations), applied to lam, the adjoint of the step's result."""
    pf, pc = fine.prob, coarse.prob
    Pi_cf = quadrature.lagrange_matrix(fine.t, coarse.t)
    Pi_fc = quadrature.lagrange_matrix(coarse.t, fine.t)
    Mf, Mc = fine.M, coarse.M
    Rf, Rc = pf.R, pc.R
    tape = {}
    mlsdc_step(fine, coarse, u0, dt, n_iter, n_coarse_sweeps, tape=tape)
    u0c = tape["u0c"]
    zf, zc = np.zeros_like(u0), np.zeros_like(u0c)
    Tfb, FIfb, FEfb = [zf.copy() for _ in range(Mf + 1)], [zf.copy() for _ in range(Mf + 1)], \
        [zf.copy() for _ in range(Mf + 1)]
    Tcb, FIcb, FEcb = [zc.copy() for _ in range(Mc + 1)], [zc.copy() for _ in range(Mc + 1)], \
        [zc.copy() for _ in range(Mc + 1)]
    Tfb[Mf] = lam.copy()

    def restrict_node_t(yb, i, acc):
        # restrict_node(vals, i) = truncate(sum_j Pi_cf[i, j] vals[j])
        pad = zero_pad(yb, Rc, Rf)
        for j in range(Mf + 1):
            acc[j] = acc[j] + Pi_cf[i, j] * pad

    for it in reversed(range(n_iter)):
        rec = tape["iters"][it]
        # D) X_f[m] += pad(sum_i Pi_fc[m, i] (X_c[i] - X_s[i])), m = 1..Mf
        Tsb, FIsb, FEsb = [zc.copy() for _ in range(Mc + 1)], [zc.copy() for _ in range(Mc + 1)], \
            [zc.copy() for _ in range(Mc + 1)]
        for m in range(1, Mf + 1):
            for Xfb, Xcb, Xsb in ((Tfb, Tcb, Tsb), (FIfb, FIcb, FIsb), (FEfb, FEcb, FEsb)):
                t = truncate(Xfb[m], Rf, Rc)
                for i in range(Mc + 1):
                    Xcb[i] = Xcb[i] + Pi_fc[m, i] * t
                    Xsb[i] = Xsb[i] - Pi_fc[m, i] * t
        # C) coarse sweeps, in reverse, accumulating the adjoint of tau
        taub = [zc.copy() for _ in range(Mc + 1)]
        for s in reversed(range(n_coarse_sweeps)):
            Tcb, FIcb, FEcb, tb = sweep_ad(coarse, dt, rec["coarse"][s], Tcb, FIcb, FEcb, True)
            taub = [taub[i] + tb[i] for i in range(Mc + 1)]
        # tau[i] = A_c[i] - restrict_node(A_f, i), A(Theta) = Theta - dt (Q x I)(F_I + F_E)
        Acb = taub
        Afb = [zf.copy() for _ in range(Mf + 1)]
        for i in range(Mc + 1):
            restrict_node_t(-taub[i], i, Afb)
        for lev, Ab, Tb, Ib, Eb in ((coarse, Acb, Tcb, FIcb, FEcb), (fine, Afb, Tfb, FIfb, FEfb)):
            n = lev.M + 1
            for mm in range(n):
                Tb[mm] = Tb[mm] + Ab[mm]
                for j in range(n):
                    Ib[j] = Ib[j] - dt * lev.Q[mm, j] * Ab[mm]
                    Eb[j] = Eb[j] - dt * lev.Q[mm, j] * Ab[mm]
        # B) the saved copies, then the restricted nodes and their F
        for i in range(Mc + 1):
            Tcb[i] = Tcb[i] + Tsb[i]
            FIcb[i] = FIcb[i] + FIsb[i]
            FEcb[i] = FEcb[i] + FEsb[i]
        for m in range(1, Mc + 1):
            g = Tcb[m] + implicit_rhs_t(pc, FIcb[m]) + explicit_rhs_ad(pc, rec["restricted"][m], FEcb[m])
            restrict_node_t(g, m, Tfb)
            Tcb[m], FIcb[m], FEcb[m] = zc.copy(), zc.copy(), zc.copy()
        # A) fine sweep
        Tfb, FIfb, FEfb, _ = sweep_ad(fine, dt, rec["fine"], Tfb, FIfb, FEfb, False)
    # coarse initialisation: node 0 value u0c = restrict_node(Theta_f, 0), F at u0c, copied to every node
    g = sum(Tcb) + implicit_rhs_t(pc, sum(FIcb)) + explicit_rhs_ad(pc, u0c, sum(FEcb))
    restrict_node_t(g, 0, Tfb)
    return zero_m0_imag(pf.grid, spread_ad(fine, u0, Tfb, FIfb, FEfb))


# ---------------------------------------------------------------------------
# the objective and its gradient over n time steps


def misfit(R: int, x: np.ndarray, phi_target: np.ndarray):
    """J = 1/2 ||Phi' - Phi_t||^2 (Parseval) and dJ/dx in the (Re, Im) inner product."""
    m, _ = spec_mn(R)
    wt = np.where(m == 0, 1.0, 2.0)
    r = x[0] - phi_target
    J = 0.5 * norm2(R, r)
    lam = np.zeros_like(x)
    lam[0] = wt * r
    lam[0][m == 0] = lam[0][m == 0].real
    return J, lam


def gradient(fine: Level, coarse: Level, u0, phi_target, dt, n_steps, n_iter, n_coarse_sweeps):
    """J(u0) after n_steps MLSDC steps and dJ/du0 (every step's start state is kept)."""
    states = [u0]
    for _ in range(n_steps):
        states.append(mlsdc_step(fine, coarse, states[-1], dt, n_iter, n_coarse_sweeps))
    J, lam = misfit(fine.prob.R, states[-1], phi_target)
    for s in reversed(range(n_steps)):
        lam = mlsdc_step_ad(fine, coarse, states[s], dt, n_iter, n_coarse_sweeps, lam)
    return J, lam, states[-1]


def objective(fine: Level, coarse: Level, u0, phi_target, dt, n_steps, n_iter, n_coarse_sweeps):
    u = u0
    for _ in range(n_steps):
        u = mlsdc_step(fine, coarse, u, dt, n_iter, n_coarse_sweeps)
    return misfit(fine.prob.R, u, phi_target)[0]
