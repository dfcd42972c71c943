"""The oracle's pins are not vacuous: each plausible mistake planted here in the
oracle (on the CPU, by monkeypatching) makes at least one pin fail."""
import numpy as np
import pytest

from oracle import quadrature, sdc, sht, swe

import test_oracle_coriolis_implicit as T_ci
import test_oracle_quadrature as T_q
import test_oracle_sdc as T_sdc
import test_oracle_sht as T_sht
import test_oracle_swe as T_swe


def _fails(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def _vector_analysis_factory(sign_div_h=-1.0, sign_curl_h=1.0):
    def vector_analysis(self, X, Y, a):
        wt = self.w / (1.0 - self.mu ** 2)
        Xm, Ym = self.fourier_analysis(X), self.fourier_analysis(Y)
        im = 1j * self.m
        div = (im * self.legendre_analysis(Xm, self.P, wt) + sign_div_h * self.legendre_analysis(Ym, self.H, wt)) / a
        curl = (im * self.legendre_analysis(Ym, self.P, wt) + sign_curl_h * self.legendre_analysis(Xm, self.H, wt)) / a
        return sht.zero_m0_imag(self, div), sht.zero_m0_imag(self, curl)
    return vector_analysis


def test_curl_sign_mistake_is_caught(monkeypatch):
    monkeypatch.setattr(sht.Grid, "vector_analysis", _vector_analysis_factory(sign_curl_h=-1.0))
    _fails(T_sht.test_solid_body_rotation_vorticity)
    _fails(T_swe.test_steady_zonal_flow_is_exact_equilibrium)


def test_div_sign_mistake_is_caught(monkeypatch):
    monkeypatch.setattr(sht.Grid, "vector_analysis", _vector_analysis_factory(sign_div_h=1.0))
    _fails(T_sht.test_laplacian_eigenfunction_through_gradient, 10, 32, 16)
    _fails(T_swe.test_tilted_rigid_rotation_preserves_degree_and_is_skew)


def test_missing_im_in_vector_synthesis_is_caught(monkeypatch):
    def vector_synthesis(self, psi, chi, a):
        U_m = (self.legendre_synthesis(chi, self.P) - self.legendre_synthesis(psi, self.H)) / a
        V_m = (self.legendre_synthesis(psi, self.P) + self.legendre_synthesis(chi, self.H)) / a
        return self.fourier_synthesis(U_m), self.fourier_synthesis(V_m)
    monkeypatch.setattr(sht.Grid, "vector_synthesis", vector_synthesis)
    _fails(T_sht.test_laplacian_eigenfunction_through_gradient, 10, 32, 16)


def test_kinetic_energy_factor_mistake_is_caught(monkeypatch):
    orig = swe.SWE.explicit_rhs

    def rhs(self, x):
        out = orig(self, x)
        g = self.grid
        psi, chi = self.inverse_laplacian(x[1]), self.inverse_laplacian(x[2])
        U, V = g.vector_synthesis(psi, chi, self.p.a)
        E = (U * U + V * V) / (2.0 * (1.0 - g.mu[:, None] ** 2))
        out[2] = out[2] - self.L * g.analysis(E)      # doubles the V.V/2 term
        return out
    monkeypatch.setattr(swe.SWE, "explicit_rhs", rhs)
    _fails(T_swe.test_steady_zonal_flow_is_exact_equilibrium)


def test_coriolis_factor_mistake_is_caught(monkeypatch):
    monkeypatch.setattr(swe, "Params", swe.Params)
    orig = swe.SWE.explicit_rhs

    def rhs(self, x):
        p = self.p
        self.p = swe.Params(p.a, p.omega / 2, p.g, p.phibar, p.nu)   # f = Omega mu
        try:
            return orig(self, x)
        finally:
            self.p = p
    monkeypatch.setattr(swe.SWE, "explicit_rhs", rhs)
    _fails(T_swe.test_coriolis_is_linear_part_closed_form, 10, 32, 16)
    _fails(T_swe.test_steady_zonal_flow_is_exact_equilibrium)


def test_implicit_solve_sign_mistake_is_caught(monkeypatch):
    def solve(self, b, alpha):
        p, L = self.p, self.L
        c = 1.0 - alpha * p.nu * L
        zeta = b[1] / c
        phi = (c * b[0] + alpha * p.phibar * b[2]) / (c * c - alpha * alpha * p.phibar * L)
        delta = (b[2] - alpha * L * phi) / c
        return np.stack([phi, zeta, delta])
    monkeypatch.setattr(swe.SWE, "implicit_solve", solve)
    _fails(T_swe.test_implicit_solve_matches_dense_solve)


def test_transposed_lu_factor_is_caught(monkeypatch):
    orig = quadrature.lu_implicit_matrix

    def upper(Q):
        QI = orig(Q)
        QI[1:, 1:] = QI[1:, 1:].T
        return QI
    monkeypatch.setattr(quadrature, "lu_implicit_matrix", upper)
    _fails(T_q.test_lu_trick_three_nodes_by_hand)
    _fails(T_q.test_lu_trick_nilpotent, 5)


def test_wrong_fas_sign_is_caught(monkeypatch):
    orig = sdc.collocation_operator

    def bad(lev, dt, Theta, FI, FE):
        n = lev.M + 1
        return [Theta[m] + dt * sum(lev.Q[m, j] * (FI[j] + FE[j]) for j in range(n)) for m in range(n)]
    monkeypatch.setattr(sdc, "collocation_operator", bad)
    _fails(T_sdc.test_mlsdc_fixed_point_is_not_moved)


def test_dropped_interpolation_of_F_is_caught(monkeypatch):
    """Step D without the F corrections: the fine F values go stale, so MLSDC
    with an identical coarse level no longer equals SDC."""
    src_interp = sdc.mlsdc_step

    def no_f_interp(fine, coarse, u0, dt, n_iter, n_coarse_sweeps=1, return_nodes=False):
        pf, pc = fine.prob, coarse.prob
        Pi_cf = quadrature.lagrange_matrix(fine.t, coarse.t)
        Pi_fc = quadrature.lagrange_matrix(coarse.t, fine.t)
        Mf, Mc = fine.M, coarse.M
        rn = lambda v, i: pf.restrict(sum(Pi_cf[i, j] * v[j] for j in range(Mf + 1)), pc)
        ip = lambda d, m: pf.interpolate(sum(Pi_fc[m, i] * d[i] for i in range(Mc + 1)), pc)
        Th_f, FI_f, FE_f = sdc.spread(fine, u0)
        u0c = rn(Th_f, 0)
        Th_c, FI_c, FE_c = [u0c] * (Mc + 1), [pc.implicit_rhs(u0c)] * (Mc + 1), [pc.explicit_rhs(u0c)] * (Mc + 1)
        for _ in range(n_iter):
            Th_f, FI_f, FE_f = sdc.sweep(fine, dt, Th_f, FI_f, FE_f)
            Th_c, FI_c, FE_c = list(Th_c), list(FI_c), list(FE_c)
            for m in range(1, Mc + 1):
                Th_c[m] = rn(Th_f, m)
                FI_c[m], FE_c[m] = pc.implicit_rhs(Th_c[m]), pc.explicit_rhs(Th_c[m])
            Th_s = list(Th_c)
            A_c = sdc.collocation_operator(coarse, dt, Th_c, FI_c, FE_c)
            A_f = sdc.collocation_operator(fine, dt, Th_f, FI_f, FE_f)
            tau = [A_c[i] - rn(A_f, i) for i in range(Mc + 1)]
            for _s in range(n_coarse_sweeps):
                Th_c, FI_c, FE_c = sdc.sweep(coarse, dt, Th_c, FI_c, FE_c, tau)
            dT = [Th_c[i] - Th_s[i] for i in range(Mc + 1)]
            Th_f = [Th_f[0]] + [Th_f[m] + ip(dT, m) for m in range(1, Mf + 1)]
        return (Th_f, FI_f, FE_f) if return_nodes else Th_f[-1]
    monkeypatch.setattr(sdc, "mlsdc_step", no_f_interp)
    _fails(T_sdc.test_mlsdc_with_identical_levels_is_sdc)
    assert src_interp is not sdc.mlsdc_step


# ---- the adjoint's pins (tests/test_oracle_adjoint.py) -----------------------
import test_oracle_adjoint as T_ad  # noqa: E402
from oracle import adjoint as oad  # noqa: E402


def test_adjoint_sign_of_im_m_mistake_is_caught(monkeypatch):
    monkeypatch.setattr(oad, "times_im_t", lambda g, x: 1j * g.m * x)
    _fails(T_ad.test_scalar_and_vector_transform_transposes)
    _fails(T_ad.test_explicit_rhs_adjoint_dot_product)


def test_adjoint_untransposed_implicit_solve_is_caught(monkeypatch):
    monkeypatch.setattr(oad, "implicit_solve_t", lambda swe_, lam, alpha: swe_.implicit_solve(lam, alpha))
    _fails(T_ad.test_implicit_transposes)
    _fails(T_ad.test_sdc_step_adjoint_dot_product)


def test_adjoint_dropped_F_I_term_in_sweep_is_caught(monkeypatch):
    monkeypatch.setattr(oad, "implicit_rhs_t", lambda swe_, lam: 0.0 * lam)
    _fails(T_ad.test_sdc_step_adjoint_dot_product)


def test_adjoint_dropped_tau_is_caught(monkeypatch):
    orig = oad.sweep_ad

    def no_tau(lev, dt, Tn, Tb, FIb, FEb, with_tau):
        Thb, FIob, FEob, taub = orig(lev, dt, Tn, Tb, FIb, FEb, with_tau)
        return Thb, FIob, FEob, ([0.0 * t for t in taub] if with_tau else None)
    monkeypatch.setattr(oad, "sweep_ad", no_tau)
    _fails(T_ad.test_mlsdc_step_adjoint_dot_product)


def test_adjoint_missing_kinetic_energy_weight_is_caught(monkeypatch):
    """The E-term adjoint without its 1/(1 - mu^2) factor."""
    orig_t = oad.analysis_t

    def bad(g, s):
        return orig_t(g, s) * (1.0 - g.mu[:, None] ** 2)
    monkeypatch.setattr(oad, "analysis_t", bad)
    _fails(T_ad.test_explicit_rhs_adjoint_dot_product)


def test_coriolis_closed_form_sign_mistake_is_caught(monkeypatch):
    def coriolis(self, x):
        p, R = self.p, self.R
        _, zeta, delta = x
        psi, chi = self.inverse_laplacian(zeta), self.inverse_laplacian(delta)
        m, _ = sht.spec_mn(R)
        tw, ia2 = 2.0 * p.omega, 1.0 / (p.a * p.a)
        lz = -tw * swe.mu_times(delta, R) - tw * ia2 * (1j * m * psi + swe.h_times(chi, R))
        ld = tw * swe.mu_times(zeta, R) - tw * ia2 * (1j * m * chi + swe.h_times(psi, R))   # sign of H psi
        return np.stack([np.zeros_like(zeta), lz, ld])
    monkeypatch.setattr(swe.SWECoriolisImplicit, "coriolis", coriolis)
    _fails(T_ci.test_closed_form_coriolis_is_the_transform_linear_part, 10, 32, 16)


def test_coupled_solve_without_coriolis_is_caught(monkeypatch):
    monkeypatch.setattr(swe.SWECoriolisImplicit, "implicit_solve", swe.SWE.implicit_solve)
    _fails(T_ci.test_coupled_solve_residual_against_transform_coriolis, 3.0e3)
    _fails(T_ci.test_fully_implicit_linear_sweeps_reach_collocation)


def test_dropped_restricted_tau_in_three_levels_is_caught(monkeypatch):
    import inspect
    import test_oracle_mlsdc_levels as T_lv
    src = inspect.getsource(sdc.mlsdc_step_levels)
    planted = src.replace("            if tau[l] is not None:\n"
                          "                tau[c] = [tau[c][i] + restrict(l, tau[l], i) for i in range(levels[c].M + 1)]\n", "")
    assert planted != src
    ns = dict(vars(sdc))
    exec(planted, ns)
    monkeypatch.setattr(sdc, "mlsdc_step_levels", ns["mlsdc_step_levels"])
    _fails(T_lv.test_three_levels_reach_the_fine_collocation_solution)


# ---- F_I's terms (tests/test_oracle_implicit_terms.py) ----------------------
import test_oracle_implicit_terms as T_fi  # noqa: E402


def test_consistent_anti_diffusion_is_caught(monkeypatch):
    """-nu lap in F_I and the matching solve (c = 1 + alpha nu L): the solve
    still inverts its F_I, so only the forward pins of F_I's terms can see it."""
    def rhs(self, x):
        p, L = self.p, self.L
        phi, zeta, delta = x
        return np.stack([-p.phibar * delta - p.nu * L * phi,
                         -p.nu * L * zeta,
                         -L * phi - p.nu * L * delta])

    def solve(self, b, alpha):
        p, L = self.p, self.L
        c = 1.0 + alpha * p.nu * L
        zeta = b[1] / c
        phi = (c * b[0] - alpha * p.phibar * b[2]) / (c * c - alpha * alpha * p.phibar * L)
        delta = (b[2] - alpha * L * phi) / c
        return np.stack([phi, zeta, delta])
    monkeypatch.setattr(swe.SWE, "implicit_rhs", rhs)
    monkeypatch.setattr(swe.SWE, "implicit_solve", solve)
    T_swe.test_implicit_solve_matches_dense_solve()       # consistent: the solve pin passes
    _fails(T_fi.test_diffusion_is_nu_div_grad, 10, 32, 16)
    _fails(T_fi.test_full_tendency_matches_the_grid_form, 10, 32, 16)
    _fails(T_fi.test_diffusion_decay_rate, 3, 4)


def test_consistent_flip_of_the_mean_geopotential_flux_is_caught(monkeypatch):
    """+Phibar delta in the Phi' row of F_I and the matching solve."""
    def rhs(self, x):
        p, L = self.p, self.L
        phi, zeta, delta = x
        return np.stack([p.phibar * delta + p.nu * L * phi,
                         p.nu * L * zeta,
                         -L * phi + p.nu * L * delta])

    def solve(self, b, alpha):
        p, L = self.p, self.L
        c = 1.0 - alpha * p.nu * L
        zeta = b[1] / c
        phi = (c * b[0] + alpha * p.phibar * b[2]) / (c * c + alpha * alpha * p.phibar * L)
        delta = (b[2] - alpha * L * phi) / c
        return np.stack([phi, zeta, delta])
    monkeypatch.setattr(swe.SWE, "implicit_rhs", rhs)
    monkeypatch.setattr(swe.SWE, "implicit_solve", solve)
    T_swe.test_implicit_solve_matches_dense_solve()
    _fails(T_fi.test_gravity_wave_dispersion_relation, 2, 3)
    _fails(T_fi.test_full_tendency_matches_the_grid_form, 10, 32, 16)


def test_flipped_pressure_gradient_term_is_caught(monkeypatch):
    """+lap Phi' in the delta row of F_I (and the matching solve): the wave
    equation's product of the two coupling terms changes sign."""
    def rhs(self, x):
        p, L = self.p, self.L
        phi, zeta, delta = x
        return np.stack([-p.phibar * delta + p.nu * L * phi,
                         p.nu * L * zeta,
                         L * phi + p.nu * L * delta])
    monkeypatch.setattr(swe.SWE, "implicit_rhs", rhs)
    _fails(T_fi.test_gravity_wave_dispersion_relation, 2, 3)
    _fails(T_fi.test_full_tendency_matches_the_grid_form, 10, 32, 16)


def test_wrong_nu_value_is_caught(monkeypatch):
    orig = swe.SWE.implicit_rhs

    def rhs(self, x):
        p = self.p
        self.p = swe.Params(p.a, p.omega, p.g, p.phibar, p.nu * 2.0)
        try:
            return orig(self, x)
        finally:
            self.p = p
    monkeypatch.setattr(swe.SWE, "implicit_rhs", rhs)
    _fails(T_fi.test_diffusion_is_nu_div_grad, 10, 32, 16)
    _fails(T_fi.test_diffusion_decay_rate, 0, 2)


# ---- PFASST (tests/test_oracle_pfasst.py) ------------------------------------
import test_oracle_pfasst as T_pf  # noqa: E402
from oracle import pfasst as opf  # noqa: E402


def _planted_pfasst(monkeypatch, old, new):
    import inspect
    src = inspect.getsource(opf.pfasst)
    assert old in src
    ns = dict(vars(opf))
    exec(src.replace(old, new), ns)
    monkeypatch.setattr(opf, "pfasst", ns["pfasst"])


def _pf_fixtures():
    from oracle import sdc as osdc
    from oracle.swe import SWE, Params
    from paper_1805_07923_gb300 import inputs
    fine = osdc.Level(SWE(T_pf.RF, 32, 16, Params()), 3)
    coarse = osdc.Level(SWE(T_pf.RC, 16, 8, Params()), 2)
    u, seq = inputs.initial_state(T_pf.RF), []
    for _ in range(T_pf.P):
        u = osdc.sdc_step(fine, u, T_pf.DT, 60)
        seq.append(u)
    return (fine, coarse), seq


def test_pfasst_without_coarse_initial_value_is_caught(monkeypatch):
    _planted_pfasst(monkeypatch, "            if p >= 1:\n                Th_c, FI_c, FE_c = with_node0(coarse, Th_c, "
                    "FI_c, FE_c, coarse_end)\n", "")
    lv, seq = _pf_fixtures()
    _fails(T_pf.test_identical_levels_one_iteration_is_serial_collocation, lv, seq)


def test_pfasst_without_fine_initial_value_is_caught(monkeypatch):
    _planted_pfasst(monkeypatch, "            if p >= 1 and k >= 1:\n", "            if False:\n")
    lv, seq = _pf_fixtures()
    _fails(T_pf.test_converges_to_serial_collocation, lv, seq)


def test_pfasst_without_tau_is_caught(monkeypatch):
    _planted_pfasst(monkeypatch, "sweep(coarse, dt, Th_c, FI_c, FE_c, tau)", "sweep(coarse, dt, Th_c, FI_c, FE_c)")
    lv, _ = _pf_fixtures()
    _fails(T_pf.test_one_slice_is_mlsdc, lv)


def test_pfasst_without_F_interpolation_is_caught(monkeypatch):
    _planted_pfasst(monkeypatch, "                FE_f[m] = FE_f[m] + interpolate_node(dE, m)\n", "")
    lv, _ = _pf_fixtures()
    _fails(T_pf.test_first_slice_is_mlsdc, lv)
