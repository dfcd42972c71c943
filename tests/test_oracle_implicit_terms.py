"""Pins of the oracle's implicit part F_I = L_G (Sec. 4.1, Eq.
linear_wave_motion_induced_by_gravitational_forces) that do not go through
SWE.implicit_rhs's own formula:

  - every term of the full tendency (Sec. 2, Eqs. geopotential_equation,
    vorticity_equation, divergence_equation) recomputed on the grid, with the
    Laplacian taken as div(grad) through the vector transforms and the mean
    geopotential's flux -div(Phibar V) formed from the synthesised wind, and
    nu read from the paper's printed value;
  - the linear gravity waves (Omega = 0, nu = 0): a single Y^m_n in Phi'
    oscillates at omega = sqrt(Phibar n(n+1))/a (the dispersion relation of
    waves of speed sqrt(Phibar) on a sphere of radius a) and the wave's
    energy (1/2) integral(Phi'^2 + Phibar |v|^2), with |v|^2 taken from the
    synthesised wind, stays constant;
  - pure diffusion (Phibar = 0): each Y^m_n decays as exp(-nu n(n+1) t/a^2)."""
import os

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import sht
from oracle.swe import SWE, Params
from paper_1805_07923_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def _paper_nu() -> float:
    with open(GOLDEN) as f:
        for line in f:
            if line.split()[:1] == ["diffusion_nu"]:
                return float(line.split()[1])
    raise KeyError("diffusion_nu")


def _lap_grid(g: sht.Grid, s: np.ndarray, a: float) -> np.ndarray:
    """Laplacian of a spectral scalar as div(grad s): the gradient's
    cos(phi)-scaled components are the Helmholtz field with chi = s, psi = 0,
    synthesised on the grid and taken back through the divergence analysis."""
    U, V = g.vector_synthesis(np.zeros_like(s), s, a)
    div, _ = g.vector_analysis(U, V, a)
    return div


def _grid_tendency(s: SWE, x: np.ndarray, nu: float) -> np.ndarray:
    """The full right-hand side of Sec. 2's three equations, every term formed
    on the grid: fluxes of (Phibar + Phi') V and (zeta + f) V, the curl, the
    Laplacian of Phi' + V.V/2 and the diffusion, all as div / curl of
    synthesised vector fields."""
    g, p = s.grid, s.p
    phi, zeta, delta = x
    psi, chi = s.inverse_laplacian(zeta), s.inverse_laplacian(delta)
    U, V = g.vector_synthesis(psi, chi, p.a)
    f = 2.0 * p.omega * g.mu[:, None]
    phi_tot = p.phibar + g.synthesis(phi)
    zf = g.synthesis(zeta) + f
    div_mass, _ = g.vector_analysis(phi_tot * U, phi_tot * V, p.a)
    div_abs, curl_abs = g.vector_analysis(zf * U, zf * V, p.a)
    ke = g.analysis((U * U + V * V) / (2.0 * (1.0 - g.mu[:, None] ** 2)))
    t_phi = -div_mass + nu * _lap_grid(g, phi, p.a)
    t_zeta = -div_abs + nu * _lap_grid(g, zeta, p.a)
    t_delta = curl_abs - _lap_grid(g, phi + ke, p.a) + nu * _lap_grid(g, delta, p.a)
    return np.stack([t_phi, t_zeta, t_delta])


def test_paper_nu_is_the_oracle_default():
    assert Params().nu == _paper_nu() == 1.0e5


@pytest.mark.parametrize("R,I,J", [(10, 32, 16), (21, 64, 32)])
def test_diffusion_is_nu_div_grad(R, I, J):
    """Each field's diffusion term alone: with Phibar = 0 (no gravity-wave
    coupling) F_I is nu lap on every field, and lap is div(grad) on the grid."""
    nu = _paper_nu()
    s = SWE(R, I, J, Params(phibar=0.0, nu=nu))
    x = inputs.initial_state(R, seed=11)
    FI = s.implicit_rhs(x)
    # only the diffusion is left once Phibar = 0 and Phi' is zero
    y = x.copy()
    y[0] = 0.0
    FIy = s.implicit_rhs(y)
    for k in (1, 2):
        want = nu * _lap_grid(s.grid, y[k], s.p.a)
        assert np.max(np.abs(FIy[k] - want)) < 1e-12 * np.max(np.abs(want)), k
    assert np.max(np.abs(FIy[0])) == 0.0
    want0 = nu * _lap_grid(s.grid, x[0], s.p.a)
    assert np.max(np.abs(FI[0] - want0)) < 1e-12 * np.max(np.abs(want0))


@pytest.mark.parametrize("R,I,J", [(10, 32, 16), (21, 64, 32)])
def test_full_tendency_matches_the_grid_form(R, I, J):
    """F_E + F_I equals Sec. 2's three right-hand sides formed on the grid.
    F_E's own terms are pinned elsewhere (steady flow, Coriolis closed form,
    advection); this fixes F_I's gravity-wave and diffusion terms with their
    signs and nu = 1e5 from the paper."""
    nu = _paper_nu()
    s = SWE(R, I, J, Params(nu=nu))
    x = inputs.initial_state(R, seed=5)
    got = s.explicit_rhs(x) + s.implicit_rhs(x)
    want = _grid_tendency(s, x, nu)
    for k in range(3):
        scale = np.max(np.abs(want[k]))
        assert np.max(np.abs(got[k] - want[k])) < 1e-11 * scale, (k, np.max(np.abs(got[k] - want[k])) / scale)


def _fi_matrix(s: SWE) -> np.ndarray:
    nc = s.nc
    A = np.zeros((3 * nc, 3 * nc), complex)
    for k in range(3 * nc):
        e = np.zeros(3 * nc, complex)
        e[k] = 1.0
        A[:, k] = s.implicit_rhs(e.reshape(3, nc)).ravel()
    return A


def _wave_energy(s: SWE, x: np.ndarray) -> float:
    """(1/2) (1/I) sum_{iota,j} w_j (Phi'^2 + Phibar |v|^2) with the wind
    synthesised from (zeta, delta): |v|^2 = (U^2 + V^2)/(1 - mu^2)."""
    g, p = s.grid, s.p
    phi_g = g.synthesis(x[0])
    U, V = g.vector_synthesis(s.inverse_laplacian(x[1]), s.inverse_laplacian(x[2]), p.a)
    v2 = (U * U + V * V) / (1.0 - g.mu[:, None] ** 2)
    dens = phi_g ** 2 + p.phibar * v2
    return 0.5 * float(np.sum(g.w[:, None] * dens)) / g.I


@pytest.mark.parametrize("m,n", [(0, 1), (0, 4), (2, 3), (5, 5), (1, 5)])
def test_gravity_wave_dispersion_relation(m, n):
    """Omega = 0, nu = 0: Phi'(0) = Y^m_n, delta(0) = 0 evolves under F_I as
    Phi'(t) = cos(omega t) Y, delta(t) = (omega/Phibar) sin(omega t) Y with
    omega = sqrt(Phibar n(n+1))/a, by the exact exponential of F_I's matrix at
    T5, and conserves the wave energy."""
    R = 5
    p = Params(omega=0.0, nu=0.0)
    s = SWE(R, 16, 8, p)
    A = _fi_matrix(s)
    nc = s.nc
    x0 = np.zeros((3, nc), complex)
    k = sht.m_slice(R, m).start + n - m
    x0[0, k] = 1.0 if m == 0 else (0.6 - 0.8j)
    om = np.sqrt(p.phibar * n * (n + 1)) / p.a
    e0 = _wave_energy(s, x0)
    for t in (0.1 / om, 1.0 / om, 2.5 / om, 7.0 / om):
        xt = (expm(t * A) @ x0.ravel()).reshape(3, nc)
        assert np.max(np.abs(xt[0] - np.cos(om * t) * x0[0])) < 1e-12
        assert np.max(np.abs(xt[2] - (om / p.phibar) * np.sin(om * t) * x0[0])) < 1e-12 * om / p.phibar
        assert np.max(np.abs(xt[1])) == 0.0
        assert abs(_wave_energy(s, xt) - e0) < 1e-12 * e0


@pytest.mark.parametrize("m,n", [(0, 2), (3, 4), (5, 5)])
def test_diffusion_decay_rate(m, n):
    """Phibar = 0: each field's Y^m_n decays as exp(-nu n(n+1) t / a^2); a
    Phi' mode also drives delta through -lap Phi', which then grows as
    (n(n+1)/a^2) t exp(-nu n(n+1) t / a^2) (the resonant solution of
    d delta/dt = (n(n+1)/a^2) Phi' - nu (n(n+1)/a^2) delta)."""
    R = 5
    nu = _paper_nu()
    p = Params(phibar=0.0, nu=nu)
    s = SWE(R, 16, 8, p)
    A = _fi_matrix(s)
    nc = s.nc
    k = sht.m_slice(R, m).start + n - m
    lam = n * (n + 1) / p.a ** 2
    t = 3.0 / (nu * lam)   # three e-folds
    for field in range(3):
        x0 = np.zeros((3, nc), complex)
        x0[field, k] = 1.0
        xt = (expm(t * A) @ x0.ravel()).reshape(3, nc)
        assert abs(xt[field, k] - np.exp(-3.0)) < 1e-13
        if field == 0:
            want = lam * t * np.exp(-3.0)
            assert abs(xt[2, k] - want) < 1e-13 * want
            xt[2, k] = 0.0
        xt[field, k] = 0.0
        assert np.max(np.abs(xt)) < 1e-13
