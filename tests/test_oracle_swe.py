"""Pins of the oracle's shallow-water right-hand sides and implicit solve
(Sec. 2, Sec. 4.1, Sec. 4.4) against facts the equations fix:
  - an exact steady zonal flow (solid-body rotation in gradient-wind balance),
  - the closed-form spectral Coriolis operator (the linear part of F_E),
  - advection by a rigid rotation (polar axis: a phase; tilted axis:
    degree-preserving and skew),
  - equivariance under rotations of the sphere when Omega = 0,
  - conservation of the mean geopotential,
  - the implicit solve against a dense solve."""
import numpy as np
import pytest

from oracle import legendre, sht
from oracle.swe import SWE, Params
from paper_1805_07923_gb300 import inputs

P0 = Params()


def inner(R, x, y):
    m, _ = sht.spec_mn(R)
    wt = np.where(m == 0, 1.0, 2.0)
    return float(np.real(np.sum(wt * x * np.conj(y))))


def mu_times(x, R):
    """Spectral coefficients of mu * field, projected on n <= R."""
    m, n = sht.spec_mn(R)
    out = np.zeros_like(x)
    for k in range(len(x)):
        mm, nn = m[k], n[k]
        if nn - 1 >= mm:
            out[k] += legendre.eps(mm, nn) * x[k - 1]
        if nn + 1 <= R:
            out[k] += legendre.eps(mm, nn + 1) * x[k + 1]
    return out


def hder(x, R):
    """Spectral coefficients of (1 - mu^2) d field / d mu, projected on n <= R."""
    m, n = sht.spec_mn(R)
    out = np.zeros_like(x)
    for k in range(len(x)):
        mm, nn = m[k], n[k]
        if nn - 1 >= mm:
            out[k] += -(nn - 1) * legendre.eps(mm, nn) * x[k - 1]
        if nn + 1 <= R:
            out[k] += (nn + 2) * legendre.eps(mm, nn + 1) * x[k + 1]
    return out


def test_steady_zonal_flow_is_exact_equilibrium():
    """u = u0 cos(phi) with Phi' = C - (a Omega u0 + u0^2/2) mu^2 is steady
    (derived from the momentum balance (zeta + f) u = -(1/a) d(Phi + u^2/2)/dphi);
    with nu = 0, F_E + F_I vanishes."""
    p = Params(nu=0.0)
    s = SWE(12, 40, 20, p)
    u0 = 35.0
    g = s.grid
    phi_grid = -(p.a * p.omega * u0 + u0 * u0 / 2) * (g.mu[:, None] ** 2 - 1.0 / 3.0) * np.ones((1, g.I))
    phi = g.analysis(phi_grid)
    zeta = np.zeros(s.nc, complex)
    zeta[1] = 2 * u0 / p.a / np.sqrt(1.5)
    x = np.stack([phi, zeta, np.zeros(s.nc, complex)])
    F = s.explicit_rhs(x) + s.implicit_rhs(x)
    scale = np.abs(s.L * phi).max()
    flux_scale = np.abs(phi).max() * u0 / p.a          # size of div(Phi' V)
    assert np.max(np.abs(F[0])) < 1e-13 * flux_scale
    vort_flux_scale = (2 * u0 / p.a + 2 * p.omega) * u0 / p.a   # size of div((zeta + f) V)
    assert np.max(np.abs(F[1])) < 1e-13 * vort_flux_scale
    assert np.max(np.abs(F[2])) < 1e-12 * scale
    assert abs(phi[0]) < 1e-10


@pytest.mark.parametrize("R,I,J", [(10, 32, 16), (21, 64, 32)])
def test_coriolis_is_linear_part_closed_form(R, I, J):
    s = SWE(R, I, J, P0)
    x = inputs.initial_state(R, seed=7)
    lin = (s.explicit_rhs(x) - s.explicit_rhs(-x)) / 2.0
    phi, zeta, delta = x
    psi, chi = s.inverse_laplacian(zeta), s.inverse_laplacian(delta)
    m, _ = sht.spec_mn(R)
    W, a = P0.omega, P0.a
    ref_zeta = -2 * W * mu_times(delta, R) - 2 * W / a ** 2 * (1j * m * psi + hder(chi, R))
    ref_delta = 2 * W * mu_times(zeta, R) - 2 * W / a ** 2 * (1j * m * chi - hder(psi, R))
    assert np.max(np.abs(lin[0])) < 1e-14 * np.max(np.abs(s.explicit_rhs(x)[0]))
    assert np.max(np.abs(lin[1] - ref_zeta)) < 1e-11 * np.max(np.abs(ref_zeta))
    assert np.max(np.abs(lin[2] - ref_delta)) < 1e-11 * np.max(np.abs(ref_delta))


def test_polar_rigid_rotation_advects_by_phase():
    R = 16
    s = SWE(R, 52, 26, P0)
    u0 = 25.0
    phi = inputs.spectrum(R, 11, 0, 100.0)
    zeta = np.zeros(s.nc, complex)
    zeta[1] = 2 * u0 / P0.a / np.sqrt(1.5)
    x = np.stack([phi, zeta, np.zeros(s.nc, complex)])
    m, _ = sht.spec_mn(R)
    F = s.explicit_rhs(x)
    ref = -1j * m * u0 / P0.a * phi
    assert np.max(np.abs(F[0] - ref)) < 1e-12 * np.max(np.abs(ref))


def test_tilted_rigid_rotation_preserves_degree_and_is_skew():
    R = 14
    s = SWE(R, 44, 22, P0)
    m, n = sht.spec_mn(R)
    psi = np.zeros(s.nc, complex)
    psi[sht.m_slice(R, 1)][0] = 3.0e7 * (0.6 - 0.8j)     # degree-1 stream function
    zeta = s.L * psi
    for n0 in (3, 9, 14):
        phi = np.where(n == n0, inputs.spectrum(R, 5, 0, 100.0), 0)
        x = np.stack([phi, zeta, np.zeros(s.nc, complex)])
        F = s.explicit_rhs(x)[0]
        big = np.max(np.abs(F))
        assert big > 0
        assert np.max(np.abs(F[n != n0])) < 1e-12 * big
        assert abs(inner(R, phi, F)) < 1e-12 * np.sqrt(inner(R, phi, phi) * inner(R, F, F))


def _eval_at(g, x, lam, mu):
    """Direct evaluation of Eq. spectral_to_physical_space at arbitrary points."""
    R = g.R
    P = legendre.assoc_legendre(R, mu)
    out = np.zeros(mu.shape)
    for m in range(R + 1):
        sl = sht.m_slice(R, m)
        Fm = x[sl] @ P[m, m:]
        out += (1.0 if m == 0 else 2.0) * np.real(Fm * np.exp(1j * m * lam))
    return out


def _rotate(g, x, beta):
    """Spectral coefficients of the field rotated by beta about the x axis."""
    lam, mu = np.meshgrid(g.lam, g.mu)
    c = np.sqrt(1 - mu * mu)
    p = np.stack([c * np.cos(lam), c * np.sin(lam), mu])
    cb, sb = np.cos(beta), np.sin(beta)
    q = np.stack([p[0], cb * p[1] + sb * p[2], -sb * p[1] + cb * p[2]])   # R_x(-beta) p
    lam_q = np.arctan2(q[1], q[0])
    vals = _eval_at(g, x, lam_q.ravel(), q[2].ravel()).reshape(mu.shape)
    return g.analysis(vals)


def test_rotation_equivariance_without_coriolis():
    p = Params(omega=0.0)
    R = 10
    s = SWE(R, 32, 16, p)
    x = inputs.initial_state(R, seed=21)
    beta = 0.7
    xr = np.stack([_rotate(s.grid, x[k], beta) for k in range(3)])
    FE = s.explicit_rhs(x)
    FEr = s.explicit_rhs(xr)
    for k in range(3):
        rot = _rotate(s.grid, FE[k], beta)
        assert np.max(np.abs(FEr[k] - rot)) < 1e-11 * np.max(np.abs(rot)), k
    FI = s.implicit_rhs(x)
    FIr = s.implicit_rhs(xr)
    for k in range(3):
        rot = _rotate(s.grid, FI[k], beta)
        assert np.max(np.abs(FIr[k] - rot)) < 1e-11 * np.max(np.abs(rot)), k


def test_mean_geopotential_is_conserved_by_rhs():
    s = SWE(21, 64, 32, P0)
    x = inputs.initial_state(21)
    x[0, 0] = 123.0
    FE = s.explicit_rhs(x)
    FI = s.implicit_rhs(x)
    assert abs(FE[0, 0]) < 1e-14 * np.max(np.abs(FE[0]))
    assert FI[0, 0] == 0.0
    assert FE[2, 0] == 0.0 or abs(FE[2, 0]) < 1e-14 * np.max(np.abs(FE[2]))


def test_implicit_solve_matches_dense_solve():
    R = 5
    s = SWE(R, 16, 8, P0)
    nc = s.nc
    alpha = 417.0
    b = inputs.initial_state(R, seed=3)
    x = s.implicit_solve(b, alpha)
    resid = x - alpha * s.implicit_rhs(x) - b
    assert np.max(np.abs(resid)) < 1e-13 * np.max(np.abs(b))
    # dense operator of F_I on the complex state vector
    Amat = np.zeros((3 * nc, 3 * nc), complex)
    for k in range(3 * nc):
        e = np.zeros(3 * nc, complex)
        e[k] = 1.0
        Amat[:, k] = s.implicit_rhs(e.reshape(3, nc)).ravel()
    xd = np.linalg.solve(np.eye(3 * nc) - alpha * Amat, b.ravel()).reshape(3, nc)
    for k in range(3):
        assert np.max(np.abs(xd[k] - x[k])) < 1e-13 * np.max(np.abs(x[k]))
