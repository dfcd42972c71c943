"""Pins of the oracle's spherical-harmonic transforms (Sec. 3; Sec. 2 for the
vector forms): round trip, Parseval, closed-form harmonics, the Laplacian
eigenvalue reached through the grid-gradient path, div/curl round trip and
solid-body rotation."""
import numpy as np
import pytest

from oracle import sht
from paper_1805_07923_gb300 import inputs

A = 6.37122e6


def _rand_spec(R, seed=0):
    rng = np.random.default_rng(seed)
    nc = sht.n_coeffs(R)
    x = rng.standard_normal(nc) + 1j * rng.standard_normal(nc)
    x[: R + 1] = x[: R + 1].real
    return x


@pytest.mark.parametrize("R,I,J", [(5, 16, 8), (21, 64, 32), (42, 128, 64), (85, 256, 128)])
def test_round_trip(R, I, J):
    g = sht.Grid(R, I, J)
    x = _rand_spec(R)
    y = g.analysis(g.synthesis(x))
    assert np.max(np.abs(y - x)) < 1e-13 * np.max(np.abs(x)) * np.sqrt(R)


def test_parseval():
    g = sht.Grid(21, 64, 32)
    x = _rand_spec(21, 3)
    f = g.synthesis(x)
    grid_norm = np.sum(g.w[:, None] * f * f) / g.I
    assert abs(grid_norm - sht.norm2(21, x)) < 1e-12 * grid_norm


def test_single_harmonics_closed_form():
    g = sht.Grid(4, 16, 8)
    lam, mu = np.meshgrid(g.lam, g.mu)
    x = np.zeros(g.nc, complex)
    x[sht.m_slice(4, 1)][0] = 1.0          # xi^1_1 = 1
    f = g.synthesis(x)
    assert np.max(np.abs(f - 2 * np.sqrt(3) / 2 * np.sqrt(1 - mu * mu) * np.cos(lam))) < 1e-15
    x = np.zeros(g.nc, complex)
    x[sht.m_slice(4, 2)][0] = 1j           # xi^2_2 = i
    f = g.synthesis(x)
    ref = 2 * np.sqrt(15) / 4 * (1 - mu * mu) * np.real(1j * np.exp(2j * lam))
    assert np.max(np.abs(f - ref)) < 1e-15
    x = np.zeros(g.nc, complex)
    x[1] = 1.0                             # xi^0_1
    assert np.max(np.abs(g.synthesis(x) - np.sqrt(1.5) * mu)) < 1e-15


def test_fourier_analysis_definition():
    g = sht.Grid(10, 32, 16)
    f = np.cos(3 * g.lam)[None, :] * np.ones((16, 1)) + 0.5
    F = g.fourier_analysis(f)
    assert np.max(np.abs(F[:, 3] - 0.5)) < 1e-15
    assert np.max(np.abs(F[:, 0] - 0.5)) < 1e-15
    F[:, 3] = 0
    F[:, 0] = 0
    assert np.max(np.abs(F)) < 1e-15


@pytest.mark.parametrize("R,I,J", [(10, 32, 16), (21, 64, 32)])
def test_laplacian_eigenfunction_through_gradient(R, I, J):
    """The gradient of Y^m_n is the Helmholtz field with chi = Y, psi = 0; its
    divergence through the vector analysis must be -n(n+1)/a^2 Y^m_n."""
    g = sht.Grid(R, I, J)
    for (m, n) in [(0, 1), (0, 5), (1, 1), (3, 7), (R, R), (2, R)]:
        x = np.zeros(g.nc, complex)
        x[sht.m_slice(R, m)][n - m] = 1.0 if m == 0 else (0.3 + 0.7j)
        U, V = g.vector_synthesis(np.zeros_like(x), x, A)
        div, curl = g.vector_analysis(U, V, A)
        assert np.max(np.abs(div + n * (n + 1) / A ** 2 * x)) < 1e-13 * n * (n + 1) / A ** 2
        assert np.max(np.abs(curl)) < 1e-13 * n * (n + 1) / A ** 2


@pytest.mark.parametrize("R,I,J", [(21, 64, 32), (42, 128, 64)])
def test_div_curl_round_trip(R, I, J):
    g = sht.Grid(R, I, J)
    zeta = _rand_spec(R, 1)
    delta = _rand_spec(R, 2)
    zeta[0] = delta[0] = 0.0
    L = g.laplacian_eigenvalues(A)
    nz = g.n > 0
    psi = np.zeros_like(zeta)
    chi = np.zeros_like(delta)
    psi[nz] = zeta[nz] / L[nz]
    chi[nz] = delta[nz] / L[nz]
    U, V = g.vector_synthesis(psi, chi, A)
    div, curl = g.vector_analysis(U, V, A)
    assert np.max(np.abs(div - delta)) < 1e-12 * np.max(np.abs(delta))
    assert np.max(np.abs(curl - zeta)) < 1e-12 * np.max(np.abs(zeta))


def test_solid_body_rotation_vorticity():
    """u = u0 cos(phi), v = 0 has vorticity 2 u0 sin(phi) / a and no divergence."""
    g = sht.Grid(10, 32, 16)
    u0 = 20.0
    U = u0 * (1 - g.mu[:, None] ** 2) * np.ones((1, g.I))
    div, curl = g.vector_analysis(U, np.zeros_like(U), A)
    ref = np.zeros(g.nc, complex)
    ref[1] = 2 * u0 / A / np.sqrt(1.5)
    assert np.max(np.abs(curl - ref)) < 1e-14 * abs(ref[1])
    assert np.max(np.abs(div)) < 1e-14 * abs(ref[1])


def test_truncate_and_pad_are_transposes():
    x = inputs.initial_state(12)[1]
    xt = sht.truncate(x, 12, 6)
    xp = sht.zero_pad(xt, 6, 12)
    assert np.array_equal(sht.truncate(xp, 12, 6), xt)
    m, n = sht.spec_mn(12)
    assert np.array_equal(xp[n <= 6], x[n <= 6])
    assert np.all(xp[n > 6] == 0)
    assert np.array_equal(inputs.truncate(x, 12, 6), xt)
