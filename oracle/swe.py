"""Shallow-water right-hand sides and the implicit solve (oracle; test infrastructure only).

Sec. 2, Eqs. geopotential_equation, vorticity_equation, divergence_equation:
  dPhi'/dt  = -div(Phi' V) - Phibar delta + nu lap Phi'
  dzeta/dt  = -div((zeta + f) V) + nu lap zeta
  ddelta/dt = k . curl((zeta + f) V) - lap(Phi + V.V/2) + nu lap delta
with f = 2 Omega mu.  Sec. 4.1 (Eqs. system_of_odes_implicit_part,
system_of_odes_explicit_part) splits F = F_I + F_E with F_I = L_G (Eq.
linear_wave_motion_induced_by_gravitational_forces: gravity-wave terms and
diffusion) and F_E = L_F + N (Coriolis terms and the nonlinear terms):
  F_I = [ -Phibar delta + nu lap Phi',  nu lap zeta,  -lap Phi' + nu lap delta ]
  F_E = [ -div(Phi' V),  -div((zeta+f) V),  curl((zeta+f) V) - lap(V.V/2) ]
The full spectral form is not printed in the paper (it cites Hack & Jakob);
the transform-method evaluation below is derived from the equations above:
grid products A = (zeta+f) U, B = (zeta+f) V, C = Phi' U, D = Phi' V,
E = (U^2 + V^2) / (2 (1 - mu^2)) = V.V/2, then
  F_E = [ -div(C, D), -div(A, B), curl(A, B) + n(n+1)/a^2 E^m_n ].
Sec. 4.4, Eq. implicit_systems: x - alpha F_I(x) = b is diagonal per
coefficient.  With L = -n(n+1)/a^2 and c = 1 - alpha nu L:
  zeta  = b_zeta / c
  c Phi' + alpha Phibar delta = b_Phi ;  alpha L Phi' + c delta = b_delta
  Phi'  = (c b_Phi - alpha Phibar b_delta) / (c^2 - alpha^2 Phibar L)
  delta = (b_delta - alpha L Phi') / c
SWECoriolisImplicit is the alternative split with L_F moved into F_I; its
implicit system couples degrees n - 1, n, n + 1 and is solved densely per m.
"""
from __future__ import annotations

from dataclasses import dataclass, replace
from functools import lru_cache

import numpy as np

from . import legendre
from .sht import Grid, spec_mn, m_slice, truncate, zero_pad, zero_m0_imag


@dataclass(frozen=True)
class Params:
    a: float = 6.37122e6        # Earth radius [m]
    omega: float = 7.292e-5     # rotation rate [1/s]
    g: float = 9.80616          # gravity [m/s^2]
    phibar: float = 9.80616e4   # mean geopotential g * 1e4 m [m^2/s^2]
    nu: float = 1.0e5           # diffusion [m^2/s] (Sec. 2)


class SWE:
    """The semi-discrete system (Eq. semidiscrete_system) at truncation R on an
    I x J Gaussian grid.  State: complex128[3, N_c] = (Phi', zeta, delta)."""

    def __init__(self, R: int, I: int, J: int, params: Params = Params()):
        self.grid = Grid(R, I, J)
        self.R = R
        self.nc = self.grid.nc
        self.p = params
        self.L = self.grid.laplacian_eigenvalues(params.a)

    def inverse_laplacian(self, x: np.ndarray) -> np.ndarray:
        """psi from zeta = lap psi (Sec. 2), zero mean (n = 0 coefficient 0)."""
        out = np.zeros_like(x)
        nz = self.grid.n > 0
        out[nz] = x[nz] / self.L[nz]
        return out

    def explicit_rhs(self, x: np.ndarray) -> np.ndarray:
        g, p = self.grid, self.p
        phi, zeta, delta = x
        psi = self.inverse_laplacian(zeta)
        chi = self.inverse_laplacian(delta)
        zeta_g = g.synthesis(zeta)
        phi_g = g.synthesis(phi)
        U, V = g.vector_synthesis(psi, chi, p.a)
        f = 2.0 * p.omega * g.mu[:, None]
        A = (zeta_g + f) * U
        B = (zeta_g + f) * V
        C = phi_g * U
        D = phi_g * V
        E = (U * U + V * V) / (2.0 * (1.0 - g.mu[:, None] ** 2))
        div_CD, _ = g.vector_analysis(C, D, p.a)
        div_AB, curl_AB = g.vector_analysis(A, B, p.a)
        E_s = g.analysis(E)
        out = np.stack([-div_CD, -div_AB, curl_AB - self.L * E_s])
        return zero_m0_imag(g, out)

    def implicit_rhs(self, x: np.ndarray) -> np.ndarray:
        p, L = self.p, self.L
        phi, zeta, delta = x
        return np.stack([-p.phibar * delta + p.nu * L * phi,
                         p.nu * L * zeta,
                         -L * phi + p.nu * L * delta])

    def implicit_solve(self, b: np.ndarray, alpha: float) -> np.ndarray:
        p, L = self.p, self.L
        c = 1.0 - alpha * p.nu * L
        zeta = b[1] / c
        phi = (c * b[0] - alpha * p.phibar * b[2]) / (c * c - alpha * alpha * p.phibar * L)
        delta = (b[2] - alpha * L * phi) / c
        return np.stack([phi, zeta, delta])

    def restrict(self, x: np.ndarray, coarse: "SWE") -> np.ndarray:
        return truncate(x, self.R, coarse.R)

    def interpolate(self, x: np.ndarray, coarse: "SWE") -> np.ndarray:
        return zero_pad(x, coarse.R, self.R)

    def total_phi_norm_rel_err(self, x: np.ndarray, ref: np.ndarray) -> float:
        """Relative L2 (Parseval) error of the total geopotential Phibar + Phi'.
        A constant Phibar has xi^0_0 = sqrt(2) Phibar."""
        from .sht import norm2
        tot = ref[0].copy()
        tot[0] += np.sqrt(2.0) * self.p.phibar
        return float(np.sqrt(norm2(self.R, x[0] - ref[0]) / norm2(self.R, tot)))


@lru_cache(maxsize=None)
def _eps_neighbours(R: int):
    """Per stored coefficient (m, n): eps^m_n (0 for n = m) and eps^m_{n+1}
    (0 for n = R), the factors of the n - 1 and n + 1 neighbours."""
    m, n = spec_mn(R)
    e_lo = np.array([legendre.eps(mm, nn) for mm, nn in zip(m, n)])
    e_hi = np.array([legendre.eps(mm, nn + 1) if nn + 1 <= R else 0.0 for mm, nn in zip(m, n)])
    return n, e_lo, e_hi


def _lower(x: np.ndarray) -> np.ndarray:
    """x[k - 1] at k (0 at k = 0); used only where eps^m_n masks the m boundary."""
    return np.concatenate([np.zeros(1, x.dtype), x[:-1]])


def _upper(x: np.ndarray) -> np.ndarray:
    """x[k + 1] at k (0 at the end); used only where eps^m_{n+1} masks n = R."""
    return np.concatenate([x[1:], np.zeros(1, x.dtype)])


def mu_times(x: np.ndarray, R: int) -> np.ndarray:
    """Spectral coefficients of mu times a field, projected on n <= R: from the
    recurrence mu P^m_n = eps^m_{n+1} P^m_{n+1} + eps^m_n P^m_{n-1} (Sec. 3),
    (mu f)^m_n = eps^m_n f^m_{n-1} + eps^m_{n+1} f^m_{n+1}."""
    _, e_lo, e_hi = _eps_neighbours(R)
    return e_lo * _lower(x) + e_hi * _upper(x)


def h_times(x: np.ndarray, R: int) -> np.ndarray:
    """Spectral coefficients of (1 - mu^2) d f / d mu, projected on n <= R: from
    H^m_n = -n eps^m_{n+1} P^m_{n+1} + (n+1) eps^m_n P^m_{n-1},
    (H f)^m_n = -(n-1) eps^m_n f^m_{n-1} + (n+2) eps^m_{n+1} f^m_{n+1}."""
    n, e_lo, e_hi = _eps_neighbours(R)
    return -(n - 1) * e_lo * _lower(x) + (n + 2) * e_hi * _upper(x)


class SWECoriolisImplicit(SWE):
    """The alternative splitting of Sec. 4.1 with the Coriolis terms treated
    implicitly: F_I = L_G + L_F, F_E = N (the paper keeps L_F explicit; this
    variant moves it).

    L_F is the linear Coriolis part of F_E, written in closed spectral form
    from Sec. 2's equations with f = 2 Omega mu and V = k x grad psi + grad chi:
      -div(f V)  = -f delta - V.grad f  = -2 Omega mu delta - (2 Omega / a^2)(i m psi + H chi)
       curl(f V) =  f zeta  + k.(grad f x V) = 2 Omega mu zeta - (2 Omega / a^2)(i m chi - H psi)
    with mu times a field and H = (1 - mu^2) d/dmu applied through the
    Legendre recurrences (mu_times, h_times), both projected on n <= R.
    N = F_E with Omega = 0 (the nonlinear terms alone).

    The implicit system x - alpha F_I(x) = b no longer decouples per
    coefficient: the Coriolis terms couple degrees n - 1, n, n + 1 of the same
    zonal wavenumber m.  It is solved as it stands, per m, as a dense complex
    linear system over the 3 (R + 1 - m) unknowns (Phi', zeta, delta) of that
    m (the blocks of F_I on each m are formed once, by applying F_I to unit
    vectors)."""

    def __init__(self, R: int, I: int, J: int, params: Params = Params()):
        super().__init__(R, I, J, params)
        self._no_rotation = SWE(R, I, J, replace(params, omega=0.0))
        self._blocks = None

    def coriolis(self, x: np.ndarray) -> np.ndarray:
        p, R = self.p, self.R
        phi, zeta, delta = x
        psi, chi = self.inverse_laplacian(zeta), self.inverse_laplacian(delta)
        m, _ = spec_mn(R)
        tw, ia2 = 2.0 * p.omega, 1.0 / (p.a * p.a)
        lz = -tw * mu_times(delta, R) - tw * ia2 * (1j * m * psi + h_times(chi, R))
        ld = tw * mu_times(zeta, R) - tw * ia2 * (1j * m * chi - h_times(psi, R))
        return np.stack([np.zeros_like(phi), lz, ld])

    def explicit_rhs(self, x: np.ndarray) -> np.ndarray:
        return self._no_rotation.explicit_rhs(x)

    def implicit_rhs(self, x: np.ndarray) -> np.ndarray:
        return SWE.implicit_rhs(self, x) + self.coriolis(x)

    def _implicit_blocks(self):
        if self._blocks is None:
            self._blocks = []
            for m in range(self.R + 1):
                sl = m_slice(self.R, m)
                nm = sl.stop - sl.start
                A = np.zeros((3 * nm, 3 * nm), complex)
                for col in range(3 * nm):
                    e = np.zeros((3, self.nc), complex)
                    e[col // nm, sl.start + col % nm] = 1.0
                    A[:, col] = self.implicit_rhs(e)[:, sl].ravel()
                self._blocks.append(A)
        return self._blocks

    def implicit_solve(self, b: np.ndarray, alpha: float) -> np.ndarray:
        x = np.zeros_like(b)
        for m, A in enumerate(self._implicit_blocks()):
            sl = m_slice(self.R, m)
            nm = sl.stop - sl.start
            x[:, sl] = np.linalg.solve(np.eye(3 * nm) - alpha * A, b[:, sl].ravel()).reshape(3, nm)
        return x
