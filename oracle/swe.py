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
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .sht import Grid, truncate, zero_pad, zero_m0_imag


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
