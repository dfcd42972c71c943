"""Spherical-harmonic transforms on a Gaussian grid (oracle; test infrastructure only).

Sec. 3:
  Eq. spectral_to_physical_space  xi(lambda, mu) = sum_{r=-R..R} sum_{s=|r|..R} xi^r_s P^r_s(mu) e^{i r lambda}
  Eq. fourier_transform           xi^r(mu) = (1/I) sum_iota xi(lambda_iota, mu) e^{-i r lambda_iota},
                                  lambda_iota = 2 pi iota / I
  Eq. legendre_transform          xi^r_s = sum_j xi^r(mu_j) P^r_s(mu_j) w_j
Readings: r is the zonal (Fourier) wavenumber m, s the total degree n (the
text swaps the words "latitudinal"/"longitudinal"); fields are real, so
xi^{-m}_n = conj(xi^m_n) and only m >= 0 is stored (Sec. 3, after Eq.
legendre_transform); Im xi^0_n is forced to zero after every analysis.
iota runs over 0..I-1 (the same longitudes as 1..I modulo 2 pi).

Vector transforms follow from the Helmholtz decomposition of Sec. 2 (Eq.
helmholtz_theorem) written with U = u cos(phi), V = v cos(phi):
  U = (1/a) [ d chi/d lambda - (1 - mu^2) d psi/d mu ]
  V = (1/a) [ d psi/d lambda + (1 - mu^2) d chi/d mu ]
and, for a vector field with cos(phi)-scaled components (X, Y),
  div  = 1/(a (1 - mu^2)) [ dX/d lambda + (1 - mu^2) dY/d mu ]
  curl = 1/(a (1 - mu^2)) [ dY/d lambda - (1 - mu^2) dX/d mu ],
whose spectral coefficients follow by Gaussian quadrature after integrating the
mu-derivative by parts (the boundary terms vanish since X, Y are zero at the
poles):
  div^m_n  = (1/a) sum_j w_j/(1 - mu_j^2) [ i m X^m_j P^m_n(mu_j) - Y^m_j H^m_n(mu_j) ]
  curl^m_n = (1/a) sum_j w_j/(1 - mu_j^2) [ i m Y^m_j P^m_n(mu_j) + X^m_j H^m_n(mu_j) ]
"""
from __future__ import annotations

import numpy as np

from . import legendre, quadrature


def n_coeffs(R: int) -> int:
    return (R + 1) * (R + 2) // 2


def spec_mn(R: int):
    """(m, n) of each stored coefficient, m-major order (m = 0..R, n = m..R)."""
    m = np.concatenate([np.full(R + 1 - k, k) for k in range(R + 1)])
    n = np.concatenate([np.arange(k, R + 1) for k in range(R + 1)])
    return m, n


def m_slice(R: int, m: int) -> slice:
    start = m * (R + 1) - m * (m - 1) // 2
    return slice(start, start + R + 1 - m)


class Grid:
    """Gaussian grid I x J (longitude x latitude, north to south) with the
    Legendre tables of a triangular truncation R."""

    def __init__(self, R: int, I: int, J: int):
        self.R, self.I, self.J = R, I, J
        self.mu, self.w = quadrature.gauss_legendre(J)
        self.lam = 2.0 * np.pi * np.arange(I) / I
        P = legendre.assoc_legendre(R + 1, self.mu)
        self.H = legendre.legendre_H(R, P)
        self.P = P[: R + 1, : R + 1]
        self.nc = n_coeffs(R)
        self.m, self.n = spec_mn(R)
        m = np.arange(R + 1)
        self._e_fwd = np.exp(-1j * np.outer(self.lam, m))  # [I, R+1]
        self._e_inv = np.exp(1j * np.outer(m, self.lam))   # [R+1, I]

    # ---- longitude: Eq. fourier_transform and its inverse ----------------
    def fourier_analysis(self, f: np.ndarray) -> np.ndarray:
        """[..., J, I] real -> [..., J, R+1] complex: (1/I) sum_iota f e^{-i m lambda}."""
        return (f @ self._e_fwd) / self.I

    def fourier_synthesis(self, F: np.ndarray) -> np.ndarray:
        """[..., J, R+1] complex -> [..., J, I] real:
        f = Re F_0 + sum_{m>=1} (F_m e^{i m lambda} + conj(F_m) e^{-i m lambda})."""
        c = np.array(F, dtype=np.complex128, copy=True)
        c[..., 1:] *= 2.0
        c[..., 0] = c[..., 0].real
        return np.real(c @ self._e_inv)

    # ---- latitude: Eq. legendre_transform and its inverse ----------------
    def legendre_synthesis(self, spec: np.ndarray, table: np.ndarray) -> np.ndarray:
        """[..., N_c] -> [..., J, R+1]: F^m(mu_j) = sum_n spec^m_n table^m_n(mu_j)."""
        out = np.zeros(spec.shape[:-1] + (self.J, self.R + 1), dtype=np.complex128)
        for m in range(self.R + 1):
            sl = m_slice(self.R, m)
            out[..., :, m] = spec[..., sl] @ table[m, m:]
        return out

    def legendre_analysis(self, F: np.ndarray, table: np.ndarray, weight: np.ndarray) -> np.ndarray:
        """[..., J, R+1] -> [..., N_c]: spec^m_n = sum_j F^m(mu_j) table^m_n(mu_j) weight_j."""
        out = np.zeros(F.shape[:-2] + (self.nc,), dtype=np.complex128)
        for m in range(self.R + 1):
            sl = m_slice(self.R, m)
            out[..., sl] = (F[..., :, m] * weight) @ table[m, m:].T
        return out

    # ---- scalar transforms ------------------------------------------------
    def synthesis(self, spec: np.ndarray) -> np.ndarray:
        """Spectral -> grid, Eq. spectral_to_physical_space. [..., N_c] -> [..., J, I]."""
        return self.fourier_synthesis(self.legendre_synthesis(spec, self.P))

    def analysis(self, f: np.ndarray) -> np.ndarray:
        """Grid -> spectral, Eqs. fourier_transform then legendre_transform."""
        out = self.legendre_analysis(self.fourier_analysis(f), self.P, self.w)
        return zero_m0_imag(self, out)

    # ---- vector transforms (Helmholtz, Sec. 2) -------------------------------
    def vector_synthesis(self, psi: np.ndarray, chi: np.ndarray, a: float):
        """(psi, chi) spectral -> (U, V) = cos(phi) (u, v) on the grid."""
        im = 1j * self.m
        U_m = (self.legendre_synthesis(im * chi, self.P) - self.legendre_synthesis(psi, self.H)) / a
        V_m = (self.legendre_synthesis(im * psi, self.P) + self.legendre_synthesis(chi, self.H)) / a
        return self.fourier_synthesis(U_m), self.fourier_synthesis(V_m)

    def vector_analysis(self, X: np.ndarray, Y: np.ndarray, a: float):
        """Spectral divergence and curl of the vector field whose cos(phi)-scaled
        components are (X, Y) on the grid."""
        wt = self.w / (1.0 - self.mu ** 2)
        Xm = self.fourier_analysis(X)
        Ym = self.fourier_analysis(Y)
        im = 1j * self.m
        div = (im * self.legendre_analysis(Xm, self.P, wt) - self.legendre_analysis(Ym, self.H, wt)) / a
        curl = (im * self.legendre_analysis(Ym, self.P, wt) + self.legendre_analysis(Xm, self.H, wt)) / a
        return zero_m0_imag(self, div), zero_m0_imag(self, curl)

    def laplacian_eigenvalues(self, a: float) -> np.ndarray:
        """Y^m_n is an eigenfunction of the surface Laplacian: -n(n+1)/a^2."""
        return -self.n * (self.n + 1.0) / (a * a)


def zero_m0_imag(g: Grid, x: np.ndarray) -> np.ndarray:
    x = np.array(x, dtype=np.complex128, copy=True)
    x[..., : g.R + 1] = x[..., : g.R + 1].real
    return x


def norm2(R: int, x: np.ndarray) -> float:
    """Parseval norm ||xi||^2 = sum |xi^0_n|^2 + 2 sum_{m>=1} |xi^m_n|^2, equal
    to (1/I) sum_{iota, j} w_j f^2 of the synthesised field."""
    m, _ = spec_mn(R)
    wt = np.where(m == 0, 1.0, 2.0)
    return float(np.sum(wt * np.abs(x) ** 2))


def truncate(x: np.ndarray, R_from: int, R_to: int) -> np.ndarray:
    """Spatial restriction D^c_f (Sec. 4.3.3, Eq. space_restriction): keep the
    coefficients with n <= R_to."""
    out = np.zeros(x.shape[:-1] + (n_coeffs(R_to),), dtype=np.complex128)
    for m in range(R_to + 1):
        out[..., m_slice(R_to, m)] = x[..., m_slice(R_from, m)][..., : R_to + 1 - m]
    return out


def zero_pad(x: np.ndarray, R_from: int, R_to: int) -> np.ndarray:
    """Spatial interpolation (D^c_f)^T (Sec. 4.3.3): pad with zeros up to R_to."""
    out = np.zeros(x.shape[:-1] + (n_coeffs(R_to),), dtype=np.complex128)
    for m in range(R_from + 1):
        out[..., m_slice(R_to, m)][..., : R_from + 1 - m] = x[..., m_slice(R_from, m)]
    return out
