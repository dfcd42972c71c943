"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the method: it only draws reproducible
random spectral coefficients in the library's storage layout, and evaluates
the analytic Gaussian-dome initial condition at grid points the caller gives
(each side then analyses that grid field with its own transform).

Storage layout (the C-ABI layout): a spectral field of triangular truncation R
holds N_c = (R+1)(R+2)/2 complex coefficients xi^m_n, 0 <= m <= n <= R, stored
m-major (for m = 0..R: n = m..R), complex values interleaved (re, im) as
float64.  A state is [3][N_c] in the order (Phi', zeta, delta).

Random numbers come from a counter-based generator (SplitMix64 finaliser of a
key built from seed, stream, m, n and re/im part, then Box-Muller), so the
coefficient (m, n) of a field does not depend on the truncation it is drawn
at: a T85 draw is exactly the truncation of the T170 draw before scaling.
"""
from __future__ import annotations

import numpy as np

_MASK = np.uint64(0xFFFFFFFFFFFFFFFF)


def n_coeffs(R: int) -> int:
    """Number of stored complex coefficients per field at truncation R."""
    return (R + 1) * (R + 2) // 2


def sh_mn(R: int) -> tuple[np.ndarray, np.ndarray]:
    """(m, n) of every stored coefficient, in storage order."""
    m = np.concatenate([np.full(R + 1 - k, k, dtype=np.int64) for k in range(R + 1)])
    n = np.concatenate([np.arange(k, R + 1, dtype=np.int64) for k in range(R + 1)])
    return m, n


def _splitmix64(x: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _MASK
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _MASK
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _MASK
        return z ^ (z >> np.uint64(31))


def _uniform(seed: int, stream: int, m: np.ndarray, n: np.ndarray, part: int, draw: int) -> np.ndarray:
    """Uniform (0, 1) numbers keyed by (seed, stream, m, n, part, draw)."""
    key = (np.uint64(seed) * np.uint64(0x100000001B3)
           ^ (np.uint64(stream) << np.uint64(48))
           ^ (m.astype(np.uint64) << np.uint64(32))
           ^ (n.astype(np.uint64) << np.uint64(16))
           ^ (np.uint64(part) << np.uint64(8))
           ^ np.uint64(draw)) & _MASK
    bits = _splitmix64(_splitmix64(key))
    return ((bits >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def _normal(seed: int, stream: int, m: np.ndarray, n: np.ndarray, part: int) -> np.ndarray:
    u1 = _uniform(seed, stream, m, n, part, 0)
    u2 = _uniform(seed, stream, m, n, part, 1)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def spectrum(R: int, seed: int, stream: int, rms: float, slope: float = -1.5) -> np.ndarray:
    """One band-limited random field with coefficient amplitude ~ n**slope, n >= 1.

    Returns complex128[N_c]; the m = 0 coefficients are real, n = 0 is zero.
    The field is scaled so that its area-mean square equals rms**2, i.e.
    (|xi^0|^2 summed + 2 |xi^m|^2 summed over m >= 1) / 2 == rms**2.
    """
    m, n = sh_mn(R)
    amp = np.where(n >= 1, np.maximum(n, 1).astype(np.float64) ** slope, 0.0)
    g1 = _normal(seed, stream, m, n, 0)
    g2 = _normal(seed, stream, m, n, 1)
    c = np.where(m == 0, amp * g1 + 0j, amp * (g1 + 1j * g2) / np.sqrt(2.0))
    weight = np.where(m == 0, 1.0, 2.0)
    ms = float(np.sum(weight * np.abs(c) ** 2)) / 2.0
    return c * (rms / np.sqrt(ms)) if ms > 0 else c


DEFAULT_RMS = (1.0e2, 1.0e-5, 1.0e-6)  # Phi' [m^2/s^2], zeta [1/s], delta [1/s]


def initial_state(R: int, seed: int = 1805, rms=DEFAULT_RMS) -> np.ndarray:
    """Seeded n^-3/2 state (Phi', zeta, delta) as complex128[3, N_c]."""
    return np.stack([spectrum(R, seed, k, rms[k]) for k in range(3)])


def truncate(x: np.ndarray, R_from: int, R_to: int) -> np.ndarray:
    """Keep the coefficients with n <= R_to of an m-major field (last axis)."""
    m, n = sh_mn(R_from)
    keep = n <= R_to
    return np.ascontiguousarray(x[..., keep])


def perturbed_member(base: np.ndarray, R_base: int, R: int, k: int, rel: float = 0.01) -> np.ndarray:
    """Ensemble member k: the base state truncated to R plus a seeded
    n^-3/2 perturbation of rel x the base rms of each field."""
    xb = truncate(base, R_base, R)
    out = np.empty_like(xb)
    for f in range(3):
        weight = np.where(sh_mn(R)[0] == 0, 1.0, 2.0)
        rms = np.sqrt(np.sum(weight * np.abs(xb[f]) ** 2) / 2.0)
        out[f] = xb[f] + spectrum(R, 3000 + k, f, rel * rms)
    return np.ascontiguousarray(out)


def to_real(x: np.ndarray) -> np.ndarray:
    """complex128[..., N] -> float64[..., 2N] interleaved (re, im), the C-ABI layout."""
    return np.ascontiguousarray(x).view(np.float64)


def from_real(x: np.ndarray) -> np.ndarray:
    """float64[..., 2N] interleaved -> complex128[..., N]."""
    return np.ascontiguousarray(x).view(np.complex128)


# The Gaussian dome of the paper's unsteady test (Sec. 5, Eq. gaussian_bump):
# u = v = 0 and h = h_bar + A exp(-alpha (d / a)^2), with d the straight-line
# (chord) distance between the point and the centre (lambda_c, phi_c) =
# (pi, pi/4) for points on the sphere of radius a, h_bar = 29400 m, A = 6000 m.
# The paper does not give alpha; DOME_ALPHA is this library's choice.
DOME_H_BAR = 29400.0
DOME_A = 6000.0
DOME_ALPHA = 10.0
DOME_CENTRE = (np.pi, np.pi / 4.0)


def dome_chord(lam: np.ndarray, mu: np.ndarray, centre=DOME_CENTRE) -> np.ndarray:
    """d / a on the unit sphere for longitudes lam (radians) and mu = sin(phi),
    broadcast against each other: sqrt(x^2 + y^2 + z^2) with x, y, z the
    Cartesian differences to the centre."""
    lc, pc = centre
    cphi = np.sqrt(1.0 - mu * mu)
    x = np.cos(lam) * cphi - np.cos(lc) * np.cos(pc)
    y = np.sin(lam) * cphi - np.sin(lc) * np.cos(pc)
    z = mu - np.sin(pc)
    return np.sqrt(x * x + y * y + z * z)


def gaussian_dome_grid(lam: np.ndarray, mu: np.ndarray, g: float = 9.80616, alpha: float = DOME_ALPHA,
                       h_bar: float = DOME_H_BAR, amp: float = DOME_A) -> tuple[np.ndarray, float]:
    """The dome's geopotential deviation Phi' = g A exp(-alpha (d/a)^2) on the
    grid lam[None, :] x mu[:, None] ([J][I], latitudes as given), and the mean
    geopotential Phibar = g h_bar the model takes as a parameter.  The
    vorticity and divergence of the dome are zero (u = v = 0)."""
    d = dome_chord(np.asarray(lam)[None, :], np.asarray(mu)[:, None])
    return g * amp * np.exp(-alpha * d * d), g * h_bar
