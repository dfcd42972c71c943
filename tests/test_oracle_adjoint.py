"""Pins of the oracle's tangent-linear and adjoint (oracle.adjoint).

- every transpose against its forward map (dot-product identity
  <y, T x> = <T^t y, x>, random x and y), so a transposed table, a dropped
  weight or a wrong sign of i m fails;
- F_E'(x) against central differences of F_E, exact for a quadratic map;
- the tangent-linear SDC / MLSDC steps against central differences of the
  nonlinear oracle steps;
- the adjoint steps against the full tangent-linear matrix, built column by
  column on a tiny truncation (brute force), and against the tangent-linear
  step by the dot-product identity at a larger one;
- the gradient of the misfit after several steps against central
  differences along 16 seeded directions (relative 1e-5, eps = 1e-6 |x|/|d|).
"""
import numpy as np
import pytest

from oracle import adjoint as ad
from oracle import sdc
from oracle.sht import Grid, spec_mn, zero_m0_imag
from oracle.swe import SWE, Params
from paper_1805_07923_gb300 import inputs

RNG = np.random.default_rng(7)


def _spec(R, shape=()):
    m, _ = spec_mn(R)
    x = RNG.standard_normal(shape + (len(m),)) + 1j * RNG.standard_normal(shape + (len(m),))
    x[..., m == 0] = x[..., m == 0].real
    return x


def _rel(a, b):
    return abs(a - b) / max(abs(a), abs(b), 1e-300)


def _nrm(x):
    return np.sqrt(ad.inner(x, x))


def _dot_err(y, Tx, Tty, x):
    """|<y, T x> - <T^t y, x>| relative to |y| |T x| (cancellation-proof scale)."""
    return abs(ad.inner(y, Tx) - ad.inner(Tty, x)) / (_nrm(y) * _nrm(Tx))


G = Grid(10, 32, 16)


def test_fourier_transposes():
    f = RNG.standard_normal((G.J, G.I))
    F = RNG.standard_normal((G.J, G.R + 1)) + 1j * RNG.standard_normal((G.J, G.R + 1))
    assert _dot_err(f, G.fourier_synthesis(F), ad.fourier_synthesis_t(G, f), F) < 1e-14
    assert _dot_err(F, G.fourier_analysis(f), ad.fourier_analysis_t(G, F), f) < 1e-14


def test_legendre_transposes():
    s = _spec(10)
    F = RNG.standard_normal((G.J, G.R + 1)) + 1j * RNG.standard_normal((G.J, G.R + 1))
    for table in (G.P, G.H):
        assert _dot_err(F, G.legendre_synthesis(s, table), ad.legendre_synthesis_t(G, F, table), s) < 1e-14
        wt = G.w / (1.0 - G.mu ** 2)
        assert _dot_err(s, G.legendre_analysis(F, table, wt), ad.legendre_analysis_t(G, s, table, wt), F) < 1e-14


def test_scalar_and_vector_transform_transposes():
    s1, s2 = _spec(10), _spec(10)
    f1, f2 = RNG.standard_normal((G.J, G.I)), RNG.standard_normal((G.J, G.I))
    assert _dot_err(f1, G.synthesis(s1), ad.synthesis_t(G, f1), s1) < 1e-14
    assert _dot_err(s1, G.analysis(f1), ad.analysis_t(G, s1), f1) < 1e-14
    a = 6.37122e6
    U, V = G.vector_synthesis(s1, s2, a)
    pb, cb = ad.vector_synthesis_t(G, f1, f2, a)
    assert _dot_err(np.stack([f1, f2]), np.stack([U, V]), np.stack([pb, cb]), np.stack([s1, s2])) < 1e-14
    d, c = G.vector_analysis(f1, f2, a)
    Xb, Yb = ad.vector_analysis_t(G, s1, s2, a)
    assert _dot_err(np.stack([s1, s2]), np.stack([d, c]), np.stack([Xb, Yb]), np.stack([f1, f2])) < 1e-14


def test_synthesis_transpose_is_weighted_analysis():
    """Closed form: S^t g = c_m I A(g / w), c_0 = 1, c_m = 2 (Sec. 3 weights)."""
    g = RNG.standard_normal((G.J, G.I))
    m, _ = spec_mn(10)
    ref = np.where(m == 0, 1.0, 2.0) * G.I * G.analysis(g / G.w[:, None])
    assert np.max(np.abs(ad.synthesis_t(G, g) - ref)) < 1e-12 * np.max(np.abs(ref))


SW = SWE(10, 32, 16, Params())


def test_explicit_rhs_tl_is_exact_central_difference():
    """F_E is quadratic in the state, so (F(x+d) - F(x-d)) / 2 = F_E'(x) d exactly."""
    x = inputs.initial_state(10)
    d = inputs.initial_state(10, seed=2000)
    fd = (SW.explicit_rhs(x + d) - SW.explicit_rhs(x - d)) / 2.0
    tl = ad.explicit_rhs_tl(SW, x, d)
    for f in range(3):
        assert np.linalg.norm(fd[f] - tl[f]) <= 1e-11 * np.linalg.norm(tl[f])


def test_explicit_rhs_adjoint_dot_product():
    x = inputs.initial_state(10)
    d = inputs.initial_state(10, seed=2001)
    lam = _spec(10, (3,)) * np.array([1e-3, 1e4, 1e4])[:, None]
    assert _dot_err(lam, ad.explicit_rhs_tl(SW, x, d), ad.explicit_rhs_ad(SW, x, lam), d) < 1e-14


def test_implicit_transposes():
    x, lam = _spec(10, (3,)), _spec(10, (3,))
    assert _dot_err(lam, SW.implicit_rhs(x), ad.implicit_rhs_t(SW, lam), x) < 1e-14
    alpha = 37.5
    assert _dot_err(lam, SW.implicit_solve(x, alpha), ad.implicit_solve_t(SW, lam, alpha), x) < 1e-14
    # residual of (I - alpha F_I^t) y = lam
    y = ad.implicit_solve_t(SW, lam, alpha)
    ay = alpha * ad.implicit_rhs_t(SW, y)
    r = y - ay - lam
    assert np.linalg.norm(r) <= 1e-15 * (np.linalg.norm(y) + np.linalg.norm(ay) + np.linalg.norm(lam))


def _levels(Rf=10, If=32, Jf=16, Rc=5, Ic=16, Jc=8, nf=5, ncn=3):
    return sdc.Level(SWE(Rf, If, Jf, Params()), nf), sdc.Level(SWE(Rc, Ic, Jc, Params()), ncn)


def test_sdc_step_tl_matches_central_difference():
    lev = sdc.Level(SW, 3)
    x = inputs.initial_state(10)
    d = inputs.initial_state(10, seed=2002)
    eps = 1e-4
    fd = (sdc.sdc_step(lev, x + eps * d, 600.0, 3) - sdc.sdc_step(lev, x - eps * d, 600.0, 3)) / (2 * eps)
    tl = ad.sdc_step_tl(lev, x, d, 600.0, 3)
    for f in range(3):
        assert np.linalg.norm(fd[f] - tl[f]) <= 1e-7 * np.linalg.norm(tl[f])


def test_mlsdc_step_tl_matches_central_difference():
    fine, coarse = _levels()
    x = inputs.initial_state(10)
    d = inputs.initial_state(10, seed=2003)
    eps = 1e-4
    fd = (sdc.mlsdc_step(fine, coarse, x + eps * d, 300.0, 2, 2)
          - sdc.mlsdc_step(fine, coarse, x - eps * d, 300.0, 2, 2)) / (2 * eps)
    tl = ad.mlsdc_step_tl(fine, coarse, x, d, 300.0, 2, 2)
    for f in range(3):
        assert np.linalg.norm(fd[f] - tl[f]) <= 1e-7 * np.linalg.norm(tl[f])


def _basis(R):
    """Unit vectors of the real degrees of freedom (Im of m = 0 excluded)."""
    m, _ = spec_mn(R)
    nc = len(m)
    out = []
    for f in range(3):
        for c in range(nc):
            for part in ((1.0,) if m[c] == 0 else (1.0, 1j)):
                e = np.zeros((3, nc), dtype=np.complex128)
                e[f, c] = part
                out.append(e)
    return out


def test_mlsdc_step_adjoint_equals_transposed_tangent_matrix():
    """Brute force on T4/T2: column k of the tangent-linear matrix is TL(e_k);
    the adjoint applied to e_l must give row l of that matrix."""
    fine, coarse = _levels(4, 16, 8, 2, 8, 4, 3, 2)
    x = inputs.initial_state(4)
    basis = _basis(4)
    cols = [ad.mlsdc_step_tl(fine, coarse, x, ek, 600.0, 2, 1) for ek in basis]
    Mtl = np.array([[ad.inner(el, c) for c in cols] for el in basis])          # [l, k]
    rows = [ad.mlsdc_step_ad(fine, coarse, x, 600.0, 2, 1, el) for el in basis]
    Mad = np.array([[ad.inner(r, ek) for ek in basis] for r in rows])           # [l, k]
    assert np.max(np.abs(Mtl - Mad)) <= 1e-12 * np.max(np.abs(Mtl))
    # and the matrix is far from symmetric, so the test would see a missing transpose
    assert np.max(np.abs(Mtl - Mtl.T)) > 1e-3 * np.max(np.abs(Mtl))


def test_sdc_step_adjoint_dot_product():
    lev = sdc.Level(SW, 5)
    x = inputs.initial_state(10)
    d = inputs.initial_state(10, seed=2004)
    lam = _spec(10, (3,)) * np.array([1e-2, 1e5, 1e5])[:, None]
    lam = zero_m0_imag(SW.grid, lam)
    assert _dot_err(lam, ad.sdc_step_tl(lev, x, d, 600.0, 4), ad.sdc_step_ad(lev, x, 600.0, 4, lam), d) < 1e-13


def test_mlsdc_step_adjoint_dot_product():
    fine, coarse = _levels()
    x = inputs.initial_state(10)
    d = inputs.initial_state(10, seed=2005)
    lam = zero_m0_imag(SW.grid, _spec(10, (3,)) * np.array([1e-2, 1e5, 1e5])[:, None])
    assert _dot_err(lam, ad.mlsdc_step_tl(fine, coarse, x, d, 300.0, 4, 2),
                    ad.mlsdc_step_ad(fine, coarse, x, 300.0, 4, 2, lam), d) < 1e-13


def test_misfit_gradient_is_exact():
    """J is quadratic in x: the central difference along any direction is exact."""
    x = inputs.initial_state(10)
    t = inputs.initial_state(10, seed=1806)[0]
    J, lam = ad.misfit(10, x, t)
    d = inputs.initial_state(10, seed=2006)
    fd = (ad.misfit(10, x + d, t)[0] - ad.misfit(10, x - d, t)[0]) / 2.0
    assert _rel(fd, ad.inner(lam, d)) < 1e-12


def test_gradient_matches_finite_differences_16_directions():
    """The paper's objective after 3 MLSDC(5,3) steps: FD along 16 seeded
    directions, eps = 1e-6 |x| / |d|, central; |FD - <g, d>| <= 1e-5 |<g, d>|."""
    fine, coarse = _levels()
    x = inputs.initial_state(10)
    target = inputs.initial_state(10, seed=1806)[0]
    args = (300.0, 3, 4, 2)
    J, g, _ = ad.gradient(fine, coarse, x, target, *args)
    nx = np.sqrt(ad.inner(x, x))
    for i in range(16):
        d = inputs.initial_state(10, seed=2000 + i)
        eps = 1e-6 * nx / np.sqrt(ad.inner(d, d))
        Jp = ad.objective(fine, coarse, x + eps * d, target, *args)
        Jm = ad.objective(fine, coarse, x - eps * d, target, *args)
        fd = (Jp - Jm) / (2 * eps)
        gd = ad.inner(g, d)
        assert abs(fd - gd) <= 1e-5 * abs(gd), (i, fd, gd)


def test_gradient_has_no_imaginary_zonal_mean_component():
    fine, coarse = _levels()
    x = inputs.initial_state(10)
    target = inputs.initial_state(10, seed=1806)[0]
    _, g, _ = ad.gradient(fine, coarse, x, target, 300.0, 2, 2, 1)
    m, _ = spec_mn(10)
    assert np.all(g[:, m == 0].imag == 0.0)
