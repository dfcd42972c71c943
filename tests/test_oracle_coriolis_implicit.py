"""Pins of the oracle's implicit-Coriolis splitting (Sec. 4.1's F = F_I + F_E
with the Coriolis part L_F moved from F_E into F_I) against facts the
equations fix:
  - the closed-form L_F equals the linear part of the transform-method F_E
    (its antisymmetric part, since F_E is quadratic plus linear);
  - the split moves only L_F: F_I + F_E is the same function as before, and
    the new F_E = N has no linear part;
  - the coupled implicit solve satisfies x - alpha F_I(x) = b with F_I's
    Coriolis part evaluated by the transforms (independent of the closed
    form), and reduces to the per-coefficient solve when Omega = 0;
  - on the linearised rotating system, where everything is now implicit,
    SDC sweeps converge to the collocation solution of the full linear
    operator, SDC(3,4) and SDC(5,8) reach orders 4 and 8 against the matrix
    exponential, and MLSDC(5,3,N,1/2) with spatial coarsening keeps the
    orders of the explicit-Coriolis split."""
import numpy as np
import pytest

from oracle import sdc, sht
from oracle.swe import SWE, SWECoriolisImplicit, Params
from paper_1805_07923_gb300 import inputs
from test_oracle_sdc import _cplx, _linear_operator, _real

scipy_linalg = pytest.importorskip("scipy.linalg")

P0 = Params()


class LinearImplicit(SWECoriolisImplicit):
    """The implicit-Coriolis system linearised about rest: the new F_E (the
    nonlinear terms) has no linear part, so the linear problem is F_I alone."""

    def explicit_rhs(self, x):
        return (SWECoriolisImplicit.explicit_rhs(self, x) - SWECoriolisImplicit.explicit_rhs(self, -x)) / 2.0


def _linear_part(prob: SWE, x):
    return (prob.explicit_rhs(x) - prob.explicit_rhs(-x)) / 2.0


@pytest.mark.parametrize("R,I,J", [(10, 32, 16), (21, 64, 32)])
def test_closed_form_coriolis_is_the_transform_linear_part(R, I, J):
    s = SWECoriolisImplicit(R, I, J, P0)
    lin = _linear_part(SWE(R, I, J, P0), inputs.initial_state(R, seed=7))
    c = s.coriolis(inputs.initial_state(R, seed=7))
    assert np.max(np.abs(c[0])) == 0.0
    for f in (1, 2):
        assert np.max(np.abs(c[f] - lin[f])) < 1e-13 * np.max(np.abs(lin[f]))


def test_split_moves_only_the_coriolis_terms():
    R, I, J = 12, 40, 20
    s, full = SWECoriolisImplicit(R, I, J, P0), SWE(R, I, J, P0)
    x = inputs.initial_state(R, seed=11)
    before = full.explicit_rhs(x) + full.implicit_rhs(x)
    after = s.explicit_rhs(x) + s.implicit_rhs(x)
    for f in range(3):
        assert np.max(np.abs(after[f] - before[f])) < 1e-13 * np.max(np.abs(before[f]))
    # the new F_E is even in the state (quadratic): no linear part left
    assert np.array_equal(s.explicit_rhs(x), s.explicit_rhs(-x))
    # F_I gained L_F (up to the rounding of the sum)
    gained = s.implicit_rhs(x) - full.implicit_rhs(x)
    for f in (1, 2):
        assert np.max(np.abs(gained[f] - s.coriolis(x)[f])) < 1e-15 * np.max(np.abs(s.implicit_rhs(x)[f]))


@pytest.mark.parametrize("alpha", [30.0, 3.0e3, 3.0e5])
def test_coupled_solve_residual_against_transform_coriolis(alpha):
    R, I, J = 10, 32, 16
    s, full = SWECoriolisImplicit(R, I, J, P0), SWE(R, I, J, P0)
    b = inputs.initial_state(R, seed=21)
    x = s.implicit_solve(b, alpha)
    FI = full.implicit_rhs(x) + _linear_part(full, x)
    r = x - alpha * FI - b
    for f in range(3):
        scale = max(np.max(np.abs(b[f])), alpha * np.max(np.abs(FI[f])))
        assert np.max(np.abs(r[f])) < 1e-13 * scale, (f, np.max(np.abs(r[f])) / scale)
    # the m = 0 solution of a real right-hand side stays real
    assert np.max(np.abs(x[:, sht.m_slice(R, 0)].imag)) == 0.0


def test_solve_without_rotation_is_the_per_coefficient_solve():
    R, I, J = 10, 32, 16
    p = Params(omega=0.0)
    b = inputs.initial_state(R, seed=5)
    x = SWECoriolisImplicit(R, I, J, p).implicit_solve(b, 250.0)
    ref = SWE(R, I, J, p).implicit_solve(b, 250.0)
    for f in range(3):
        assert np.max(np.abs(x[f] - ref[f])) < 1e-14 * np.max(np.abs(ref[f]))


def test_fully_implicit_linear_sweeps_reach_collocation():
    """With F_E = 0 the sweeps are a fixed-point iteration for the collocation
    problem (Eq. collocation_problem) of u' = A u, A the matrix of F_I."""
    R = 5
    prob = LinearImplicit(R, 16, 8, P0)
    assert np.max(np.abs(prob.explicit_rhs(inputs.initial_state(R, seed=3)))) == 0.0
    lev = sdc.Level(prob, 3)
    u0 = inputs.initial_state(R, seed=99, rms=(3e3, 1e-5, 1e-5))
    A = _linear_operator(prob)
    dt = 1800.0
    n = lev.M + 1
    K = np.eye(n * A.shape[0]) - dt * np.kron(lev.Q, A)
    coll = np.linalg.solve(K, np.tile(_real(u0), n)).reshape(n, -1)
    Theta, FI, FE = sdc.spread(lev, u0)
    for _ in range(40):
        Theta, FI, FE = sdc.sweep(lev, dt, Theta, FI, FE)
    for m in range(n):
        ref = _cplx(coll[m], prob.nc)
        for f in range(3):
            assert np.max(np.abs(Theta[m][f] - ref[f])) < 1e-12 * np.max(np.abs(ref[f]))


@pytest.mark.parametrize("n_nodes,n_sweeps,order", [(3, 4, 4), (5, 8, 8)])
def test_sdc_order_with_implicit_coriolis(n_nodes, n_sweeps, order):
    R = 5
    prob = LinearImplicit(R, 16, 8, P0)
    u0 = inputs.initial_state(R, seed=99, rms=(3e3, 1e-5, 1e-5))
    T = 7200.0
    exact = _cplx(scipy_linalg.expm(T * _linear_operator(prob)) @ _real(u0), prob.nc)
    lev = sdc.Level(prob, n_nodes)
    errs = []
    for nsteps in ((1, 2) if order == 8 else (8, 16)):
        dt = T / nsteps
        u = u0.copy()
        for _ in range(nsteps):
            u = sdc.sdc_step(lev, u, dt, n_sweeps)
        errs.append(np.sqrt(sht.norm2(R, (u - exact)[0]) / sht.norm2(R, exact[0])))
    observed = np.log2(errs[0] / errs[1])
    assert errs[1] > 1e-14
    assert order - 0.6 < observed < order + 0.8, (errs, observed)


@pytest.mark.parametrize("n_iter,lo,hi", [(4, 3.3, 4.6), (12, 7.4, 8.8)])
def test_mlsdc_order_with_implicit_coriolis(n_iter, lo, hi):
    Rf, Rc = 6, 3
    pf = LinearImplicit(Rf, 32, 16, P0)
    pc = LinearImplicit(Rc, 16, 8, P0)
    u0 = inputs.initial_state(Rf, seed=99, rms=(3e3, 1e-5, 1e-5))
    T = 7200.0
    exact = _cplx(scipy_linalg.expm(T * _linear_operator(pf)) @ _real(u0), pf.nc)
    fine, coarse = sdc.Level(pf, 5), sdc.Level(pc, 3)
    errs = []
    for nsteps in (1, 2):
        dt = T / nsteps
        u = u0.copy()
        for _ in range(nsteps):
            u = sdc.mlsdc_step(fine, coarse, u, dt, n_iter, 1)
        errs.append(np.sqrt(sht.norm2(Rf, (u - exact)[0]) / sht.norm2(Rf, exact[0])))
    observed = np.log2(errs[0] / errs[1])
    assert errs[1] > 1e-14
    assert lo < observed < hi, (errs, observed)


def test_mean_geopotential_conserved_with_implicit_coriolis():
    """Phi'^0_0 has no tendency (div V has zero mean and delta^0_0 = 0; L_F
    and the coupled solve leave the n = 0 row alone): an MLSDC step keeps it."""
    R, Rc = 10, 5
    pf, pc = SWECoriolisImplicit(R, 32, 16, P0), SWECoriolisImplicit(Rc, 16, 8, P0)
    u = inputs.initial_state(R, seed=13)
    u[0, 0] = 55.0
    fine, coarse = sdc.Level(pf, 5), sdc.Level(pc, 3)
    for _ in range(3):
        u = sdc.mlsdc_step(fine, coarse, u, 600.0, 2, 2)
    assert abs(u[0, 0] - 55.0) <= 1e-13 * 55.0
    # delta^0_0 stays zero to the rounding of the dense per-m solve
    assert abs(u[2, 0]) <= 1e-15 * np.max(np.abs(u[2]))
