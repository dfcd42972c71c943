"""Pins of the oracle's IMEX SDC sweep and two-level MLSDC (Sec. 4.2, Sec. 4.3,
Algorithm 1) against closed forms and exact solutions:
  - Dahlquist IMEX: sweeps converge to the collocation solution, which has
    the Lobatto IIIA order 2M;
  - linearised rotating shallow water on a tiny truncation: the exact
    solution by matrix exponential gives observed orders 4 for SDC(3,4) and 8
    for SDC(5,8) (Sec. 5 reports these orders);
  - MLSDC with an identical coarse level is SDC with (1 + n_c) sweeps per
    iteration (derived: tau vanishes, restriction is the identity);
  - MLSDC iterated to convergence reaches the fine collocation solution (the
    FAS property shown after Eq. tau_term_level_l+1);
  - MLSDC(5,3,N,1/2) on the linearised system: observed order near 4 for
    N = 4 and near 8 for N = 12 (the behaviour Sec. 5 reports);
  - the mean geopotential is conserved."""
import numpy as np
import pytest

from oracle import sdc, sht
from oracle.swe import SWE, Params
from paper_1805_07923_gb300 import inputs

scipy_linalg = pytest.importorskip("scipy.linalg")


class Dahlquist:
    def __init__(self, lam_i, lam_e):
        self.li, self.le = lam_i, lam_e

    def explicit_rhs(self, y):
        return self.le * y

    def implicit_rhs(self, y):
        return self.li * y

    def implicit_solve(self, b, alpha):
        return b / (1.0 - alpha * self.li)


@pytest.mark.parametrize("n_nodes", [3, 5])
def test_dahlquist_sweeps_reach_collocation(n_nodes):
    prob = Dahlquist(-1.0 + 0.5j, 0.3j)
    lev = sdc.Level(prob, n_nodes)
    dt = 0.4
    y0 = np.array([1.0 + 0j])
    Theta, FI, FE = sdc.spread(lev, y0)
    for _ in range(40):
        Theta, FI, FE = sdc.sweep(lev, dt, Theta, FI, FE)
    lam = prob.li + prob.le
    coll = np.linalg.solve(np.eye(n_nodes) - dt * lam * lev.Q, np.ones(n_nodes))
    assert np.max(np.abs(np.array([t[0] for t in Theta]) - coll)) < 1e-14


@pytest.mark.parametrize("n_nodes,order", [(3, 4), (5, 8)])
def test_collocation_order(n_nodes, order):
    lam = -1.0 + 2.0j
    lev = sdc.Level(Dahlquist(lam, 0.0), n_nodes)
    errs = []
    for dt in (0.2, 0.1):
        coll = np.linalg.solve(np.eye(n_nodes) - dt * lam * lev.Q, np.ones(n_nodes))[-1]
        errs.append(abs(coll - np.exp(lam * dt)))
    assert abs(np.log2(errs[0] / errs[1]) - (order + 1)) < 0.3   # local error dt^(2M+1)


class LinearSWE(SWE):
    """The rotating shallow-water system linearised about rest: F_E is
    quadratic in the state, so its antisymmetric part is exactly its linear
    (Coriolis) part."""

    def explicit_rhs(self, x):
        return (SWE.explicit_rhs(self, x) - SWE.explicit_rhs(self, -x)) / 2.0


def _real(x):
    return np.concatenate([x.real.ravel(), x.imag.ravel()])


def _cplx(v, nc):
    h = v.size // 2
    return (v[:h] + 1j * v[h:]).reshape(3, nc)


def _linear_operator(prob):
    nc = prob.nc
    n = 6 * nc
    A = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        x = _cplx(e, nc)
        A[:, k] = _real(prob.explicit_rhs(x) + prob.implicit_rhs(x))
    return A


@pytest.mark.parametrize("n_nodes,n_sweeps,order", [(3, 4, 4), (5, 8, 8)])
def test_sdc_order_on_linearised_swe(n_nodes, n_sweeps, order):
    R = 5
    prob = LinearSWE(R, 16, 8, Params())
    u0 = inputs.initial_state(R, seed=99, rms=(3e3, 1e-5, 1e-5))
    A = _linear_operator(prob)
    T = 7200.0
    exact = _cplx(scipy_linalg.expm(T * A) @ _real(u0), prob.nc)
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


def test_mlsdc_with_identical_levels_is_sdc():
    R = 10
    prob = SWE(R, 32, 16, Params())
    u0 = inputs.initial_state(R, seed=5)
    fine = sdc.Level(prob, 3)
    coarse = sdc.Level(prob, 3)
    dt = 900.0
    n_iter, n_c = 2, 2
    u_ml = sdc.mlsdc_step(fine, coarse, u0, dt, n_iter, n_c)
    u_sdc = sdc.sdc_step(fine, u0, dt, (1 + n_c) * n_iter)
    for k in range(3):
        assert np.max(np.abs(u_ml[k] - u_sdc[k])) < 1e-14 * np.max(np.abs(u_sdc[k])), k


def test_mlsdc_converges_to_fine_collocation_solution():
    Rf, Rc = 10, 5
    pf = SWE(Rf, 32, 16, Params())
    pc = SWE(Rc, 16, 8, Params())
    u0 = inputs.initial_state(Rf, seed=8)
    fine, coarse = sdc.Level(pf, 5), sdc.Level(pc, 3)
    dt = 600.0
    u_sdc = sdc.sdc_step(fine, u0, dt, 40)
    u_ml = sdc.mlsdc_step(fine, coarse, u0, dt, 25, 1)
    u_ml_few = sdc.mlsdc_step(fine, coarse, u0, dt, 2, 1)
    for k in range(3):
        scale = np.max(np.abs(u_sdc[k] - u0[k]))
        assert np.max(np.abs(u_ml[k] - u_sdc[k])) < 1e-11 * scale, k
    # and two iterations are not yet converged (the pin is not vacuous)
    assert np.max(np.abs(u_ml_few[2] - u_sdc[2])) > 1e-9 * np.max(np.abs(u_sdc[2] - u0[2]))


def test_mlsdc_fixed_point_is_not_moved():
    """Starting MLSDC from the fine collocation solution, one iteration changes nothing."""
    Rf, Rc = 8, 4
    pf = SWE(Rf, 26, 13, Params())
    pc = SWE(Rc, 14, 7, Params())
    u0 = inputs.initial_state(Rf, seed=12)
    fine, coarse = sdc.Level(pf, 5), sdc.Level(pc, 3)
    dt = 600.0
    Theta, FI, FE = sdc.spread(fine, u0)
    for _ in range(40):
        Theta, FI, FE = sdc.sweep(fine, dt, Theta, FI, FE)
    # one MLSDC iteration from these nodes (Algorithm 1 steps A-D)
    Th2, FI2, FE2 = _one_mlsdc_iteration(fine, coarse, dt, Theta, FI, FE)
    for m in range(5):
        for k in range(3):
            scale = np.max(np.abs(Theta[-1][k] - u0[k]))
            assert np.max(np.abs(Th2[m][k] - Theta[m][k])) < 1e-12 * scale


def _one_mlsdc_iteration(fine, coarse, dt, Theta, FI, FE):
    """Run mlsdc_step's iteration body on given fine nodes by seeding the
    oracle with a fake spread."""
    orig = sdc.spread

    def seeded(lev, u0):
        if lev is fine:
            return list(Theta), list(FI), list(FE)
        return orig(lev, u0)

    sdc.spread = seeded
    try:
        return sdc.mlsdc_step(fine, coarse, Theta[0], dt, 1, 1, return_nodes=True)
    finally:
        sdc.spread = orig


def test_mean_geopotential_conserved_over_steps():
    Rf, Rc = 10, 5
    pf, pc = SWE(Rf, 32, 16, Params()), SWE(Rc, 16, 8, Params())
    fine, coarse = sdc.Level(pf, 5), sdc.Level(pc, 3)
    u = inputs.initial_state(Rf, seed=2)
    u[0, 0] = 50.0
    for _ in range(3):
        u = sdc.mlsdc_step(fine, coarse, u, 600.0, 2, 1)
    assert abs(u[0, 0] - 50.0) < 1e-12 * 50.0
    assert abs(u[2, 0]) < 1e-20


@pytest.mark.parametrize("n_iter,lo,hi", [(4, 3.2, 4.6), (12, 7.4, 8.8)])
def test_mlsdc_order_with_spatial_coarsening(n_iter, lo, hi):
    """Sec. 5: MLSDC(5,3,4,1/2) converges at fourth order in the range of small
    time steps (spatial coarsening limits the coarse correction), and more
    iterations recover the eighth order of the fine collocation solution.  On
    the linearised rotating system, fine T6 and coarse T3 (spatial and
    temporal coarsening), against the exact solution by matrix exponential:
    4 iterations give an observed order near 4, 12 iterations near 8.  A
    wrong FAS term or transfer moves the fixed point away from the fine
    collocation solution and caps the second."""
    Rf, Rc = 6, 3
    pf = LinearSWE(Rf, 32, 16, Params())
    pc = LinearSWE(Rc, 16, 8, Params())
    u0 = inputs.initial_state(Rf, seed=99, rms=(3e3, 1e-5, 1e-5))
    A = _linear_operator(pf)
    T = 7200.0
    exact = _cplx(scipy_linalg.expm(T * A) @ _real(u0), pf.nc)
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
