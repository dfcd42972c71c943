"""Pins of the oracle's MLSDC on three or more space-time levels (the V-cycle
reading of Sec. 4.3 with the general FAS term of Eq. tau_term_level_l+1,
tau_{l+1} = A_{l+1}(R Theta_l) - R A_l(Theta_l) + R tau_l):
  - with two levels it is Algorithm 1 (mlsdc_step), bit for bit;
  - with three identical levels (same truncation and nodes) every tau is zero
    and restriction and interpolation copy, so one iteration is 2 + 2 n_c
    sweeps of single-level SDC (one fine sweep, n_c on each coarser level, one
    on the middle level going up): equal to SDC with that many sweeps;
  - iterated, it converges to the fine level's collocation solution on the
    linearised system (the FAS fixed point; dropping R tau_l moves it);
  - MLSDC(5,3,2,N,1/2,1/2) on the linearised system: observed order about 4
    for N = 4 and about 8 for N = 12 against the matrix exponential."""
import numpy as np
import pytest

from oracle import sdc, sht
from oracle.swe import SWE, Params
from paper_1805_07923_gb300 import inputs
from test_oracle_sdc import LinearSWE, _cplx, _linear_operator, _real

scipy_linalg = pytest.importorskip("scipy.linalg")


def _linear_levels():
    probs = [LinearSWE(8, 32, 16, Params()), LinearSWE(4, 16, 8, Params()), LinearSWE(2, 8, 4, Params())]
    return probs, [sdc.Level(probs[0], 5), sdc.Level(probs[1], 3), sdc.Level(probs[2], 2)]


def test_two_levels_are_algorithm_1():
    p, pc = SWE(10, 32, 16), SWE(5, 16, 8)
    u0 = inputs.initial_state(10, seed=5)
    f, c = sdc.Level(p, 5), sdc.Level(pc, 3)
    assert np.array_equal(sdc.mlsdc_step_levels([f, c], u0, 900.0, 2, 2), sdc.mlsdc_step(f, c, u0, 900.0, 2, 2))


@pytest.mark.parametrize("n_c", [1, 2])
def test_identical_levels_are_sdc(n_c):
    p = SWE(10, 32, 16)
    u0 = inputs.initial_state(10, seed=5)
    levs = [sdc.Level(p, 3) for _ in range(3)]
    a = sdc.mlsdc_step_levels(levs, u0, 900.0, 2, n_c)
    b = sdc.sdc_step(levs[0], u0, 900.0, (2 + 2 * n_c) * 2)
    for k in range(3):
        assert np.max(np.abs(a[k] - b[k])) <= 1e-14 * np.max(np.abs(b[k]))


def test_three_levels_reach_the_fine_collocation_solution():
    probs, levs = _linear_levels()
    u0 = inputs.initial_state(8, seed=99, rms=(3e3, 1e-5, 1e-5))
    A = _linear_operator(probs[0])
    dt, n = 1800.0, 5
    coll = np.linalg.solve(np.eye(n * A.shape[0]) - dt * np.kron(levs[0].Q, A), np.tile(_real(u0), n)).reshape(n, -1)
    Th, _, _ = sdc.mlsdc_step_levels(levs, u0, dt, 40, 1, return_nodes=True)
    for m in range(n):
        ref = _cplx(coll[m], probs[0].nc)
        for f in range(3):
            assert np.max(np.abs(Th[m][f] - ref[f])) <= 2e-12 * np.max(np.abs(ref[f])), (m, f)


@pytest.mark.parametrize("n_iter,lo,hi", [(4, 3.4, 4.7), (12, 7.2, 8.8)])
def test_three_level_order(n_iter, lo, hi):
    probs, levs = _linear_levels()
    u0 = inputs.initial_state(8, seed=99, rms=(3e3, 1e-5, 1e-5))
    T = 7200.0
    exact = _cplx(scipy_linalg.expm(T * _linear_operator(probs[0])) @ _real(u0), probs[0].nc)
    errs = []
    for nsteps in (2, 4):
        u = u0.copy()
        for _ in range(nsteps):
            u = sdc.mlsdc_step_levels(levs, u, T / nsteps, n_iter, 1)
        errs.append(np.sqrt(sht.norm2(8, (u - exact)[0]) / sht.norm2(8, exact[0])))
    observed = np.log2(errs[0] / errs[1])
    assert errs[1] > 1e-14
    assert lo < observed < hi, (errs, observed)
