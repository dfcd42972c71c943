"""Pins of the oracle's two-level PFASST (oracle/pfasst.py) against what the
iteration must reduce to:
  - one time slice is Algorithm 1's MLSDC step, bit for bit;
  - slice 0 of several is the MLSDC step from u0 (nothing flows backwards);
  - with enough iterations every slice reaches the serial sequence of fine
    collocation steps (each from the previous slice's end value), computed
    independently by single-level SDC with many sweeps, and so does serial
    MLSDC with the same iteration count;
  - the coarse pipeline speeds the iteration up: the last of four slices
    gains orders of magnitude between 2 and 8 iterations."""
import numpy as np
import pytest

from oracle import pfasst, sdc
from oracle.swe import SWE, Params
from paper_1805_07923_gb300 import inputs

RF, RC, DT, P = 10, 5, 600.0, 4


@pytest.fixture(scope="module")
def levels():
    return sdc.Level(SWE(RF, 32, 16, Params()), 3), sdc.Level(SWE(RC, 16, 8, Params()), 2)


@pytest.fixture(scope="module")
def collocation_sequence(levels):
    fine, _ = levels
    u, out = inputs.initial_state(RF), []
    for _ in range(P):
        u = sdc.sdc_step(fine, u, DT, 60)
        out.append(u)
    return out


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_one_slice_is_mlsdc(levels):
    fine, coarse = levels
    u0 = inputs.initial_state(RF, seed=7)
    for n_iter, n_c in ((1, 1), (3, 2)):
        a = pfasst.pfasst(fine, coarse, u0, DT, 1, n_iter, n_c)
        b = sdc.mlsdc_step(fine, coarse, u0, DT, n_iter, n_c)
        assert np.array_equal(a, b)


def test_first_slice_is_mlsdc(levels):
    fine, coarse = levels
    u0 = inputs.initial_state(RF)
    ends = pfasst.pfasst(fine, coarse, u0, DT, P, 3, 2, return_slices=True)
    assert np.array_equal(ends[0], sdc.mlsdc_step(fine, coarse, u0, DT, 3, 2))


def test_converges_to_serial_collocation(levels, collocation_sequence):
    fine, coarse = levels
    u0 = inputs.initial_state(RF)
    ends = pfasst.pfasst(fine, coarse, u0, DT, P, 16, 2, return_slices=True)
    for p in range(P):
        assert rel(ends[p], collocation_sequence[p]) < 1e-13, p
    # serial MLSDC with the same iteration count reaches the same values
    u = u0
    for p in range(P):
        u = sdc.mlsdc_step(fine, coarse, u, DT, 16, 2)
        assert rel(ends[p], u) < 1e-13, p


def test_coarse_pipeline_accelerates(levels, collocation_sequence):
    fine, coarse = levels
    u0 = inputs.initial_state(RF)
    err = {K: rel(pfasst.pfasst(fine, coarse, u0, DT, P, K, 2), collocation_sequence[-1]) for K in (2, 4, 8)}
    assert err[4] < 0.1 * err[2]
    assert err[8] < 1e-5


def test_identical_levels_one_iteration_is_serial_collocation(levels, collocation_sequence):
    """Coarse level = fine level (the FAS term vanishes) with converged coarse
    sweeps and no predictor: in one iteration the coarse pipeline passes each
    slice the exact end value of the slice before, so every slice ends on the
    serial collocation sequence.  Only the coarse initial value handed down
    the slices within the iteration can do this."""
    fine, _ = levels
    u0 = inputs.initial_state(RF)
    ends = pfasst.pfasst(fine, fine, u0, DT, P, 1, 60, return_slices=True, n_predictor_sweeps=0)
    for p in range(P):
        assert rel(ends[p], collocation_sequence[p]) < 1e-12, (p, rel(ends[p], collocation_sequence[p]))
