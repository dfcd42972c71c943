"""MLSDC on three levels on the GPU (through the C ABI) against the oracle's
mlsdc_step_levels, and its reductions: with two levels the object gives
mlsdc_step's result bit for bit (the same operation list); with three
identical levels it equals single-level SDC with 2 + 2 n_c sweeps per
iteration (to rounding: the zero FAS terms and the copy-back go through the
transfer kernels).  Bar: relative L2 <= 1e-12 per field and step, float64."""
import numpy as np
import pytest
import torch

from oracle import sdc as osdc
from oracle import sht as osht
from oracle.swe import SWE, Params
from paper_1805_07923_gb300 import inputs
from paper_1805_07923_gb300 import mlsdc as M

pytestmark = pytest.mark.gpu


def rel_l2(R, got, ref):
    return float(np.sqrt(osht.norm2(R, got - ref) / max(osht.norm2(R, ref), 1e-300)))


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("sizes,nodes,dt,n_c", [
    (((42, 128, 64), (21, 64, 32), (10, 32, 16)), (5, 3, 2), 600.0, 1),
    (((85, 256, 128), (42, 128, 64), (21, 64, 32)), (5, 3, 3), 300.0, 2),
])
def test_three_level_step_matches_oracle(sizes, nodes, dt, n_c):
    R0 = sizes[0][0]
    olv = [osdc.Level(SWE(R, I, J, Params()), n) for (R, I, J), n in zip(sizes, nodes)]
    plans = [M.Plan(R, I, J, "fp64", max(1, n - 1)) for (R, I, J), n in zip(sizes, nodes)]
    levels = [M.Level(p, n) for p, n in zip(plans, nodes)]
    ml = M.MLSDCLevels(levels)
    x = dev(inputs.initial_state(R0))
    for step in range(2):
        u = host(x)
        M.mlsdc_levels_step(ml, x, dt, 3, n_c, use_graph=(step == 1))
        ref = osdc.mlsdc_step_levels(olv, u, dt, 3, n_c)
        got = host(x)
        for k in range(3):
            assert rel_l2(R0, got[k], ref[k]) <= 1e-12, (step, k, rel_l2(R0, got[k], ref[k]))
    assert ml.launch_count() > 0


def test_two_levels_equal_mlsdc_step():
    pf, pc = M.Plan(85, 256, 128), M.Plan(42, 128, 64, "fp64", 2)
    lf, lc = M.Level(pf, 5), M.Level(pc, 3)
    u = inputs.initial_state(85)
    a, b = dev(u), dev(u)
    ml2 = M.MLSDC(lf, lc)
    for _ in range(2):
        M.mlsdc_step(ml2, a, 300.0, 4, 2, use_graph=True)
    mlv = M.MLSDCLevels([lf, lc])
    for _ in range(2):
        M.mlsdc_levels_step(mlv, b, 300.0, 4, 2, use_graph=True)
    assert np.array_equal(host(a), host(b))


def test_identical_levels_equal_sdc():
    R = 42
    plans = [M.Plan(R, 128, 64) for _ in range(3)]
    levels = [M.Level(p, 3) for p in plans]
    ml = M.MLSDCLevels(levels)
    u = inputs.initial_state(R)
    a, b = dev(u), dev(u)
    M.mlsdc_levels_step(ml, a, 600.0, 2, 2)
    single = M.Level(M.Plan(R, 128, 64), 3)
    M.sdc_step(single, b, 600.0, (2 + 2 * 2) * 2)
    ga, gb = host(a), host(b)
    for k in range(3):
        assert rel_l2(R, ga[k], gb[k]) <= 1e-13


def test_levels_are_checked():
    p = M.Plan(21, 64, 32)
    lv = M.Level(p, 3)
    with pytest.raises(M.MlsdcError):
        M.MLSDCLevels([lv, lv])                       # a level twice
    with pytest.raises(M.MlsdcError):
        M.MLSDCLevels([M.Level(M.Plan(10, 32, 16), 3), lv])   # coarser first


def test_three_levels_with_implicit_coriolis_match_oracle():
    """The implicit-Coriolis splitting on every level of a three-level MLSDC
    (the factored chains prepared for each level before the step)."""
    from oracle.swe import SWECoriolisImplicit
    sizes, nodes, dt = ((42, 128, 64), (21, 64, 32), (10, 32, 16)), (5, 3, 2), 600.0
    olv = [osdc.Level(SWECoriolisImplicit(R, I, J, Params()), n) for (R, I, J), n in zip(sizes, nodes)]
    plans = [M.Plan(R, I, J, "fp64", max(1, n - 1)) for (R, I, J), n in zip(sizes, nodes)]
    levels = [M.Level(p, n, coriolis_implicit=True) for p, n in zip(plans, nodes)]
    ml = M.MLSDCLevels(levels)
    x = dev(inputs.initial_state(42))
    u = host(x)
    M.mlsdc_levels_step(ml, x, dt, 3, 1, use_graph=True)
    ref = osdc.mlsdc_step_levels(olv, u, dt, 3, 1)
    got = host(x)
    for k in range(3):
        assert rel_l2(42, got[k], ref[k]) <= 1e-12, (k, rel_l2(42, got[k], ref[k]))
