"""Tensor-core (tcgen05, TMA-fed) Legendre contractions: TF32 and split-BF16
(hi/lo, three products) against the float64 oracle per F_E evaluation, and
the run-level criterion on the headline workload: total-geopotential relative
L2 <= 1e-6 after 400 steps against the float64 GPU path (split-BF16; TF32
does not meet it and is reported only)."""
import numpy as np
import pytest
import torch

from oracle import sht as osht
from oracle.swe import SWE, Params
from paper_1805_07923_gb300 import inputs
from paper_1805_07923_gb300 import mlsdc as M

pytestmark = pytest.mark.gpu

TC = ["tf32", "bf16x3"]
# Per-evaluation bounds: the operand rounding of each mode (tf32: 2^-11,
# bf16 hi+lo: 2^-16 relative per product) times the cancellation of each
# tendency, with margin over the largest error measured on T21..T170.
PER_EVAL_TOL = {"tf32": (5e-3, 1e-1, 3e-1), "bf16x3": (2e-4, 5e-3, 2e-2)}
# Run-level bound on the total geopotential after 400 steps: the 1e-6 bar
# for split BF16.  TF32 (10-bit operand mantissas) fails that bar (about
# 5e-6 on GB300); its run is reported, never bounded by a looser number and
# never the headline variant.
RUN_TOL = {"bf16x3": 1e-6}

_or = {}


def oracle(R, I, J):
    if (R, I, J) not in _or:
        _or[(R, I, J)] = SWE(R, I, J, Params())
    return _or[(R, I, J)]


def rel_l2(R, got, ref):
    return float(np.sqrt(osht.norm2(R, got - ref) / max(osht.norm2(R, ref), 1e-300)))


@pytest.mark.parametrize("kernels", ["tc", "auto"])
@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("R,I,J", [(1, 16, 4), (13, 64, 22), (21, 64, 32), (45, 256, 70), (85, 256, 128),
                                   (170, 512, 256)])
def test_tensorcore_rhs_vs_oracle(prec, R, I, J, kernels):
    """kernels="tc": both Legendre stages on tcgen05; "auto": the plan's size
    rule (CUDA-core float32 kernels where they are faster)."""
    o = oracle(R, I, J)
    x = inputs.initial_state(R)
    plan = M.Plan(R, I, J, prec)
    plan.set_stage_kernels(kernels, kernels)
    FE = torch.full((3, o.nc), float("nan"), dtype=torch.complex128, device="cuda")
    M.swe_explicit_rhs(plan, M.swe_params(), torch.from_numpy(x).cuda(), FE)
    assert plan.device_error() == 0
    got = FE.cpu().numpy()
    ref = o.explicit_rhs(x)
    errs = [rel_l2(R, got[k], ref[k]) for k in range(3)]
    print(f"{prec} T{R}: per-field F_E rel L2 {errs}")
    assert np.all(np.isfinite(got))
    for k in range(3):
        assert errs[k] <= PER_EVAL_TOL[prec][k], (prec, k, errs[k])


def _run(prec, u0, steps):
    pf, pc = M.Plan(170, 512, 256, prec), M.Plan(85, 256, 128, prec)
    lf, lc = M.Level(pf, 5), M.Level(pc, 3)
    ml = M.MLSDC(lf, lc)
    x = torch.from_numpy(u0).cuda()
    for _ in range(steps):
        M.mlsdc_step(ml, x, 150.0, 4, 2, use_graph=True)
    torch.cuda.synchronize()
    assert pf.device_error() == 0 and pc.device_error() == 0
    return x.cpu().numpy()


@pytest.mark.parametrize("prec", TC)
def test_tensorcore_headline_run_total_geopotential(prec):
    u0 = inputs.initial_state(170)
    ref = _run("fp64", u0, 400)
    got = _run(prec, u0, 400)
    tot = ref[0].copy()
    tot[0] += np.sqrt(2.0) * 9.80616e4
    err = float(np.sqrt(osht.norm2(170, got[0] - ref[0]) / osht.norm2(170, tot)))
    print(f"{prec}: total Phi rel L2 after 400 steps = {err:.3e}; Phi' {rel_l2(170, got[0], ref[0]):.2e} "
          f"zeta {rel_l2(170, got[1], ref[1]):.2e} delta {rel_l2(170, got[2], ref[2]):.2e}")
    assert np.all(np.isfinite(got))
    if prec in RUN_TOL:
        assert err <= RUN_TOL[prec]


def test_bounded_wait_gives_up_and_context_survives():
    """Failure detection without a fault: one CTA waits on an mbarrier that
    nothing completes, with the tensor-core kernels' bounded wait and a 20 ms
    limit.  The wait must give up (code 2) within a bounded time, and the
    context must stay usable: a tensor-core F_E evaluation afterwards still
    matches the oracle and records no device error."""
    import time
    t0 = time.perf_counter()
    assert M.selftest_wait_timeout(20) == 2
    assert time.perf_counter() - t0 < 10.0
    R, I, J = 21, 64, 32
    o = oracle(R, I, J)
    x = inputs.initial_state(R)
    plan = M.Plan(R, I, J, "bf16x3")
    plan.set_stage_kernels("tc", "tc")
    FE = torch.empty((3, o.nc), dtype=torch.complex128, device="cuda")
    M.swe_explicit_rhs(plan, M.swe_params(), torch.from_numpy(x).cuda(), FE)
    assert plan.device_error() == 0
    got = FE.cpu().numpy()
    ref = o.explicit_rhs(x)
    for k in range(3):
        assert rel_l2(R, got[k], ref[k]) <= PER_EVAL_TOL["bf16x3"][k]
    with pytest.raises(M.MlsdcError):
        M.selftest_wait_timeout(0)
