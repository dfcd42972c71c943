"""Mixed-precision path (float32 Legendre sums and FFTs, float64 state and
implicit solve) against the float64 oracle and the float64 GPU path.

Bars: per F_E evaluation, relative L2 per field within a bound derived from
float32 rounding (u = 6e-8) times the cancellation of each tendency (the
vorticity and divergence tendencies cancel to ~1e-2 of their parts); per run,
the acceptance criterion: relative L2 of the total geopotential Phibar + Phi'
<= 1e-6 after the 400-step headline run, against the float64 path (itself
parity-pinned to the oracle per step at 1e-12)."""
import numpy as np
import pytest
import torch

from oracle import sht as osht
from oracle.swe import SWE, Params
from paper_1805_07923_gb300 import inputs
from paper_1805_07923_gb300 import mlsdc as M

pytestmark = pytest.mark.gpu

MP = ["fp32"]
# Per-evaluation bounds: float32 rounding u = 6e-8 times the cancellation of
# each tendency, with a factor 3 margin over the largest error measured on
# T21..T170 (Phi' 5e-7, zeta 2e-5, delta 8.5e-5).  The acceptance criterion
# of the mixed-precision path is the run-level total-Phi bound below.
PER_EVAL_TOL = {"fp32": (2e-6, 6e-5, 3e-4)}

_or = {}


def oracle(R, I, J):
    if (R, I, J) not in _or:
        _or[(R, I, J)] = SWE(R, I, J, Params())
    return _or[(R, I, J)]


def rel_l2(R, got, ref):
    return float(np.sqrt(osht.norm2(R, got - ref) / max(osht.norm2(R, ref), 1e-300)))


def total_phi_rel(R, got, ref, phibar=9.80616e4):
    tot = ref[0].copy()
    tot[0] += np.sqrt(2.0) * phibar
    return float(np.sqrt(osht.norm2(R, got[0] - ref[0]) / osht.norm2(R, tot)))


@pytest.mark.parametrize("prec", MP)
@pytest.mark.parametrize("R,I,J", [(1, 16, 4), (13, 64, 22), (21, 64, 32), (45, 256, 70), (85, 256, 128),
                                   (170, 512, 256)])
def test_mixed_explicit_rhs_vs_oracle(prec, R, I, J):
    o = oracle(R, I, J)
    x = inputs.initial_state(R)
    plan = M.Plan(R, I, J, prec)
    FE = torch.empty((3, o.nc), dtype=torch.complex128, device="cuda")
    M.swe_explicit_rhs(plan, M.swe_params(), torch.from_numpy(x).cuda(), FE)
    torch.cuda.synchronize()
    got = FE.cpu().numpy()
    ref = o.explicit_rhs(x)
    for k in range(3):
        err = rel_l2(R, got[k], ref[k])
        assert err <= PER_EVAL_TOL[prec][k], (prec, k, err)


def _run(prec, u0, steps, Rf=170, Rc=85):
    pf, pc = M.Plan(Rf, 512, 256, prec), M.Plan(Rc, 256, 128, prec)
    lf, lc = M.Level(pf, 5), M.Level(pc, 3)
    ml = M.MLSDC(lf, lc)
    x = torch.from_numpy(u0).cuda()
    for _ in range(steps):
        M.mlsdc_step(ml, x, 150.0, 4, 2, use_graph=True)
    torch.cuda.synchronize()
    return x.cpu().numpy()


@pytest.mark.parametrize("prec", MP)
def test_mixed_headline_run_total_geopotential(prec):
    u0 = inputs.initial_state(170)
    ref = _run("fp64", u0, 400)
    got = _run(prec, u0, 400)
    err = total_phi_rel(170, got, ref)
    print(f"{prec}: total Phi rel L2 after 400 steps = {err:.3e}; "
          f"Phi' {rel_l2(170, got[0], ref[0]):.2e} zeta {rel_l2(170, got[1], ref[1]):.2e} "
          f"delta {rel_l2(170, got[2], ref[2]):.2e}")
    assert np.all(np.isfinite(got))
    assert err <= 1e-6
