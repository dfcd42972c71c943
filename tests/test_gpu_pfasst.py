"""Two-level PFASST on the GPU (pfasst_step, through the C ABI) against the
oracle's PFASST (oracle/pfasst.py), slice by slice: the time slices are the
members of batched levels, the fine sweeps, restriction, coarse evaluations,
FAS term and interpolation run batched, the coarse sweeps slice after slice.

Bars: float64 per slice and field <= 1e-12 (the per-step bar); one slice is
the GPU's own MLSDC step bit for bit; graph replay equals direct launches;
split BF16 at the headline sizes meets the total-geopotential bar against
the float64 GPU PFASST."""
import numpy as np
import pytest
import torch

from oracle import pfasst as opf
from oracle import sdc as osdc
from oracle import sht as osht
from oracle.swe import SWE, Params
from paper_1805_07923_gb300 import inputs
from paper_1805_07923_gb300 import mlsdc as M

pytestmark = pytest.mark.gpu


def rel_l2(R, got, ref):
    return float(np.sqrt(osht.norm2(R, got - ref) / osht.norm2(R, ref)))


def build(Rf, If, Jf, Rc, Ic, Jc, P, prec="fp64", nf=5, ncn=3):
    pf = M.Plan(Rf, If, Jf, prec, max_members=P)
    pc = M.Plan(Rc, Ic, Jc, prec, max_members=P * ncn)
    lf, lc = M.Level(pf, nf, members=P), M.Level(pc, ncn, members=P)
    return M.PFASST(lf, lc), (pf, pc, lf, lc)


def run(pf, u0, dt, n_iter, n_c, n_pred=-1, use_graph=False):
    x = torch.from_numpy(u0).cuda()
    ends = torch.full((pf.slices,) + tuple(x.shape), float("nan"), dtype=torch.complex128, device="cuda")
    M.pfasst_step(pf, x, ends, dt, n_iter, n_c, n_pred, use_graph)
    torch.cuda.synchronize()
    return ends.cpu().numpy()


@pytest.mark.parametrize("Rf,If,Jf,Rc,Ic,Jc,P,n_iter", [(21, 64, 32, 10, 32, 16, 4, 3), (85, 256, 128, 42, 128, 64, 3, 2)])
def test_pfasst_matches_oracle(Rf, If, Jf, Rc, Ic, Jc, P, n_iter):
    dt, n_c = 300.0, 2
    u0 = inputs.initial_state(Rf)
    pf, keep = build(Rf, If, Jf, Rc, Ic, Jc, P)
    got = run(pf, u0, dt, n_iter, n_c)
    fine = osdc.Level(SWE(Rf, If, Jf, Params()), 5)
    coarse = osdc.Level(SWE(Rc, Ic, Jc, Params()), 3)
    ref = opf.pfasst(fine, coarse, u0, dt, P, n_iter, n_c, return_slices=True)
    for p in range(P):
        for k in range(3):
            assert rel_l2(Rf, got[p][k], ref[p][k]) <= 1e-12, (p, k, rel_l2(Rf, got[p][k], ref[p][k]))
    assert pf.launch_count() > 0


def test_pfasst_with_a_small_coarse_plan_and_no_predictor_matches_oracle():
    """A coarse plan too small for every slice's coarse nodes in one launch
    (node-by-node evaluation) and no predictor sweeps."""
    Rf, Rc, P = 21, 10, 3
    u0 = inputs.initial_state(Rf, seed=9)
    pf_ = M.Plan(Rf, 64, 32, "fp64", max_members=P)
    pc_ = M.Plan(Rc, 32, 16, "fp64", max_members=P)
    pf = M.PFASST(M.Level(pf_, 3, members=P), M.Level(pc_, 2, members=P))
    got = run(pf, u0, 450.0, 3, 1, 0)
    fine = osdc.Level(SWE(Rf, 64, 32, Params()), 3)
    coarse = osdc.Level(SWE(Rc, 32, 16, Params()), 2)
    ref = opf.pfasst(fine, coarse, u0, 450.0, P, 3, 1, return_slices=True, n_predictor_sweeps=0)
    for p in range(P):
        for k in range(3):
            assert rel_l2(Rf, got[p][k], ref[p][k]) <= 1e-12, (p, k)


def test_one_slice_is_the_mlsdc_step():
    Rf, Rc = 42, 21
    u0 = inputs.initial_state(Rf)
    pf, keep = build(Rf, 128, 64, Rc, 64, 32, 1)
    got = run(pf, u0, 300.0, 4, 2)[0]
    ml = M.MLSDC(M.Level(M.Plan(Rf, 128, 64), 5), M.Level(M.Plan(Rc, 64, 32, "fp64", 3), 3))
    x = torch.from_numpy(u0).cuda()
    M.mlsdc_step(ml, x, 300.0, 4, 2)
    assert np.array_equal(got, x.cpu().numpy())


def test_graph_replay_equals_direct_launches():
    pf, keep = build(21, 64, 32, 10, 32, 16, 4)
    u0 = inputs.initial_state(21)
    a = run(pf, u0, 300.0, 3, 2)
    x = torch.from_numpy(u0).cuda()
    ends = torch.empty((4,) + tuple(x.shape), dtype=torch.complex128, device="cuda")
    for _ in range(2):  # capture, then replay
        M.pfasst_step(pf, x, ends, 300.0, 3, 2, -1, True)
    torch.cuda.synchronize()
    assert np.array_equal(a, ends.cpu().numpy())


def test_bf16x3_pfasst_at_the_headline_sizes_meets_the_bar():
    """Four slices of T170/T85, four iterations: split BF16 against float64."""
    u0 = inputs.initial_state(170)
    out = {}
    for prec in ("fp64", "bf16x3"):
        pf, keep = build(170, 512, 256, 85, 256, 128, 4, prec)
        out[prec] = run(pf, u0, 150.0, 4, 2, use_graph=True)
        assert keep[0].device_error() == 0 and keep[1].device_error() == 0
    for p in range(4):
        ref, got = out["fp64"][p], out["bf16x3"][p]
        tot = ref[0].copy()
        tot[0] += np.sqrt(2.0) * 9.80616e4
        err = float(np.sqrt(osht.norm2(170, got[0] - ref[0]) / osht.norm2(170, tot)))
        print(f"slice {p}: total Phi {err:.2e}, fields {[rel_l2(170, got[k], ref[k]) for k in range(3)]}")
        assert np.all(np.isfinite(got))
        assert err <= 1e-6
