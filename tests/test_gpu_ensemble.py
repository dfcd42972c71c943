"""Ensemble batching: members advanced in lockstep through batched kernels
(member index on the grid, member-major arrays; on the tensor-core path the
members form the GEMM's N dimension) must reproduce each member run alone.
Float64 and float32 batched kernels do each member's arithmetic in the same
order, so the results are bitwise equal; the tensor-core results are compared
within 1e-12 relative (the MMA columns are independent).  A launch with
several members also stores the analysis input latitude-contiguous (one
member: m-contiguous); T45 on 70 latitudes and T13 on 22 (35 and 11 per
hemisphere, not multiples of the tensor-core kernels' latitude groups) cover
the ragged tail, R = 1 on 16 x 4 the smallest legal plan."""
import numpy as np
import pytest
import torch

from paper_1805_07923_gb300 import inputs
from paper_1805_07923_gb300 import mlsdc as M

pytestmark = pytest.mark.gpu


def members_state(R, k, base_R=None):
    base = inputs.initial_state(base_R or R)
    return np.stack([inputs.perturbed_member(base, base_R or R, R, k0) for k0 in range(k)])


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16x3"])
@pytest.mark.parametrize("R,I,J,B", [(1, 16, 4, 3), (13, 64, 22, 4), (13, 64, 22, 9), (21, 64, 32, 5),
                                     (45, 256, 70, 3), (85, 256, 128, 17)])
def test_batched_rhs_equals_single(prec, R, I, J, B):
    x = members_state(R, B)
    pb = M.Plan(R, I, J, prec, max_members=B)
    p1 = M.Plan(R, I, J, prec)
    if prec in ("tf32", "bf16x3"):
        # compare the tensor-core kernels batched and single (the size rule
        # could pick different kernels for 1 and B members)
        for p in (pb, p1):
            p.set_stage_kernels("tc", "tc")
    prm = M.swe_params()
    xs = torch.from_numpy(x).cuda()
    FEb = torch.empty_like(xs)
    M.swe_explicit_rhs_batched(pb, prm, xs, FEb, B)
    got = FEb.cpu().numpy()
    for b in range(B):
        FE1 = torch.empty_like(xs[b])
        M.swe_explicit_rhs(p1, prm, xs[b].contiguous(), FE1)
        ref = FE1.cpu().numpy()
        if prec in ("fp64", "fp32"):
            assert np.array_equal(got[b], ref), (prec, b)
        else:
            assert rel(got[b], ref) <= 1e-12, (prec, b, rel(got[b], ref))
    assert pb.device_error() == 0


def test_batched_mlsdc_step_equals_single_fp64():
    Rf, Rc, B = 42, 21, 3
    x = members_state(Rf, B)
    pf, pc = M.Plan(Rf, 128, 64, "fp64", B), M.Plan(Rc, 64, 32, "fp64", B)
    ml = M.MLSDC(M.Level(pf, 5, members=B), M.Level(pc, 3, members=B))
    xs = torch.from_numpy(x).cuda()
    for _ in range(3):
        M.mlsdc_step(ml, xs, 300.0, 4, 2, use_graph=True)
    got = xs.cpu().numpy()
    qf, qc = M.Plan(Rf, 128, 64), M.Plan(Rc, 64, 32)
    m1 = M.MLSDC(M.Level(qf, 5), M.Level(qc, 3))
    for b in range(B):
        y = torch.from_numpy(x[b]).cuda()
        for _ in range(3):
            M.mlsdc_step(m1, y, 300.0, 4, 2, use_graph=False)
        assert np.array_equal(got[b], y.cpu().numpy()), b


def test_batched_sdc_step_equals_single_fp64():
    R, B = 21, 4
    x = members_state(R, B)
    pb = M.Plan(R, 64, 32, "fp64", B)
    lb = M.Level(pb, 3, members=B)
    xs = torch.from_numpy(x).cuda()
    M.sdc_step(lb, xs, 600.0, 4)
    l1 = M.Level(M.Plan(R, 64, 32), 3)
    for b in range(B):
        y = torch.from_numpy(x[b]).cuda()
        M.sdc_step(l1, y, 600.0, 4)
        assert np.array_equal(xs[b].cpu().numpy(), y.cpu().numpy()), b


def _group(Rf, If, Jf, Rc, Ic, Jc, B, prec):
    pf, pc = M.Plan(Rf, If, Jf, prec, B), M.Plan(Rc, Ic, Jc, prec, B)
    if prec in ("tf32", "bf16x3"):
        for p in (pf, pc):
            p.set_stage_kernels("tc", "tc")
    lf, lc = M.Level(pf, 5, members=B), M.Level(pc, 3, members=B)
    return M.MLSDC(lf, lc), (pf, pc, lf, lc)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_uneven_ensemble_in_one_graph_equals_members_alone(prec):
    """Groups T21/T10 (3 members), T42/T21 (2), T85/T42 (2) stepped together
    through one CUDA graph with one branch per group."""
    specs = [(21, 64, 32, 10, 32, 16, 3), (42, 128, 64, 21, 64, 32, 2), (85, 256, 128, 42, 128, 64, 2)]
    base = inputs.initial_state(85)
    groups, keep, states, init = [], [], [], []
    for (Rf, If, Jf, Rc, Ic, Jc, B) in specs:
        ml, k = _group(Rf, If, Jf, Rc, Ic, Jc, B, prec)
        groups.append(ml)
        keep.append(k)
        x = np.stack([inputs.perturbed_member(base, 85, Rf, j) for j in range(B)])
        init.append(x)
        states.append(torch.from_numpy(x).cuda())
    ens = M.Ensemble(groups)
    for _ in range(2):
        M.mlsdc_ensemble_step(ens, states, 300.0, 4, 2, use_graph=True)
    torch.cuda.synchronize()
    assert ens.launch_count() > 0
    for (Rf, If, Jf, Rc, Ic, Jc, B), x, s in zip(specs, init, states):
        ml1, k1 = _group(Rf, If, Jf, Rc, Ic, Jc, 1, prec)
        got = s.cpu().numpy()
        for b in range(B):
            y = torch.from_numpy(x[b][None]).cuda()
            for _ in range(2):
                M.mlsdc_step(ml1, y, 300.0, 4, 2, use_graph=False)
            ref = y.cpu().numpy()[0]
            if prec == "fp64":
                assert np.array_equal(got[b], ref), (Rf, b)
            else:
                assert rel(got[b], ref) <= 1e-12, (Rf, b, rel(got[b], ref))
        for p in k1[:2]:
            assert p.device_error() == 0


@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
def test_tensor_core_configs_agree(prec):
    """Every feasible tensor-core launch configuration (members per CTA, K
    stages, warp-specialised batched analysis) reproduces the single-member
    results to 1e-12.  T85 on 256 x 160 has two (bf16) or four (tf32) K blocks
    of latitudes per tile, so one-stage configurations refill their stage
    within a tile; 17 members leave a ragged last member chunk for every chunk
    size; the warp-specialised CTAs loop over several tiles each, alternating
    their two accumulator buffers."""
    R, I, J, B = 85, 256, 160, 17
    x = members_state(R, B)
    prm = M.swe_params()
    xs = torch.from_numpy(x).cuda()
    p1 = M.Plan(R, I, J, prec)
    p1.set_stage_kernels("tc", "tc")
    refs = []
    for b in range(B):
        FE1 = torch.empty_like(xs[b])
        M.swe_explicit_rhs(p1, prm, xs[b].contiguous(), FE1)
        refs.append(FE1.cpu().numpy())
    pb = M.Plan(R, I, J, prec, max_members=B)
    pb.set_stage_kernels("tc", "tc")
    tried = 0
    for cfg in [(1, 1, 0), (1, 2, 0), (2, 1, 0), (2, 2, 0), (4, 1, 0), (4, 2, 0), (8, 1, 0), (16, 1, 0),
                (1, 1, 1), (1, 2, 1), (2, 2, 1), (4, 1, 1), (4, 2, 1), (8, 1, 1)]:
        try:
            pb.set_tc_config(cfg[0], cfg[1], 0, stage="synthesis")
            pb.set_tc_config(*cfg, stage="analysis")
        except RuntimeError:
            continue  # shared memory of this choice does not fit a CTA
        assert pb.tc_config("analysis") == cfg and pb.tc_config("synthesis") == (cfg[0], cfg[1], 0)
        FEb = torch.full_like(xs, float("nan"))
        M.swe_explicit_rhs_batched(pb, prm, xs, FEb, B)
        got = FEb.cpu().numpy()
        assert pb.device_error() == 0, cfg
        for b in range(B):
            assert rel(got[b], refs[b]) <= 1e-12, (prec, cfg, b, rel(got[b], refs[b]))
        tried += 1
    assert tried >= 5
