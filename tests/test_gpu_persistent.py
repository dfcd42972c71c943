"""The ensemble step as one persistent kernel launch (mlsdc_ensemble_step_persistent).

The persistent kernel runs the recorded launches of every group's step as
lockstep phases with a bounded grid barrier between them (or the dataflow
schedule), with the kernels' own device code, so its results must equal the
graph of per-stage launches up to the compiler's contraction choices: float64
to 1e-13 per field (measured 5e-16), split BF16 to 1e-6 (measured: identical
bit for bit); one member is also checked against the float64 oracle directly.  The barrier's bound is
exercised without any fault: a self-test barrier that never completes must
give up, report code 3, and leave the context usable.
"""
import time

import numpy as np
import pytest
import torch

from oracle import sdc as osdc
from oracle import sht as osht
from oracle.swe import SWE, Params
from paper_1805_07923_gb300 import inputs
from paper_1805_07923_gb300 import mlsdc as M

pytestmark = pytest.mark.gpu


def group(spec, prec, coriolis_implicit=False):
    Rf, If, Jf, Rc, Ic, Jc, B = spec
    pf, pc = M.Plan(Rf, If, Jf, prec, B), M.Plan(Rc, Ic, Jc, prec, B)
    lf = M.Level(pf, 5, members=B, coriolis_implicit=coriolis_implicit)
    lc = M.Level(pc, 3, members=B, coriolis_implicit=coriolis_implicit)
    return M.MLSDC(lf, lc), (pf, pc, lf, lc)


def ensemble_states(specs, base_R=170):
    base = inputs.initial_state(base_R)
    out, k0 = [], 0
    for spec in specs:
        R, B = spec[0], spec[-1]
        out.append(np.stack([inputs.perturbed_member(base, base_R, R, k0 + j) for j in range(B)]))
        k0 += B
    return out


def run(specs, prec, steps, persistent, dt=150.0, schedule="lockstep"):
    groups, keep = [], []
    for spec in specs:
        ml, k = group(spec, prec)
        groups.append(ml)
        keep.append(k)
    ens = M.Ensemble(groups)
    if persistent:
        ens.set_persistent_schedule(schedule)
    states = [torch.from_numpy(x).cuda() for x in ensemble_states(specs)]
    for _ in range(steps):
        if persistent:
            M.mlsdc_ensemble_step_persistent(ens, states, dt, 4, 2)
        else:
            M.mlsdc_ensemble_step(ens, states, dt, 4, 2, use_graph=True)
    torch.cuda.synchronize()
    for k in keep:
        assert k[0].device_error() == 0 and k[1].device_error() == 0
    info = ens.persistent_info() if persistent else None
    err = ens.device_error()
    launches = ens.launch_count()
    return [s.cpu().numpy() for s in states], info, err, launches


def test_grid_barrier_timeout_gives_up_and_context_survives():
    t0 = time.perf_counter()
    code = M.selftest_grid_barrier_timeout(20)
    dt = time.perf_counter() - t0
    assert code == 3
    assert dt < 1.5, dt
    # the context still runs kernels correctly
    plan = M.Plan(21, 64, 32)
    x = torch.from_numpy(inputs.initial_state(21)).cuda()
    fe = torch.empty_like(x)
    M.swe_explicit_rhs(plan, M.swe_params(), x, fe)
    torch.cuda.synchronize()
    assert torch.isfinite(fe).all()


SMALL = [(21, 64, 32, 10, 32, 16, 3), (42, 128, 64, 21, 64, 32, 2)]


def field_diffs(specs, a, b):
    out = []
    for spec, x, y in zip(specs, a, b):
        R = spec[0]
        for m in range(spec[-1]):
            out.append([float(np.sqrt(osht.norm2(R, y[m][k] - x[m][k]) / osht.norm2(R, x[m][k]))) for k in range(3)])
    return np.array(out)


@pytest.mark.parametrize("schedule", ["dataflow", "lockstep"])
def test_persistent_fp64_equals_graph(schedule):
    a, _, _, _ = run(SMALL, "fp64", 3, False)
    b, info, err, launches = run(SMALL, "fp64", 3, True, schedule=schedule)
    assert err == 0
    assert launches == 1
    assert info["phases"] > 100 and info["ctas"] >= 1
    d = field_diffs(SMALL, a, b)
    print(info, "max field difference", d.max(), "bitwise", all(np.array_equal(x, y) for x, y in zip(a, b)))
    assert d.max() <= 1e-13


def test_persistent_one_member_matches_oracle():
    spec = (42, 128, 64, 21, 64, 32, 2)
    got, _, err, _ = run([spec], "fp64", 1, True)
    assert err == 0
    x0 = ensemble_states([spec])[0]
    fine = osdc.Level(SWE(42, 128, 64, Params()), 5)
    coarse = osdc.Level(SWE(21, 64, 32, Params()), 3)
    for b in range(2):
        ref = osdc.mlsdc_step(fine, coarse, x0[b], 150.0, 4, 2)
        for k in range(3):
            e = float(np.sqrt(osht.norm2(42, got[0][b][k] - ref[k]) / osht.norm2(42, ref[k])))
            assert e <= 1e-12, (b, k, e)


# the ensemble's own group shapes (16 x T170/T85 runs both Legendre stages
# on tcgen05, the analysis warp-specialised) next to CUDA-core groups
MIXED = [(42, 128, 64, 21, 64, 32, 4), (85, 256, 128, 42, 128, 64, 4), (170, 512, 256, 85, 256, 128, 16)]


@pytest.mark.parametrize("schedule", ["dataflow", "lockstep"])
def test_persistent_bf16x3_equals_graph(schedule):
    a, _, _, _ = run(MIXED, "bf16x3", 2, False)
    b, info, err, _ = run(MIXED, "bf16x3", 2, True, schedule=schedule)
    assert err == 0
    for y in b:
        assert np.all(np.isfinite(y))
    d = field_diffs(MIXED, a, b)
    print(info, "max field difference", d.max(axis=0), "bitwise", all(np.array_equal(x, y) for x, y in zip(a, b)))
    assert d.max() <= 1e-6


def test_implicit_coriolis_group_is_refused():
    ml, keep = group((21, 64, 32, 10, 32, 16, 2), "fp64", coriolis_implicit=True)
    ens = M.Ensemble([ml])
    states = [torch.from_numpy(ensemble_states([(21, 64, 32, 10, 32, 16, 2)])[0]).cuda()]
    with pytest.raises(M.MlsdcError):
        M.mlsdc_ensemble_step_persistent(ens, states, 150.0, 4, 2)


def test_lockstep_phase_times_cover_every_phase():
    spec = (42, 128, 64, 21, 64, 32, 2)
    ml, keep = group(spec, "fp64")
    ens = M.Ensemble([ml])
    states = [torch.from_numpy(ensemble_states([spec])[0]).cuda()]
    M.mlsdc_ensemble_step_persistent(ens, states, 150.0, 4, 2)
    times = ens.persistent_phase_times()
    assert len(times) == ens.persistent_info()["phases"]
    assert all(us > 0 for _, us in times)
    assert {b for b, _ in times} >= {"SynthF64", "GridF64x1", "AnalF64", "SweepNode0_4", "SweepNodeS"}
