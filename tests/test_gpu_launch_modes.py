"""Launch-mode variants of the MLSDC step give the results of the plain
schedule.

- Step B batching: with one member and a coarse plan sized for M_c states
  (max_members >= M_c), the F_I and F_E evaluations at the restricted coarse
  nodes 1..M_c run as one batched launch per stage (the nodes are the batch).
  The float64 and float32 kernels treat batch entries independently, so the
  step is bitwise the unbatched one; the tensor-core kernels pack the entries
  along N of one MMA (equal to 1e-12).  The batched float64 step also matches
  the oracle per step to 1e-12, and its adjoint the oracle's adjoint.
- Programmatic dependent launch (MLSDC_PDL=1), off by default, changes only
  how kernels start, never what they compute: bitwise equal.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from oracle import adjoint as oad
from oracle import sdc as osdc
from oracle import sht as osht
from oracle.swe import SWE, Params
from paper_1805_07923_gb300 import inputs
from paper_1805_07923_gb300 import mlsdc as M

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel_l2(R, got, ref):
    return float(np.sqrt(osht.norm2(R, got - ref) / max(osht.norm2(R, ref), 1e-300)))


def _mlsdc(Rf, If, Jf, Rc, Ic, Jc, prec, coarse_members):
    pf = M.Plan(Rf, If, Jf, prec)
    pc = M.Plan(Rc, Ic, Jc, prec, coarse_members)
    if prec in ("tf32", "bf16x3"):
        for p in (pf, pc):  # the tensor-core kernels themselves, batched and not
            p.set_stage_kernels("tc", "tc")
    lf, lc = M.Level(pf, 5), M.Level(pc, 3)
    return M.MLSDC(lf, lc), (pf, pc, lf, lc)


def _steps(prec, coarse_members, n=3, sizes=(85, 256, 128, 42, 128, 64), dt=300.0):
    ml, keep = _mlsdc(*sizes, prec, coarse_members)
    x = dev(inputs.initial_state(sizes[0]))
    for _ in range(n):
        M.mlsdc_step(ml, x, dt, 4, 2, use_graph=True)
    return host(x)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_step_b_batching_is_bitwise_for_simt_kernels(prec):
    a = _steps(prec, 1)
    b = _steps(prec, 2)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
def test_step_b_batching_tensor_core(prec):
    a = _steps(prec, 1, n=1)
    b = _steps(prec, 2, n=1)
    for f in range(3):
        assert rel_l2(85, b[f], a[f]) <= 1e-12


def test_step_b_batched_fp64_step_matches_oracle():
    ml, keep = _mlsdc(85, 256, 128, 42, 128, 64, "fp64", 2)
    of = osdc.Level(SWE(85, 256, 128, Params()), 5)
    oc = osdc.Level(SWE(42, 128, 64, Params()), 3)
    u = inputs.initial_state(85)
    x = dev(u)
    M.mlsdc_step(ml, x, 300.0, 4, 2, use_graph=True)
    ref = osdc.mlsdc_step(of, oc, u, 300.0, 4, 2)
    got = host(x)
    for f in range(3):
        assert rel_l2(85, got[f], ref[f]) <= 1e-12


def test_step_b_batched_adjoint_matches_oracle():
    ml, keep = _mlsdc(21, 64, 32, 10, 32, 16, "fp64", 2)
    adj = M.Adjoint(ml, 2, 1, 600.0, 3, 2)
    x = inputs.initial_state(21)
    xT = torch.empty((3, keep[0].nc), dtype=torch.complex128, device="cuda")
    adj.forward(dev(x), xT)
    m, _ = osht.spec_mn(21)
    rng = np.random.default_rng(5)
    lam = (rng.standard_normal((3, len(m))) + 1j * rng.standard_normal((3, len(m)))) * np.array([1e-2, 1e5, 1e5])[:, None]
    lam[:, m == 0] = lam[:, m == 0].real
    g = torch.empty_like(xT)
    adj.backward(dev(lam), g)
    fine = osdc.Level(SWE(21, 64, 32, Params()), 5)
    coarse = osdc.Level(SWE(10, 32, 16, Params()), 3)
    x1 = osdc.mlsdc_step(fine, coarse, x, 600.0, 3, 2)
    ref = oad.mlsdc_step_ad(fine, coarse, x, 600.0, 3, 2, oad.mlsdc_step_ad(fine, coarse, x1, 600.0, 3, 2, lam))
    got = host(g)
    for f in range(3):
        assert rel_l2(21, got[f], ref[f]) <= 1e-11


_CHILD = r"""
import sys, json, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1805_07923_gb300 import inputs
from paper_1805_07923_gb300 import mlsdc as M
out = {}
for prec in ("fp64", "bf16x3"):
    pf, pc = M.Plan(85, 256, 128, prec), M.Plan(42, 128, 64, prec, 2)
    ml = M.MLSDC(M.Level(pf, 5), M.Level(pc, 3))
    x = torch.from_numpy(inputs.initial_state(85)).cuda()
    for _ in range(3):
        M.mlsdc_step(ml, x, 300.0, 4, 2, use_graph=True)
    torch.cuda.synchronize()
    out[prec] = x.cpu().numpy().view(np.float64).tolist()
# three ensemble members in lockstep (member-batched kernels)
pf, pc = M.Plan(42, 128, 64, "fp32", 3), M.Plan(21, 64, 32, "fp32", 3)
ml = M.MLSDC(M.Level(pf, 5, members=3), M.Level(pc, 3, members=3))
base = inputs.initial_state(42)
x = torch.from_numpy(np.stack([inputs.perturbed_member(base, 42, 42, k) for k in range(3)])).cuda()
for _ in range(2):
    M.mlsdc_step(ml, x, 300.0, 3, 2, use_graph=False)
torch.cuda.synchronize()
out["ens_fp32"] = x.cpu().numpy().view(np.float64).tolist()
print(json.dumps(out))
"""


def test_launch_modes_do_not_change_results():
    """Programmatic dependent launch (MLSDC_PDL=1) changes only how the same
    arithmetic is launched: results are bitwise equal."""
    res = {}
    for name, env_add in (("default", {}), ("pdl", {"MLSDC_PDL": "1"})):
        env = dict(os.environ, **env_add)
        r = subprocess.run([sys.executable, "-c", _CHILD, ROOT], env=env, capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        res[name] = json.loads(r.stdout.strip().splitlines()[-1])
    for name in ("pdl",):
        for key in ("fp64", "bf16x3", "ens_fp32"):
            assert np.array_equal(np.array(res[name][key]), np.array(res["default"][key])), (name, key)
