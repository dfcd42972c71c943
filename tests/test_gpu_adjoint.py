"""The CUDA adjoint (float64, through the C ABI) against the oracle's adjoint
and against finite differences of the CUDA forward path.

- F_E'(x)^t: dot-product identity with the exact central difference of the
  quadratic F_E (GPU forward), and equality with the oracle's transpose, at
  sizes with ragged work items (T45 on 256 x 70) and the T85 / T170 grids;
- one MLSDC step's adjoint equals the oracle's (Algorithm 1 reversed);
- the gradient of J = 1/2 ||Phi'(T) - Phi_t||^2 after 48 steps of
  MLSDC(5,3) T85/T42 at dt 300 s with a checkpoint every 8 steps equals the
  oracle's (tests/golden/adjoint_T85_T42_48.npz, written by
  make_adjoint_reference.py from the oracle alone) to 1e-10, and matches
  central differences of the GPU objective along 16 seeded directions to
  1e-5 (eps = 1e-6 |x| / |d|);
- the result does not depend on the checkpoint interval or on graph replay;
- torch.autograd through MLSDCFunction gives the same gradient.
"""
import os

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

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "adjoint_T85_T42_48.npz")
CFG4 = dict(dt=300.0, n_steps=48, every=8, n_iter=4, n_c=2)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def inner(a, b):
    return float(np.sum(np.real(np.conj(a) * b)))


def rel_l2(R, got, ref):
    return float(np.sqrt(osht.norm2(R, got - ref) / max(osht.norm2(R, ref), 1e-300)))


def rand_lam(R, seed, scale=(1e-2, 1e5, 1e5)):
    m, _ = osht.spec_mn(R)
    rng = np.random.default_rng(seed)
    lam = rng.standard_normal((3, len(m))) + 1j * rng.standard_normal((3, len(m)))
    lam[:, m == 0] = lam[:, m == 0].real
    return lam * np.array(scale)[:, None]


@pytest.mark.parametrize("R,I,J", [(21, 64, 32), (45, 256, 70), (85, 256, 128), (170, 512, 256)])
def test_fe_adjoint_dot_product_and_oracle(R, I, J):
    plan = M.Plan(R, I, J)
    prm = M.swe_params()
    x = inputs.initial_state(R)
    d = inputs.initial_state(R, seed=2000)
    lam = rand_lam(R, 11)
    # GPU forward: (F(x+d) - F(x-d)) / 2 = F_E'(x) d exactly (F_E is quadratic)
    Fp, Fm = torch.empty((3, plan.nc), dtype=torch.complex128, device="cuda"), \
        torch.empty((3, plan.nc), dtype=torch.complex128, device="cuda")
    M.swe_explicit_rhs(plan, prm, dev(x + d), Fp)
    M.swe_explicit_rhs(plan, prm, dev(x - d), Fm)
    tl = (host(Fp) - host(Fm)) / 2.0
    xb = torch.zeros((3, plan.nc), dtype=torch.complex128, device="cuda")
    lt = dev(lam)
    M.swe_explicit_rhs_adjoint(plan, prm, dev(x), lt, xb)
    got = host(xb)
    assert np.all(host(lt) == 0)                     # the output adjoint is consumed
    err = abs(inner(lam, tl) - inner(got, d)) / (np.sqrt(inner(lam, lam)) * np.sqrt(inner(tl, tl)))
    assert err < 1e-12, err
    ref = oad.explicit_rhs_ad(SWE(R, I, J, Params()), x, lam)
    for f in range(3):
        assert rel_l2(R, got[f], ref[f]) <= 1e-12, (f, rel_l2(R, got[f], ref[f]))


def test_fe_adjoint_accumulates():
    plan = M.Plan(21, 64, 32)
    prm = M.swe_params()
    x = inputs.initial_state(21)
    lam = rand_lam(21, 12)
    base = rand_lam(21, 13)
    xb = dev(base)
    M.swe_explicit_rhs_adjoint(plan, prm, dev(x), dev(lam), xb)
    xb0 = torch.zeros_like(xb)
    M.swe_explicit_rhs_adjoint(plan, prm, dev(x), dev(lam), xb0)
    assert np.allclose(host(xb), base + host(xb0), rtol=0, atol=1e-12 * np.max(np.abs(host(xb0))))


def _mlsdc(Rf, If, Jf, Rc, Ic, Jc, nf=5, ncn=3):
    pf, pc = M.Plan(Rf, If, Jf), M.Plan(Rc, Ic, Jc)
    lf, lc = M.Level(pf, nf), M.Level(pc, ncn)
    return M.MLSDC(lf, lc), (pf, pc, lf, lc)


def test_adjoint_forward_equals_mlsdc_step():
    ml, keep = _mlsdc(42, 128, 64, 21, 64, 32)
    adj = M.Adjoint(ml, 5, 2, 300.0, 4, 2)
    x0 = dev(inputs.initial_state(42))
    xT = torch.empty_like(x0)
    adj.forward(x0, xT)
    y = x0.clone()
    for _ in range(5):
        M.mlsdc_step(ml, y, 300.0, 4, 2, use_graph=True)
    torch.cuda.synchronize()
    assert torch.equal(xT, y)


@pytest.mark.parametrize("sizes,n_iter,n_c", [((21, 64, 32, 10, 32, 16), 2, 1), ((85, 256, 128, 42, 128, 64), 4, 2)])
def test_one_step_adjoint_matches_oracle(sizes, n_iter, n_c):
    Rf, If, Jf, Rc, Ic, Jc = sizes
    ml, keep = _mlsdc(*sizes)
    adj = M.Adjoint(ml, 1, 1, 300.0, n_iter, n_c)
    x = inputs.initial_state(Rf)
    xT = torch.empty((3, keep[0].nc), dtype=torch.complex128, device="cuda")
    adj.forward(dev(x), xT)
    lam = rand_lam(Rf, 21)
    g = torch.empty_like(xT)
    adj.backward(dev(lam), g)
    got = host(g)
    fine = osdc.Level(SWE(Rf, If, Jf, Params()), 5)
    coarse = osdc.Level(SWE(Rc, Ic, Jc, Params()), 3)
    ref = oad.mlsdc_step_ad(fine, coarse, x, 300.0, n_iter, n_c, lam)
    for f in range(3):
        assert rel_l2(Rf, got[f], ref[f]) <= 1e-11, (f, rel_l2(Rf, got[f], ref[f]))


@pytest.fixture(scope="module")
def cfg4():
    ml, keep = _mlsdc(85, 256, 128, 42, 128, 64)
    x0 = inputs.initial_state(85, seed=1805)
    target = inputs.initial_state(85, seed=1806)[0]
    return ml, keep, x0, target


def _gradient(ml, keep, x0, target, every=8, use_graph=True):
    c = CFG4
    plan = keep[0]
    adj = M.Adjoint(ml, c["n_steps"], every, c["dt"], c["n_iter"], c["n_c"], use_graph=use_graph)
    xT = torch.empty((3, plan.nc), dtype=torch.complex128, device="cuda")
    adj.forward(dev(x0), xT)
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    lam = torch.empty_like(xT)
    M.mlsdc_phi_misfit(plan, xT, dev(target), J, lam)
    g = torch.empty_like(xT)
    adj.backward(lam, g)
    return float(host(J)[0]), host(g), host(xT)


def _objective(ml, keep, x, target):
    c = CFG4
    plan = keep[0]
    y = dev(x)
    for _ in range(c["n_steps"]):
        M.mlsdc_step(ml, y, c["dt"], c["n_iter"], c["n_c"], use_graph=True)
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    lam = torch.empty_like(y)
    M.mlsdc_phi_misfit(plan, y, dev(target), J, lam)
    return float(host(J)[0])


def test_gradient_matches_oracle_golden(cfg4):
    ml, keep, x0, target = cfg4
    J, g, xT = _gradient(ml, keep, x0, target)
    ref = np.load(GOLDEN)
    assert abs(J - float(ref["J"])) <= 1e-11 * abs(float(ref["J"]))
    errs = [rel_l2(85, g[f], ref["grad"][f]) for f in range(3)]
    print(f"cfg4 gradient vs oracle: J rel {abs(J / float(ref['J']) - 1):.2e}, fields {errs}")
    assert max(errs) <= 1e-10
    m, _ = osht.spec_mn(85)
    assert np.all(g[:, m == 0].imag == 0.0)


def test_gradient_matches_finite_differences_16_directions(cfg4):
    ml, keep, x0, target = cfg4
    _, g, _ = _gradient(ml, keep, x0, target)
    nx = np.sqrt(inner(x0, x0))
    worst = 0.0
    for i in range(16):
        d = inputs.initial_state(85, seed=2000 + i)
        eps = 1e-6 * nx / np.sqrt(inner(d, d))
        fd = (_objective(ml, keep, x0 + eps * d, target) - _objective(ml, keep, x0 - eps * d, target)) / (2 * eps)
        gd = inner(g, d)
        worst = max(worst, abs(fd - gd) / abs(gd))
        assert abs(fd - gd) <= 1e-5 * abs(gd), (i, fd, gd)
    print(f"cfg4 FD check, 16 directions: worst relative error {worst:.2e}")


def test_gradient_independent_of_checkpoint_interval_and_graphs(cfg4):
    ml, keep, x0, target = cfg4
    J8, g8, _ = _gradient(ml, keep, x0, target, every=8)
    for every, graph in ((1, True), (48, True), (5, False)):
        J, g, _ = _gradient(ml, keep, x0, target, every=every, use_graph=graph)
        assert J == J8 and np.array_equal(g, g8), (every, graph)


def test_autograd_function_gives_the_same_gradient(cfg4):
    ml, keep, x0, target = cfg4
    c = CFG4
    _, g_ref, _ = _gradient(ml, keep, x0, target)
    adj = M.Adjoint(ml, c["n_steps"], c["every"], c["dt"], c["n_iter"], c["n_c"])
    x = dev(x0).requires_grad_(True)
    xT = M.MLSDCFunction.apply(x, adj)
    m, _ = osht.spec_mn(85)
    w = torch.from_numpy(np.where(m == 0, 1.0, 2.0)).cuda()
    loss = 0.5 * torch.sum(w * (xT[0] - dev(target)).abs() ** 2)
    loss.backward()
    got = host(x.grad)
    for f in range(3):
        assert rel_l2(85, got[f], g_ref[f]) <= 1e-13
