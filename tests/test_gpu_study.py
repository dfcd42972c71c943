"""The Gaussian-dome workload and the time-refinement study on the GPU.

Parity: the dome's spectral state (the library's own analysis of the
analytic grid field) and an MLSDC step from it match the float64 oracle to
1e-12.  Behaviour (Sec. 5): on T42/T21 over 4 hours against an SDC(5,8)
reference at 60 s, SDC(3,4) and SDC(5,8) converge at their orders 4 and 8;
MLSDC(3,2,2,1/2) has the error of SDC(3,4) at large steps; MLSDC(5,3,4,1/2)
is more accurate than SDC(3,4) at every step size and settles near fourth
order once spatial coarsening limits the coarse correction (the regime the
paper describes for small steps)."""
import numpy as np
import pytest
import torch

from oracle import sdc as osdc
from oracle import sht as osht
from oracle.swe import SWE, Params
from paper_1805_07923_gb300 import inputs
from paper_1805_07923_gb300 import mlsdc as M
from paper_1805_07923_gb300 import study

pytestmark = pytest.mark.gpu

G = 9.80616


def rel_l2(R, got, ref):
    return float(np.sqrt(osht.norm2(R, got - ref) / max(osht.norm2(R, ref), 1e-300)))


@pytest.fixture(scope="module")
def small():
    return study.Study("dome", 42, 128, 64, 21, 64, 32)


def test_dome_state_matches_oracle(small):
    o = SWE(42, 128, 64, Params(phibar=G * inputs.DOME_H_BAR))
    phi, _ = inputs.gaussian_dome_grid(o.grid.lam, o.grid.mu)
    ref = o.grid.analysis(phi)
    got = small.x0.cpu().numpy()
    assert rel_l2(42, got[0], ref) <= 1e-12
    assert np.all(got[1:] == 0)


def test_dome_mlsdc_step_matches_oracle(small):
    p = Params(phibar=G * inputs.DOME_H_BAR)
    of, oc = osdc.Level(SWE(42, 128, 64, p), 5), osdc.Level(SWE(21, 64, 32, p), 3)
    u = small.x0.cpu().numpy()
    x, _, _ = small.run("MLSDC(5,3,4,1/2)", 600.0, 600.0)
    ref = osdc.mlsdc_step(of, oc, u, 600.0, 4, 1)
    got = x.cpu().numpy()
    for k in range(3):
        assert rel_l2(42, got[k], ref[k]) <= 1e-12, (k, rel_l2(42, got[k], ref[k]))


def test_refinement_orders_on_dome(small):
    T = 4 * 3600.0
    ref, _, _ = small.run("SDC(5,8)", 60.0, T)
    norm = small.linf(ref, 0)
    dts = [1800.0, 900.0, 450.0, 300.0]
    err = {}
    for scheme in study.SCHEMES:
        err[scheme] = [small.linf(small.run(scheme, dt, T)[0] - ref, 0) / norm for dt in dts]
    order = {s: study.observed_orders(dts, e) for s, e in err.items()}
    print({s: ["%.2e" % v for v in e] for s, e in err.items()}, order)
    assert 3.3 < order["SDC(3,4)"][-1] < 4.7
    assert 7.0 < order["SDC(5,8)"][-1] < 9.5
    assert err["MLSDC(3,2,2,1/2)"][0] < 1.3 * err["SDC(3,4)"][0]
    assert err["MLSDC(3,2,2,1/2)"][1] < 1.3 * err["SDC(3,4)"][1]
    assert all(a < b for a, b in zip(err["MLSDC(5,3,4,1/2)"], err["SDC(3,4)"]))
    assert 3.0 < order["MLSDC(5,3,4,1/2)"][-1] < 4.8
