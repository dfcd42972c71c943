"""The float32 synthesis with its Legendre tables streamed into shared
memory by TMA against the same kernel reading them with plain loads: the
same sums in the same order, so F_E must be identical bit for bit, at every
truncation and batch size the plans use (boxes of 32 rows: R = 21 one box,
R = 85 three, R = 170 six; J2 below, equal to and above the 32-latitude box
width), with no bounded wait giving up."""
import numpy as np
import pytest
import torch

from paper_1805_07923_gb300 import inputs
from paper_1805_07923_gb300 import mlsdc as M

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("R,I,J,B", [(10, 32, 16, 1), (21, 64, 32, 3), (42, 128, 64, 16), (85, 256, 128, 1),
                                     (85, 256, 128, 5), (170, 512, 256, 2)])
@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_tma_synthesis_equals_plain_loads(R, I, J, B, prec):
    base = inputs.initial_state(170)
    x = torch.from_numpy(np.stack([inputs.perturbed_member(base, 170, R, k) for k in range(B)])).cuda()
    p = M.Plan(R, I, J, prec, B)
    out = {}
    for mode in ("loads", "tma", "auto"):
        p.set_synth_tma(mode)
        fe = torch.full_like(x, float("nan"))
        M.swe_explicit_rhs_batched(p, M.swe_params(), x, fe, B)
        torch.cuda.synchronize()
        out[mode] = fe.cpu().numpy()
    assert p.device_error() == 0
    assert np.all(np.isfinite(out["tma"]))
    assert np.array_equal(out["tma"], out["loads"])
    assert np.array_equal(out["auto"], out["loads"])
