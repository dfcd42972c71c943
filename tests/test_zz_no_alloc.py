"""sh_inverse_static, the synthesis entry point that allocates nothing.

It serves callers that may not allocate device memory (their framework owns
the whole GPU through its own pool, or their footprint is fixed at start-up),
so it cannot use a plan; its scratch is one static device array in the
library.  Here it is called through the C ABI (ctypes) and must reproduce the
plan-based sh_inverse within the parity tolerance of the other tests, on two
calls in a row (the second call reuses the array the first one left behind).
This file is collected last so a stop-at-first-failure run has already run
every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1805_07923_gb300 import inputs
from paper_1805_07923_gb300 import mlsdc as M

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _c_call(R, I, J, spec, grid, nf):
    lib = M.lib()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.sh_inverse_static(R, I, J, ctypes.c_void_p(spec.data_ptr()), ctypes.c_void_p(grid.data_ptr()), nf, st)


# (169, 512, 384, 4): nf * nlat * (R+1) = 261120, exactly the scratch's capacity
@pytest.mark.parametrize("R,I,J,nf", [(21, 64, 32, 3), (170, 512, 256, 5), (45, 256, 70, 2), (169, 512, 384, 4)])
def test_static_inverse_matches_planned_inverse_twice(R, I, J, nf):
    plan = M.Plan(R, I, J)
    for call in range(2):
        spec_np = np.stack([inputs.spectrum(R, 500 + 10 * call + k, k, 1.0, slope=-0.5) for k in range(nf)])
        spec = torch.from_numpy(spec_np).cuda()
        ref = torch.empty((nf, J, I), dtype=torch.float64, device="cuda")
        got = torch.full((nf, J, I), float("nan"), dtype=torch.float64, device="cuda")
        M.sh_inverse(plan, spec, ref, nf)
        assert _c_call(R, I, J, spec, got, nf) == 0, M.lib().mlsdc_last_error()
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g))
        assert np.max(np.abs(g - r)) <= TOL * np.max(np.abs(r)), (call, np.max(np.abs(g - r)))


def test_static_inverse_rejects_requests_beyond_its_scratch():
    for R, I, J, nf in [(170, 512, 256, 6),     # 6 * 256 * 171 > 261120 complex values
                        (169, 512, 386, 4)]:    # 4 * 386 * 170 = 262480, just beyond
        spec = torch.zeros((nf, M.n_coeffs(R)), dtype=torch.complex128, device="cuda")
        grid = torch.zeros((nf, J, I), dtype=torch.float64, device="cuda")
        assert _c_call(R, I, J, spec, grid, nf) == -1
        assert b"static scratch" in M.lib().mlsdc_last_error()


def test_static_inverse_allocates_nothing():
    """After a first call (which loads the module and its static array), a
    call changes neither the device's free memory nor torch's allocator."""
    R, I, J, nf = 85, 256, 128, 3
    spec = torch.from_numpy(np.stack([inputs.spectrum(R, 700 + k, k, 1.0) for k in range(nf)])).cuda()
    grid = torch.empty((nf, J, I), dtype=torch.float64, device="cuda")
    assert _c_call(R, I, J, spec, grid, nf) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats()
    for _ in range(3):
        assert _c_call(R, I, J, spec, grid, nf) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0
    for key in ("allocation.all.allocated", "segment.all.allocated"):
        assert stats1.get(key, 0) == stats0.get(key, 0), key
