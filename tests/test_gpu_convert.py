"""The float32 -> float64 conversion the analysis kernels perform by
rearranging IEEE 754 bit fields on the integer pipes must equal the hardware
conversion bit for bit: every class of float32 bit pattern (normal numbers
across the whole exponent range, zeros of both signs, subnormals,
infinities, NaNs) from random bit patterns, plus the edges of the normal
range."""
import numpy as np
import pytest
import torch

from paper_1805_07923_gb300 import mlsdc as M

pytestmark = pytest.mark.gpu


def test_widening_equals_the_hardware():
    rng = np.random.default_rng(1805)
    bits = rng.integers(0, 2 ** 32, 1_000_000, dtype=np.uint64).astype(np.uint32)
    edges = np.array([0x00000000, 0x80000000, 0x00000001, 0x007fffff, 0x00800000, 0x80800000, 0x7f7fffff,
                      0xff7fffff, 0x7f800000, 0xff800000, 0x7fc00000, 0x7f800001, 0x3f800000, 0xbf800000],
                     dtype=np.uint32)
    bits = np.concatenate([edges, bits])
    f = torch.from_numpy(bits.view(np.float32).copy()).cuda()
    ours, hw = M.selftest_convert(f)
    torch.cuda.synchronize()
    o, h = ours.cpu().numpy().view(np.uint64), hw.cpu().numpy().view(np.uint64)
    bad = np.nonzero(o != h)[0]
    assert bad.size == 0, [(hex(bits[i]), hex(o[i]), hex(h[i])) for i in bad[:5]]
