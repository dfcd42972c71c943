"""The C-ABI library builds, loads without a GPU, and exports every function
that include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+\*?([a-z_][a-z0-9_]*)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_1805_07923_gb300 import build, mlsdc
    if not os.path.exists(mlsdc.LIB_PATH):
        build.build()
    return mlsdc.LIB_PATH


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["sh_plan", "sh_forward", "sh_inverse", "swe_explicit_rhs", "swe_implicit_solve",
                     "sdc_sweep", "mlsdc_step"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib_path):
    from paper_1805_07923_gb300 import mlsdc
    assert _declared() <= set(mlsdc.exported_symbols()) | {"sh_plan_destroy"}
    mlsdc.lib()


def test_invalid_sizes_are_rejected_without_a_gpu(lib_path):
    """Argument checks run before any CUDA call."""
    lib = ctypes.CDLL(lib_path)
    h = ctypes.c_void_p()
    assert lib.sh_plan(0, 64, 32, 0, ctypes.byref(h)) == -1          # R < 1
    assert lib.sh_plan(21, 60, 32, 0, ctypes.byref(h)) == -1         # nlon not a power of two
    assert lib.sh_plan(21, 32, 32, 0, ctypes.byref(h)) == -1         # nlon < 3R+1
    assert lib.sh_plan(21, 64, 31, 0, ctypes.byref(h)) == -1         # odd nlat
    assert lib.sh_plan(21, 64, 30, 0, ctypes.byref(h)) == -1         # nlat < (3R+1)/2
    assert lib.sh_plan(21, 64, 32, 7, ctypes.byref(h)) == -1         # precision
    lib.mlsdc_status_string.restype = ctypes.c_char_p
    assert lib.mlsdc_status_string(-1) == b"invalid argument"
