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


def test_static_inverse_argument_errors_name_the_problem(lib_path):
    """sh_inverse_static refuses bad sizes and pointers that are not 16-byte
    aligned before any CUDA call, each with its own message (the pointers
    here are never dereferenced)."""
    lib = ctypes.CDLL(lib_path)
    lib.mlsdc_last_error.restype = ctypes.c_char_p
    f = lib.sh_inverse_static
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                  ctypes.c_void_p]
    good, odd = 0x10000, 0x10008
    assert f(21, 60, 32, good, good, 1, None) == -1
    assert b"nlon" in lib.mlsdc_last_error()
    assert f(21, 64, 31, good, good, 1, None) == -1
    assert b"nlat" in lib.mlsdc_last_error()
    assert f(21, 64, 32, good, good, 0, None) == -1
    assert b"nf" in lib.mlsdc_last_error()
    assert f(21, 64, 32, None, good, 1, None) == -1
    assert b"null" in lib.mlsdc_last_error()
    assert f(21, 64, 32, odd, good, 1, None) == -1
    assert b"spec is not 16-byte aligned" in lib.mlsdc_last_error()
    assert f(21, 64, 32, good, odd, 1, None) == -1
    assert b"grid is not 16-byte aligned" in lib.mlsdc_last_error()


def test_planned_entry_points_refuse_misaligned_pointers(lib_path):
    """The alignment check runs before the plan is touched, so a fake plan
    handle is never dereferenced either."""
    lib = ctypes.CDLL(lib_path)
    lib.mlsdc_last_error.restype = ctypes.c_char_p
    fake_plan, good, odd = 0x20000, 0x10000, 0x10008
    lib.sh_inverse.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    assert lib.sh_inverse(fake_plan, odd, good, 1, None) == -1
    assert b"sh_inverse: spec is not 16-byte aligned" in lib.mlsdc_last_error()
    lib.sh_forward.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    assert lib.sh_forward(fake_plan, good, odd, 1, None) == -1
    assert b"sh_forward: spec is not 16-byte aligned" in lib.mlsdc_last_error()


def test_persistent_body_names_follow_the_body_enum():
    """The binding's names of the persistent kernel's bodies (phase timing)
    are the Body enumerators of the library, in order."""
    import re
    from paper_1805_07923_gb300 import mlsdc as M
    src = open(os.path.join(ROOT, "paper_1805_07923_gb300", "csrc", "vblock.cuh")).read()
    body = re.search(r"enum class Body : int \{(.*?)\};", src, re.S).group(1)
    names = [n.strip() for n in body.split(",") if n.strip() and n.strip() != "Count"]
    assert names == M.Ensemble.BODIES


def test_persistent_entry_points_refuse_bad_arguments(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.mlsdc_ensemble_persistent_schedule.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert lib.mlsdc_ensemble_persistent_schedule(None, 0) == -1
    lib.mlsdc_ensemble_persistent_info.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 4
    assert lib.mlsdc_ensemble_persistent_info(None, None, None, None, None) == -1
    lib.mlsdc_selftest_grid_barrier_timeout.argtypes = [ctypes.c_int, ctypes.c_void_p]
    code = ctypes.c_int()
    assert lib.mlsdc_selftest_grid_barrier_timeout(0, ctypes.byref(code)) == -1
    assert lib.mlsdc_selftest_grid_barrier_timeout(5000, ctypes.byref(code)) == -1
