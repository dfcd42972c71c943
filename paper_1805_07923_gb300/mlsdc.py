"""Thin ctypes binding of the C-ABI library libmlsdc_sh.so (include/mlsdc_sh.h).

Functions keep the C names; arguments are torch CUDA tensors (float64,
contiguous; complex values as interleaved (re, im) pairs, i.e. a
complex128 tensor or a float64 tensor of twice the length).  The binding only
marshals pointers and sizes: every step of the computation runs in the
library's CUDA kernels.  There is no CPU fallback: if the library is missing
or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmlsdc_sh.so")

MLSDC_FP64, MLSDC_TF32, MLSDC_BF16X3, MLSDC_FP32 = 0, 1, 2, 3
PRECISIONS = {"fp64": MLSDC_FP64, "tf32": MLSDC_TF32, "bf16x3": MLSDC_BF16X3, "fp32": MLSDC_FP32}

_lib = None


class SweParams(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("omega", ctypes.c_double), ("g", ctypes.c_double),
                ("phibar", ctypes.c_double), ("nu", ctypes.c_double)]


DEFAULT_PARAMS = dict(a=6.37122e6, omega=7.292e-5, g=9.80616, phibar=9.80616e4, nu=1.0e5)

_VP, _DP, _I, _D, _I64 = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64

_SIGS = {
    "mlsdc_status_string": ([_I], ctypes.c_char_p),
    "mlsdc_last_error": ([], ctypes.c_char_p),
    "sh_plan": ([_I, _I, _I, _I, ctypes.POINTER(_VP)], _I),
    "sh_plan_batched": ([_I, _I, _I, _I, _I, ctypes.POINTER(_VP)], _I),
    "swe_explicit_rhs_batched": ([_VP, ctypes.POINTER(SweParams), _DP, _DP, _I, _VP], _I),
    "sdc_level_create_batched": ([_VP, ctypes.POINTER(SweParams), _I, _I, ctypes.POINTER(_VP)], _I),
    "mlsdc_levels_create": ([ctypes.POINTER(_VP), _I, ctypes.POINTER(_VP)], _I),
    "mlsdc_levels_destroy": ([_VP], _I),
    "mlsdc_levels_step": ([_VP, _DP, _D, _I, _I, _I, _VP], _I),
    "mlsdc_levels_launch_count": ([_VP, ctypes.POINTER(_I64)], _I),
    "pfasst_create": ([_VP, _VP, ctypes.POINTER(_VP)], _I),
    "pfasst_destroy": ([_VP], _I),
    "pfasst_step": ([_VP, _DP, _DP, _D, _I, _I, _I, _I, _VP], _I),
    "pfasst_launch_count": ([_VP, ctypes.POINTER(_I64)], _I),
    "mlsdc_profile_node": ([_VP, _D, _I, ctypes.POINTER(ctypes.c_float), _VP], _I),
    "sdc_level_create_ex": ([_VP, ctypes.POINTER(SweParams), _I, _I, _I, ctypes.POINTER(_VP)], _I),
    "swe_implicit_rhs_ex": ([_VP, ctypes.POINTER(SweParams), _DP, _DP, _I, _VP], _I),
    "swe_implicit_solve_ex": ([_VP, ctypes.POINTER(SweParams), _D, _DP, _DP, _I, _VP], _I),
    "mlsdc_ensemble_create": ([ctypes.POINTER(_VP), _I, ctypes.POINTER(_VP)], _I),
    "mlsdc_ensemble_destroy": ([_VP], _I),
    "mlsdc_ensemble_step": ([_VP, ctypes.POINTER(_VP), _D, _I, _I, _I, _VP], _I),
    "mlsdc_ensemble_launch_count": ([_VP, ctypes.POINTER(_I64)], _I),
    "sh_plan_set_synth_tma": ([_VP, _I], _I),
    "mlsdc_selftest_convert": ([_DP, _I, _DP, _DP, _VP], _I),
    "mlsdc_ensemble_step_persistent": ([_VP, ctypes.POINTER(_VP), _D, _I, _I, _VP], _I),
    "mlsdc_ensemble_persistent_info": ([_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                                        ctypes.POINTER(_I)], _I),
    "mlsdc_ensemble_device_error": ([_VP, ctypes.POINTER(_I)], _I),
    "mlsdc_ensemble_persistent_schedule": ([_VP, _I], _I),
    "mlsdc_ensemble_persistent_phase_times": ([_VP, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_I), _I, _VP],
                                              _I),
    "mlsdc_selftest_grid_barrier_timeout": ([_I, ctypes.POINTER(_I)], _I),
    "sh_plan_destroy": ([_VP], _I),
    "sh_plan_grid": ([_VP, _DP, _DP], _I),
    "sh_plan_device_bytes": ([_VP, ctypes.POINTER(_I64)], _I),
    "sh_plan_device_error": ([_VP, ctypes.POINTER(_I)], _I),
    "sh_inverse": ([_VP, _DP, _DP, _I, _VP], _I),
    "sh_forward": ([_VP, _DP, _DP, _I, _VP], _I),
    "sh_inverse_static": ([_I, _I, _I, _DP, _DP, _I, _VP], _I),
    "swe_explicit_rhs": ([_VP, ctypes.POINTER(SweParams), _DP, _DP, _VP], _I),
    "swe_implicit_rhs": ([_VP, ctypes.POINTER(SweParams), _DP, _DP, _VP], _I),
    "swe_implicit_solve": ([_VP, ctypes.POINTER(SweParams), _D, _DP, _DP, _VP], _I),
    "sdc_level_create": ([_VP, ctypes.POINTER(SweParams), _I, ctypes.POINTER(_VP)], _I),
    "sdc_level_destroy": ([_VP], _I),
    "sdc_level_matrices": ([_VP, _DP, _DP, _DP, _DP], _I),
    "sdc_sweep": ([_VP, _D, _DP, _DP, _DP, _DP, _DP, _DP, _VP], _I),
    "sdc_step": ([_VP, _DP, _D, _I, _VP], _I),
    "mlsdc_create": ([_VP, _VP, ctypes.POINTER(_VP)], _I),
    "mlsdc_destroy": ([_VP], _I),
    "mlsdc_step": ([_VP, _DP, _D, _I, _I, _I, _VP], _I),
    "mlsdc_launch_count": ([_VP, ctypes.POINTER(_I64)], _I),
    "mlsdc_check_finite": ([_DP, _I64, ctypes.POINTER(_I), _VP], _I),
    "mlsdc_profile_rhs": ([_VP, ctypes.POINTER(SweParams), _DP, _DP, _I, ctypes.POINTER(ctypes.c_float), _VP], _I),
    "mlsdc_profile_rhs_batched": ([_VP, ctypes.POINTER(SweParams), _DP, _DP, _I, _I, ctypes.POINTER(ctypes.c_float),
                                   _VP], _I),
    "sh_plan_stage_kernels": ([_VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)], _I),
    "sh_plan_set_stage_kernels": ([_VP, _I, _I], _I),
    "sh_plan_tc_config": ([_VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)], _I),
    "sh_plan_set_tc_config": ([_VP, _I, _I, _I, _I], _I),
    "mlsdc_selftest_wait_timeout": ([_I, ctypes.POINTER(_I)], _I),
    "swe_explicit_rhs_adjoint": ([_VP, ctypes.POINTER(SweParams), _DP, _DP, _DP, _VP], _I),
    "mlsdc_phi_misfit": ([_VP, _DP, _DP, _DP, _DP, _VP], _I),
    "mlsdc_adjoint_create": ([_VP, _I, _I, _D, _I, _I, ctypes.POINTER(_VP)], _I),
    "mlsdc_adjoint_destroy": ([_VP], _I),
    "mlsdc_adjoint_forward": ([_VP, _DP, _DP, _I, _VP], _I),
    "mlsdc_adjoint_backward": ([_VP, _DP, _DP, _I, _VP], _I),
    "mlsdc_adjoint_launch_count": ([_VP, ctypes.POINTER(_I64), ctypes.POINTER(_I64)], _I),
    "mlsdc_profile_rhs_adjoint": ([_VP, ctypes.POINTER(SweParams), _DP, _DP, _DP, _I, ctypes.POINTER(ctypes.c_float),
                                   _VP], _I),
}


def lib():
    """Load the library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


class MlsdcError(RuntimeError):
    pass


def _check(status: int, what: str):
    if status != 0:
        L = lib()
        raise MlsdcError(f"{what}: {L.mlsdc_status_string(status).decode()} "
                         f"({L.mlsdc_last_error().decode()})")


def _ptr(t: torch.Tensor | None, numel_f64: int | None = None):
    if t is None:
        return None
    if not t.is_cuda:
        raise MlsdcError("tensor must live on a CUDA device")
    if t.dtype not in (torch.float64, torch.complex128):
        raise MlsdcError(f"tensor must be float64 or complex128, got {t.dtype}")
    if not t.is_contiguous():
        raise MlsdcError("tensor must be contiguous")
    if t.data_ptr() % 16 != 0:
        raise MlsdcError("tensor data must be 16-byte aligned (complex values are read as 16-byte words)")
    if numel_f64 is not None:
        n = t.numel() * (2 if t.dtype == torch.complex128 else 1)
        if n < numel_f64:
            raise MlsdcError(f"tensor holds {n} doubles, {numel_f64} needed")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def swe_params(**kw) -> SweParams:
    d = dict(DEFAULT_PARAMS)
    d.update(kw)
    return SweParams(**d)


def n_coeffs(R: int) -> int:
    return (R + 1) * (R + 2) // 2


class Plan:
    """sh_plan: Gaussian grid and Legendre tables of one truncation."""

    def __init__(self, R: int, nlon: int, nlat: int, precision="fp64", max_members: int = 1):
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        h = ctypes.c_void_p()
        if max_members == 1:
            _check(lib().sh_plan(R, nlon, nlat, prec, ctypes.byref(h)), "sh_plan")
        else:
            _check(lib().sh_plan_batched(R, nlon, nlat, prec, int(max_members), ctypes.byref(h)), "sh_plan_batched")
        self.h, self.R, self.I, self.J, self.precision = h, R, nlon, nlat, prec
        self.max_members = max_members
        self.nc = n_coeffs(R)

    def close(self):
        if self.h:
            lib().sh_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def grid(self):
        import numpy as np
        mu = np.zeros(self.J)
        w = np.zeros(self.J)
        _check(lib().sh_plan_grid(self.h, mu.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p)),
               "sh_plan_grid")
        return mu, w

    def device_error(self) -> int:
        """Error code recorded by the plan's tensor-core kernels (0 = none)."""
        c = ctypes.c_int()
        _check(lib().sh_plan_device_error(self.h, ctypes.byref(c)), "sh_plan_device_error")
        return c.value

    def device_bytes(self) -> int:
        b = ctypes.c_int64()
        _check(lib().sh_plan_device_bytes(self.h, ctypes.byref(b)), "sh_plan_device_bytes")
        return b.value

    STAGE_MODES = {"auto": 0, "tc": 1, "simt": 2}

    def stage_kernels(self, members: int = 1) -> tuple[bool, bool]:
        """(synthesis on tensor cores, analysis on tensor cores) for a launch of `members` states."""
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(lib().sh_plan_stage_kernels(self.h, int(members), ctypes.byref(a), ctypes.byref(b)),
               "sh_plan_stage_kernels")
        return bool(a.value), bool(b.value)

    TC_STAGES = {"synthesis": 0, "analysis": 2}

    def tc_config(self, stage: str = "analysis") -> tuple[int, int, int]:
        """(members per CTA, K-pipeline stages, warp-specialised batched analysis) of one
        tensor-core Legendre stage; zeros for other precisions."""
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().sh_plan_tc_config(self.h, self.TC_STAGES[stage], ctypes.byref(a), ctypes.byref(b),
                                       ctypes.byref(c)), "sh_plan_tc_config")
        return a.value, b.value, c.value

    def set_tc_config(self, members_per_cta: int, stages: int, warp_specialised: int = 0, stage: str = "analysis"):
        """Replace the autotuned configuration of one tensor-core Legendre stage."""
        _check(lib().sh_plan_set_tc_config(self.h, self.TC_STAGES[stage], int(members_per_cta), int(stages),
                                           int(warp_specialised)), "sh_plan_set_tc_config")

    def set_stage_kernels(self, synth: str = "auto", anal: str = "auto"):
        """Per-stage kernel mode of a tensor-core plan: "auto" (the size rule), "tc" or "simt"."""
        _check(lib().sh_plan_set_stage_kernels(self.h, self.STAGE_MODES[synth], self.STAGE_MODES[anal]),
               "sh_plan_set_stage_kernels")

    def set_synth_tma(self, mode: str = "auto"):
        """How the float32 synthesis reads its tables: "auto" (the size rule), "tma" or "loads"."""
        _check(lib().sh_plan_set_synth_tma(self.h, {"auto": 0, "tma": 1, "loads": 2}[mode]), "sh_plan_set_synth_tma")


def selftest_wait_timeout(timeout_ms: int = 20) -> int:
    """Run the bounded-wait check (one CTA waiting on an mbarrier nothing completes);
    returns the code the kernel recorded (2: the wait gave up, as it must)."""
    c = ctypes.c_int()
    _check(lib().mlsdc_selftest_wait_timeout(int(timeout_ms), ctypes.byref(c)), "mlsdc_selftest_wait_timeout")
    return c.value


def sh_inverse(plan: Plan, spec: torch.Tensor, grid: torch.Tensor, nf: int, stream=None):
    _check(lib().sh_inverse(plan.h, _ptr(spec, 2 * nf * plan.nc), _ptr(grid, nf * plan.I * plan.J), nf,
                            _stream(stream)), "sh_inverse")


def sh_inverse_static(R: int, nlon: int, nlat: int, spec: torch.Tensor, grid: torch.Tensor, nf: int, stream=None):
    """Plan-free synthesis that allocates nothing (static device scratch)."""
    nc = n_coeffs(R)
    _check(lib().sh_inverse_static(int(R), int(nlon), int(nlat), _ptr(spec, 2 * nf * nc), _ptr(grid, nf * nlon * nlat),
                                   int(nf), _stream(stream)), "sh_inverse_static")


def sh_forward(plan: Plan, grid: torch.Tensor, spec: torch.Tensor, nf: int, stream=None):
    _check(lib().sh_forward(plan.h, _ptr(grid, nf * plan.I * plan.J), _ptr(spec, 2 * nf * plan.nc), nf,
                            _stream(stream)), "sh_forward")


def swe_explicit_rhs(plan: Plan, prm: SweParams, state: torch.Tensor, FE: torch.Tensor, stream=None):
    _check(lib().swe_explicit_rhs(plan.h, ctypes.byref(prm), _ptr(state, 6 * plan.nc), _ptr(FE, 6 * plan.nc),
                                  _stream(stream)), "swe_explicit_rhs")


def swe_explicit_rhs_batched(plan: Plan, prm: SweParams, states: torch.Tensor, FE: torch.Tensor, members: int,
                             stream=None):
    n = 6 * plan.nc * members
    _check(lib().swe_explicit_rhs_batched(plan.h, ctypes.byref(prm), _ptr(states, n), _ptr(FE, n), int(members),
                                          _stream(stream)), "swe_explicit_rhs_batched")


# option bit of the splitting (include/mlsdc_sh.h): the Coriolis terms in F_I
CORIOLIS_IMPLICIT = 1


def swe_implicit_rhs(plan: Plan, prm: SweParams, state: torch.Tensor, FI: torch.Tensor, stream=None,
                     coriolis_implicit: bool = False):
    _check(lib().swe_implicit_rhs_ex(plan.h, ctypes.byref(prm), _ptr(state, 6 * plan.nc), _ptr(FI, 6 * plan.nc),
                                     CORIOLIS_IMPLICIT if coriolis_implicit else 0, _stream(stream)),
           "swe_implicit_rhs_ex")


def swe_implicit_solve(plan: Plan, prm: SweParams, alpha: float, b: torch.Tensor, x: torch.Tensor, stream=None,
                       coriolis_implicit: bool = False):
    _check(lib().swe_implicit_solve_ex(plan.h, ctypes.byref(prm), float(alpha), _ptr(b, 6 * plan.nc),
                                       _ptr(x, 6 * plan.nc), CORIOLIS_IMPLICIT if coriolis_implicit else 0,
                                       _stream(stream)), "swe_implicit_solve_ex")


class Level:
    """sdc_level: a plan, the physics and n Gauss-Lobatto nodes (with
    coriolis_implicit: the splitting with the Coriolis terms in F_I)."""

    def __init__(self, plan: Plan, n_nodes: int, prm: SweParams | None = None, members: int = 1,
                 coriolis_implicit: bool = False):
        self.plan = plan
        self.prm = prm if prm is not None else swe_params()
        h = ctypes.c_void_p()
        opts = CORIOLIS_IMPLICIT if coriolis_implicit else 0
        _check(lib().sdc_level_create_ex(plan.h, ctypes.byref(self.prm), n_nodes, int(members), opts, ctypes.byref(h)),
               "sdc_level_create_ex")
        self.h, self.n, self.members = h, n_nodes, members
        self.coriolis_implicit = bool(coriolis_implicit)

    def close(self):
        if self.h:
            lib().sdc_level_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def matrices(self):
        import numpy as np
        n = self.n
        t, Q, QE, QI = np.zeros(n), np.zeros(n * n), np.zeros(n * n), np.zeros(n * n)
        args = [a.ctypes.data_as(ctypes.c_void_p) for a in (t, Q, QE, QI)]
        _check(lib().sdc_level_matrices(self.h, *args), "sdc_level_matrices")
        return t, Q.reshape(n, n), QE.reshape(n, n), QI.reshape(n, n)


def mlsdc_profile_node(level: Level, dt: float, reps: int = 20, stream=None) -> list[float]:
    """Device milliseconds of each node update m = 0..n-2 of the level."""
    out = (ctypes.c_float * (level.n - 1))()
    _check(lib().mlsdc_profile_node(level.h, float(dt), int(reps), out, _stream(stream)), "mlsdc_profile_node")
    return list(out)


def sdc_sweep(level: Level, dt: float, Theta, FI_old, FE_old, FI_new, FE_new, tau=None, stream=None):
    n = 6 * level.n * level.plan.nc * level.members
    _check(lib().sdc_sweep(level.h, float(dt), _ptr(Theta, n), _ptr(FI_old, n), _ptr(FE_old, n), _ptr(FI_new, n),
                           _ptr(FE_new, n), _ptr(tau, n), _stream(stream)), "sdc_sweep")


def sdc_step(level: Level, state: torch.Tensor, dt: float, n_sweeps: int, stream=None):
    _check(lib().sdc_step(level.h, _ptr(state, 6 * level.plan.nc * level.members), float(dt), int(n_sweeps), _stream(stream)),
           "sdc_step")


class MLSDC:
    """Two-level MLSDC object (fine and coarse levels must outlive it)."""

    def __init__(self, fine: Level, coarse: Level):
        self.fine, self.coarse = fine, coarse
        h = ctypes.c_void_p()
        _check(lib().mlsdc_create(fine.h, coarse.h, ctypes.byref(h)), "mlsdc_create")
        self.h = h

    def close(self):
        if self.h:
            lib().mlsdc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch_count(self) -> int:
        v = ctypes.c_int64()
        _check(lib().mlsdc_launch_count(self.h, ctypes.byref(v)), "mlsdc_launch_count")
        return v.value


def mlsdc_step(ml: MLSDC, state: torch.Tensor, dt: float, n_iter: int, n_coarse_sweeps: int, use_graph: bool = False,
               stream=None):
    _check(lib().mlsdc_step(ml.h, _ptr(state, 6 * ml.fine.plan.nc * ml.fine.members), float(dt), int(n_iter), int(n_coarse_sweeps),
                            1 if use_graph else 0, _stream(stream)), "mlsdc_step")


class MLSDCLevels:
    """MLSDC on two or more levels (levels[0] finest; the levels must outlive it)."""

    def __init__(self, levels: list[Level]):
        self.levels = list(levels)
        arr = (ctypes.c_void_p * len(levels))(*[lv.h.value for lv in levels])
        h = ctypes.c_void_p()
        _check(lib().mlsdc_levels_create(arr, len(levels), ctypes.byref(h)), "mlsdc_levels_create")
        self.h = h

    def close(self):
        if self.h:
            lib().mlsdc_levels_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch_count(self) -> int:
        v = ctypes.c_int64()
        _check(lib().mlsdc_levels_launch_count(self.h, ctypes.byref(v)), "mlsdc_levels_launch_count")
        return v.value


def mlsdc_levels_step(ml: MLSDCLevels, state: torch.Tensor, dt: float, n_iter: int, n_coarse_sweeps: int,
                      use_graph: bool = False, stream=None):
    f = ml.levels[0]
    _check(lib().mlsdc_levels_step(ml.h, _ptr(state, 6 * f.plan.nc * f.members), float(dt), int(n_iter),
                                   int(n_coarse_sweeps), 1 if use_graph else 0, _stream(stream)), "mlsdc_levels_step")


class PFASST:
    """pfasst_create: two-level PFASST over P time slices, the P members of the
    batched fine and coarse levels (which must outlive it)."""

    def __init__(self, fine: Level, coarse: Level):
        self.fine, self.coarse = fine, coarse
        h = ctypes.c_void_p()
        _check(lib().pfasst_create(fine.h, coarse.h, ctypes.byref(h)), "pfasst_create")
        self.h = h
        self.slices = fine.members

    def close(self):
        if self.h:
            lib().pfasst_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch_count(self) -> int:
        v = ctypes.c_int64()
        _check(lib().pfasst_launch_count(self.h, ctypes.byref(v)), "pfasst_launch_count")
        return v.value


def pfasst_step(pf: PFASST, u0: torch.Tensor, ends: torch.Tensor, dt: float, n_iter: int, n_coarse_sweeps: int,
                n_predictor_sweeps: int = -1, use_graph: bool = False, stream=None):
    """Advance u0 ([3][N_c]) over pf.slices slices of length dt; ends
    ([slices][3][N_c]) receives every slice's end value."""
    nc = pf.fine.plan.nc
    _check(lib().pfasst_step(pf.h, _ptr(u0, 6 * nc), _ptr(ends, 6 * nc * pf.slices), float(dt), int(n_iter),
                             int(n_coarse_sweeps), int(n_predictor_sweeps), 1 if use_graph else 0, _stream(stream)),
           "pfasst_step")


def mlsdc_check_finite(x: torch.Tensor, stream=None) -> bool:
    ok = ctypes.c_int()
    n = x.numel() * (2 if x.dtype == torch.complex128 else 1)
    _check(lib().mlsdc_check_finite(_ptr(x), n, ctypes.byref(ok), _stream(stream)), "mlsdc_check_finite")
    return bool(ok.value)


def mlsdc_profile_rhs(plan: Plan, prm: SweParams, state: torch.Tensor, FE: torch.Tensor, reps: int = 50,
                      stream=None, members: int = 1) -> list[float]:
    """Mean ms per launch of the three F_E stage kernels (synthesis, grid, analysis)."""
    out = (ctypes.c_float * 3)()
    n = 6 * plan.nc * members
    _check(lib().mlsdc_profile_rhs_batched(plan.h, ctypes.byref(prm), _ptr(state, n), _ptr(FE, n), int(members),
                                           int(reps), out, _stream(stream)), "mlsdc_profile_rhs_batched")
    return [float(v) for v in out]


class Ensemble:
    """MLSDC groups of uneven truncation stepped together (one graph per step)."""

    def __init__(self, groups: list[MLSDC]):
        self.groups = list(groups)
        arr = (ctypes.c_void_p * len(groups))(*[g.h for g in groups])
        h = ctypes.c_void_p()
        _check(lib().mlsdc_ensemble_create(arr, len(groups), ctypes.byref(h)), "mlsdc_ensemble_create")
        self.h = h

    def close(self):
        if self.h:
            lib().mlsdc_ensemble_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch_count(self) -> int:
        v = ctypes.c_int64()
        _check(lib().mlsdc_ensemble_launch_count(self.h, ctypes.byref(v)), "mlsdc_ensemble_launch_count")
        return v.value

    def persistent_info(self) -> dict:
        """phases, records, ctas, in_graph of the last persistent step."""
        v = [ctypes.c_int() for _ in range(4)]
        _check(lib().mlsdc_ensemble_persistent_info(self.h, *[ctypes.byref(x) for x in v]),
               "mlsdc_ensemble_persistent_info")
        return dict(zip(("phases", "records", "ctas", "in_graph"), (x.value for x in v)))

    def set_persistent_schedule(self, schedule: str):
        """'lockstep' (default) or 'dataflow' for later persistent steps."""
        code = {"lockstep": 0, "dataflow": 1}[schedule]
        _check(lib().mlsdc_ensemble_persistent_schedule(self.h, code), "mlsdc_ensemble_persistent_schedule")

    def device_error(self) -> int:
        c = ctypes.c_int()
        _check(lib().mlsdc_ensemble_device_error(self.h, ctypes.byref(c)), "mlsdc_ensemble_device_error")
        return c.value

    # the persistent kernel's bodies, in the library's Body order (vblock.cuh)
    BODIES = ["SynthF32", "SynthF64", "GridF32x1", "GridF32x2", "GridF64x1", "AnalF32", "AnalF64", "TcSynthTf32",
              "TcSynthBf16", "TcAnalTf32", "TcAnalBf16", "TcAnalWsTf32", "TcAnalWsBf16", "ImplicitRhs", "SweepNode",
              "SweepNode0_2", "SweepNode0_3", "SweepNode0_4", "SweepNode0_5", "SweepNode0_6", "SweepNode0_7",
              "SweepNode0_8", "SweepNodeS", "Broadcast", "Restrict", "FasTau", "Interp", "PadAdd", "Copy2D",
              "SynthF32Tma"]

    def persistent_phase_times(self, stream=None) -> list[tuple[str, float]]:
        """One more persistent step with per-phase timer readings: (body, microseconds) per phase."""
        n = self.persistent_info()["phases"]
        us = (ctypes.c_float * n)()
        body = (ctypes.c_int * n)()
        _check(lib().mlsdc_ensemble_persistent_phase_times(self.h, us, body, n, _stream(stream)),
               "mlsdc_ensemble_persistent_phase_times")
        return [(self.BODIES[body[i]], float(us[i])) for i in range(n)]


def mlsdc_ensemble_step_persistent(ens: Ensemble, states: list[torch.Tensor], dt: float, n_iter: int,
                                   n_coarse_sweeps: int, stream=None):
    """The ensemble step as one persistent kernel launch (captured in a graph)."""
    if len(states) != len(ens.groups):
        raise MlsdcError("one state tensor per group")
    ptrs = [_ptr(s, 6 * g.fine.plan.nc * g.fine.members) for s, g in zip(states, ens.groups)]
    arr = (ctypes.c_void_p * len(ptrs))(*[p.value for p in ptrs])
    _check(lib().mlsdc_ensemble_step_persistent(ens.h, arr, float(dt), int(n_iter), int(n_coarse_sweeps),
                                                _stream(stream)), "mlsdc_ensemble_step_persistent")


def selftest_convert(f_in: torch.Tensor, stream=None):
    """The library's float32 -> float64 conversion next to the hardware's: (d_ours, d_hw)."""
    if f_in.dtype != torch.float32:
        raise MlsdcError("selftest_convert: f_in must be float32")
    n = f_in.numel()
    d_ours = torch.empty(n, dtype=torch.float64, device=f_in.device)
    d_hw = torch.empty_like(d_ours)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    _check(lib().mlsdc_selftest_convert(p(f_in), n, p(d_ours), p(d_hw), _stream(stream)), "mlsdc_selftest_convert")
    return d_ours, d_hw


def selftest_grid_barrier_timeout(timeout_ms: int = 20) -> int:
    """Two CTAs at a grid barrier that never completes: returns the code they leave (3 = gave up)."""
    c = ctypes.c_int(-1)
    _check(lib().mlsdc_selftest_grid_barrier_timeout(int(timeout_ms), ctypes.byref(c)),
           "mlsdc_selftest_grid_barrier_timeout")
    return c.value


def mlsdc_ensemble_step(ens: Ensemble, states: list[torch.Tensor], dt: float, n_iter: int, n_coarse_sweeps: int,
                        use_graph: bool = True, stream=None):
    if len(states) != len(ens.groups):
        raise MlsdcError("one state tensor per group")
    ptrs = [_ptr(s, 6 * g.fine.plan.nc * g.fine.members) for s, g in zip(states, ens.groups)]
    arr = (ctypes.c_void_p * len(ptrs))(*[p.value for p in ptrs])
    _check(lib().mlsdc_ensemble_step(ens.h, arr, float(dt), int(n_iter), int(n_coarse_sweeps), 1 if use_graph else 0,
                                     _stream(stream)), "mlsdc_ensemble_step")


# ---------------------------------------------------------------------------
# adjoint (reverse mode with respect to the initial state)


def swe_explicit_rhs_adjoint(plan: Plan, prm: SweParams, state: torch.Tensor, lam: torch.Tensor,
                             state_bar: torch.Tensor, stream=None):
    """state_bar += F_E'(state)^t lam; lam is zeroed (consumed)."""
    n = 6 * plan.nc
    _check(lib().swe_explicit_rhs_adjoint(plan.h, ctypes.byref(prm), _ptr(state, n), _ptr(lam, n), _ptr(state_bar, n),
                                          _stream(stream)), "swe_explicit_rhs_adjoint")


def mlsdc_phi_misfit(plan: Plan, state: torch.Tensor, phi_target: torch.Tensor, J: torch.Tensor, lam: torch.Tensor,
                     stream=None):
    """J[0] = 1/2 ||Phi'(state) - phi_target||^2 (Parseval) and lam = dJ/dstate, on the device."""
    _check(lib().mlsdc_phi_misfit(plan.h, _ptr(state, 6 * plan.nc), _ptr(phi_target, 2 * plan.nc), _ptr(J, 1),
                                  _ptr(lam, 6 * plan.nc), _stream(stream)), "mlsdc_phi_misfit")


def mlsdc_profile_rhs_adjoint(plan: Plan, prm: SweParams, state: torch.Tensor, lam: torch.Tensor,
                              state_bar: torch.Tensor, reps: int = 50, stream=None) -> list[float]:
    """Mean ms per launch of the three F_E-adjoint stage kernels."""
    out = (ctypes.c_float * 3)()
    n = 6 * plan.nc
    _check(lib().mlsdc_profile_rhs_adjoint(plan.h, ctypes.byref(prm), _ptr(state, n), _ptr(lam, n),
                                           _ptr(state_bar, n), int(reps), out, _stream(stream)),
           "mlsdc_profile_rhs_adjoint")
    return [float(v) for v in out]


class Adjoint:
    """mlsdc_adjoint: n_steps MLSDC steps and their reverse mode, with a
    checkpoint every `checkpoint_every` steps."""

    def __init__(self, ml: MLSDC, n_steps: int, checkpoint_every: int, dt: float, n_iter: int, n_coarse_sweeps: int,
                 use_graph: bool = True):
        self.ml = ml
        self.nc = ml.fine.plan.nc
        self.use_graph = 1 if use_graph else 0
        h = ctypes.c_void_p()
        _check(lib().mlsdc_adjoint_create(ml.h, int(n_steps), int(checkpoint_every), float(dt), int(n_iter),
                                          int(n_coarse_sweeps), ctypes.byref(h)), "mlsdc_adjoint_create")
        self.h = h

    def close(self):
        if self.h:
            lib().mlsdc_adjoint_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, state0: torch.Tensor, state_T: torch.Tensor, stream=None):
        n = 6 * self.nc
        _check(lib().mlsdc_adjoint_forward(self.h, _ptr(state0, n), _ptr(state_T, n), self.use_graph,
                                           _stream(stream)), "mlsdc_adjoint_forward")

    def backward(self, lam_T: torch.Tensor, lam_0: torch.Tensor, stream=None):
        n = 6 * self.nc
        _check(lib().mlsdc_adjoint_backward(self.h, _ptr(lam_T, n), _ptr(lam_0, n), self.use_graph,
                                            _stream(stream)), "mlsdc_adjoint_backward")

    def launch_counts(self) -> tuple[int, int]:
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().mlsdc_adjoint_launch_count(self.h, ctypes.byref(a), ctypes.byref(b)), "mlsdc_adjoint_launch_count")
        return a.value, b.value


class MLSDCFunction(torch.autograd.Function):
    """state_T = (n_steps MLSDC steps)(state0) with the library's hand-written
    adjoint as its backward: MLSDCFunction.apply(state0, adjoint) for a
    complex128 [3][N_c] CUDA tensor; gradients follow PyTorch's complex
    convention (dL/dRe + i dL/dIm), Im of m = 0 excluded."""

    @staticmethod
    def forward(ctx, state0: torch.Tensor, adj: Adjoint):
        x0 = state0.detach().contiguous()
        out = torch.empty_like(x0)
        adj.forward(x0, out)
        ctx.adj = adj
        return out

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        g = grad_out.detach().contiguous().clone()
        out = torch.empty_like(g)
        ctx.adj.backward(g, out)
        return out, None
