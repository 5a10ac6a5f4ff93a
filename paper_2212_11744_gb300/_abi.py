"""ctypes mirror of include/lqt.h: structs, prototypes and library loading.

Argument marshalling only.  The library is loaded from the package's `_lib`
directory; if it is missing the import of any entry point raises, so a GPU run
can never silently fall back to another implementation.
"""
from __future__ import annotations

import ctypes as ct
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblqt_gb300.so")

LQT_OK, LQT_EINVAL, LQT_EWORKSPACE, LQT_ENONFINITE, LQT_ESINGULAR, LQT_ETIMEOUT, LQT_ECUDA, LQT_EUNSUPPORTED = range(8)
LQT_CONST, LQT_PER_INTERVAL, LQT_PER_STAGE = 0, 1, 2
(LQT_WS_BUILD, LQT_WS_VALUE, LQT_WS_TRAJ, LQT_WS_SOLVE, LQT_WS_SEQUENTIAL, LQT_WS_BACKWARD, LQT_WS_DENSIFY,
 LQT_WS_METHOD2, LQT_WS_SOLVE_METHOD2, LQT_WS_INVARIANT, LQT_WS_SOLVE_INVARIANT) = range(11)
LQT_TUNE_INVARIANT_BUILD = 1
LQT_STATIC_SCRATCH_BYTES = 16 << 20

EXPORTED = (
    "lqt_workspace_size", "lqt_build_elements", "lqt_scan_value", "lqt_scan_trajectory", "lqt_solve",
    "lqt_solve_sequential", "lqt_host_staging_size", "lqt_solve_host", "lqt_get_status", "lqt_strerror",
    "lqt_last_launch_count", "lqt_scan_value_noalloc", "lqt_backward", "lqt_batch_workspace_size",
    "lqt_batch_boundaries", "lqt_batch_plan", "lqt_solve_batched", "lqt_solve_mixed", "lqt_densify",
    "lqt_build_elements_forward", "lqt_trajectory_method2", "lqt_solve_method2", "lqt_build_elements_invariant",
    "lqt_solve_invariant", "lqt_grid_workspace_size", "lqt_grid_block", "lqt_grid_combine", "lqt_grid_values",
    "lqt_probe_fma_rate",
)

_dp = ct.POINTER(ct.c_double)


class lqt_coef(ct.Structure):
    _fields_ = [("ptr", ct.c_void_p), ("mode", ct.c_int32)]


class lqt_problem(ct.Structure):
    _fields_ = [
        ("n", ct.c_int32), ("m", ct.c_int32), ("nr", ct.c_int32),
        ("T", ct.c_int64), ("K", ct.c_int32),
        ("t", ct.c_void_p),
        ("F", lqt_coef), ("L", lqt_coef), ("c", lqt_coef), ("H", lqt_coef), ("X", lqt_coef), ("U", lqt_coef),
        ("r", lqt_coef),
        ("Hf", ct.c_void_p), ("Xf", ct.c_void_p), ("rf", ct.c_void_p),
    ]


class lqt_elements(ct.Structure):
    _fields_ = [("A", ct.c_void_p), ("b", ct.c_void_p), ("C", ct.c_void_p), ("eta", ct.c_void_p),
                ("J", ct.c_void_p), ("zeta", ct.c_void_p)]


class lqt_batch(ct.Structure):
    _fields_ = [("count", ct.c_int32), ("problems", ct.POINTER(lqt_problem)), ("x0", ct.POINTER(ct.c_void_p))]


class lqt_tuning(ct.Structure):
    _fields_ = [("chunk", ct.c_int32), ("flags", ct.c_int32)]


class lqt_grid_problem(ct.Structure):
    _fields_ = [("G", ct.c_int32), ("x_min", ct.c_double), ("dx", ct.c_double), ("d0", ct.c_double),
                ("d1", ct.c_double), ("d2", ct.c_double), ("q", ct.c_double), ("rho", ct.c_double),
                ("qf", ct.c_double), ("tau", ct.c_double), ("substeps", ct.c_int32), ("T", ct.c_int64),
                ("interp", ct.c_int32)]


class LQTError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} (status {code})")


_lib = None


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"LQT CUDA library not built ({LIB_PATH} missing); run __graft_entry__.build()")
    L = ct.CDLL(LIB_PATH)
    P = ct.POINTER(lqt_problem)
    E = ct.POINTER(lqt_elements)
    v = ct.c_void_p
    L.lqt_workspace_size.argtypes = [P, ct.c_int32]
    L.lqt_workspace_size.restype = ct.c_size_t
    L.lqt_build_elements.argtypes = [P, E, v, ct.c_size_t, v]
    L.lqt_scan_value.argtypes = [P, E, v, v, v, v, ct.c_size_t, v]
    L.lqt_scan_trajectory.argtypes = [P, E, v, v, v, v, v, v, ct.c_size_t, v]
    L.lqt_solve.argtypes = [P, v, v, v, v, v, v, v, v, ct.c_size_t, v]
    L.lqt_solve_sequential.argtypes = [P, v, v, v, v, v, v, v, v, ct.c_size_t, v]
    L.lqt_densify.argtypes = [P, v, v, v, v, v, v, v, v, v, v, ct.c_size_t, v]
    L.lqt_build_elements_forward.argtypes = [P, ct.POINTER(lqt_elements), v, ct.c_size_t, v]
    L.lqt_trajectory_method2.argtypes = [P, ct.POINTER(lqt_elements), v, v, v, v, v, v, ct.c_size_t, v]
    L.lqt_solve_method2.argtypes = [P, v, v, v, v, v, v, v, v, ct.c_size_t, v]
    L.lqt_build_elements_invariant.argtypes = [P, ct.POINTER(lqt_elements), v, ct.c_size_t, v]
    L.lqt_solve_invariant.argtypes = [P, v, v, v, v, v, v, v, v, ct.c_size_t, v]
    L.lqt_solve_mixed.argtypes = [P, v, v, v, v, v, v, v, v, ct.c_size_t, v]
    L.lqt_solve_mixed.restype = ct.c_int
    L.lqt_host_staging_size.argtypes = [P]
    L.lqt_host_staging_size.restype = ct.c_size_t
    L.lqt_solve_host.argtypes = [P, v, v, v, v, v, v, v, v, ct.c_size_t, v]
    L.lqt_get_status.argtypes = [v, ct.c_int32]
    L.lqt_strerror.argtypes = [ct.c_int]
    L.lqt_strerror.restype = ct.c_char_p
    L.lqt_backward.argtypes = [P, v, v, v, v, v, v, v, v, v, ct.c_double, v, v, v, v, v, v, v, v, v, ct.c_size_t, v]
    L.lqt_backward.restype = ct.c_int
    Bp = ct.POINTER(lqt_batch)
    L.lqt_batch_workspace_size.argtypes = [Bp]
    L.lqt_batch_workspace_size.restype = ct.c_size_t
    L.lqt_batch_boundaries.argtypes = [Bp]
    L.lqt_batch_boundaries.restype = ct.c_int64
    L.lqt_batch_plan.argtypes = [Bp, v, ct.c_size_t, v]
    L.lqt_batch_plan.restype = ct.c_int
    L.lqt_solve_batched.argtypes = [Bp, ct.POINTER(lqt_tuning), v, v, v, v, v, v, v, ct.c_size_t, v]
    L.lqt_solve_batched.restype = ct.c_int
    L.lqt_scan_value_noalloc.argtypes = [P, E, v, v, v, v]
    L.lqt_scan_value_noalloc.restype = ct.c_int
    GP = ct.POINTER(lqt_grid_problem)
    L.lqt_grid_workspace_size.argtypes = [GP, ct.c_int32]
    L.lqt_grid_workspace_size.restype = ct.c_size_t
    L.lqt_grid_block.argtypes = [GP, v, v, ct.c_size_t, v]
    L.lqt_grid_combine.argtypes = [GP, v, v, v, v]
    L.lqt_grid_values.argtypes = [GP, v, v, v, ct.c_size_t, v]
    L.lqt_probe_fma_rate.argtypes = [ct.c_int32, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_int32, v, v]
    L.lqt_probe_fma_rate.restype = ct.c_int
    L.lqt_last_launch_count.argtypes = []
    L.lqt_last_launch_count.restype = ct.c_int32
    for f in ("lqt_build_elements", "lqt_scan_value", "lqt_scan_trajectory", "lqt_solve", "lqt_solve_sequential",
              "lqt_densify", "lqt_build_elements_forward", "lqt_trajectory_method2", "lqt_solve_method2",
              "lqt_build_elements_invariant", "lqt_solve_invariant", "lqt_grid_block", "lqt_grid_combine",
              "lqt_grid_values", "lqt_solve_host", "lqt_get_status"):
        getattr(L, f).restype = ct.c_int
    _lib = L
    return L


def strerror(code: int) -> str:
    try:
        return lib().lqt_strerror(code).decode()
    except RuntimeError:
        return f"status {code}"


def check(code: int, where: str):
    if code != LQT_OK:
        raise LQTError(code, where)
