"""ctypes declarations of the C interface in ``include/kkt.h``.

Argument marshalling only: every computation happens inside ``libkkt.so``.
Loading fails loudly when the library has not been built; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

KKT_OK = 0
KKT_ERR_ARG = 1
KKT_ERR_PATTERN = 2
KKT_ERR_ALLOC = 3
KKT_ERR_CUDA = 4
KKT_ERR_NONFINITE = 5
KKT_ERR_NOT_CONVERGED = 6
KKT_ERR_TIMEOUT = 7
KKT_ERR_STATE = 8
KKT_ERR_INTERNAL = 9
KKT_WARN_PERTURBED = 100

ORDER_AMD, ORDER_NATURAL, ORDER_USER = 0, 1, 2
REFINE_CLASSIC, REFINE_FGMRES, REFINE_AUTO, REFINE_FGMRES_JACOBI = 0, 1, 2, 3


class Options(C.Structure):
    _fields_ = [
        ("factor_fp32", C.c_int),
        ("equilibrate", C.c_int),
        ("ordering", C.c_int),
        ("user_perm", C.POINTER(C.c_int)),
        ("refine_mode", C.c_int),
        ("fgmres_restart", C.c_int),
        ("max_refine", C.c_int),
        ("tol", C.c_double),
        ("pivot_tau_rel", C.c_double),
        ("spin_limit", C.c_longlong),
        ("device", C.c_int),
        ("max_batch", C.c_int),
        ("cta_warps", C.c_int),
        ("refactor_ctas", C.c_int),
        ("solve_ctas", C.c_int),
        ("update_map_budget", C.c_size_t),
        ("trace", C.c_int),
        ("poll_ns_max", C.c_int),
        ("unpublished_row", C.c_int),
        ("refactor_big_warps", C.c_int),
        ("symmetric", C.c_int),
        ("jacobi_sweeps", C.c_int),
        ("user_row_perm", C.POINTER(C.c_int)),
        ("dense_block", C.c_int),
        ("refactor_row_cap", C.c_int),
        ("refine_auto_ratio", C.c_double),
        ("solve_far_blocks", C.c_int),
        ("solve_far_ctas", C.c_int),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("n", C.c_int),
        ("nnz_a", C.c_longlong),
        ("nnz_sym", C.c_longlong),
        ("nnz_lu", C.c_longlong),
        ("n_levels", C.c_int),
        ("n_levels_u", C.c_int),
        ("max_row", C.c_int),
        ("flops_refactor", C.c_double),
        ("bytes_refactor", C.c_double),
        ("bytes_solve", C.c_double),
        ("bytes_spmv", C.c_double),
        ("device_bytes", C.c_size_t),
        ("grid_ctas", C.c_int),
        ("solve_ctas", C.c_int),
        ("warps_per_cta", C.c_int),
        ("last_refine_iters", C.c_int),
        ("last_omega", C.c_double),
        ("factor_fp32", C.c_int),
        ("kernel_launches", C.c_longlong),
        ("update_map_entries", C.c_longlong),
        ("n_tasks", C.c_int),
        ("max_task", C.c_int),
        ("refactor_big_warps", C.c_int),
        ("refactor_big_cap", C.c_int),
        ("dense_rows", C.c_int),
        ("refactor_row_cap", C.c_int),
        ("solve_far_rows", C.c_int),
        ("solve_far_ctas", C.c_int),
    ]


class RefineInfo(C.Structure):
    _fields_ = [
        ("iters", C.c_int),
        ("converged", C.c_int),
        ("omega", C.c_double),
        ("omega_hist", C.c_double * 64),
        ("n_hist", C.c_int),
    ]


# name -> (restype, argtypes); every function declared in include/kkt.h
_vp = C.c_void_p
_ip = C.POINTER(C.c_int)
SIGNATURES = {
    "kkt_default_options": (None, [C.POINTER(Options)]),
    "kkt_status_string": (C.c_char_p, [C.c_int]),
    "kkt_last_error": (C.c_char_p, []),
    "kkt_analyze": (C.c_int, [C.c_int, _ip, _ip, C.POINTER(Options), C.POINTER(_vp)]),
    "kkt_destroy": (None, [_vp]),
    "kkt_refactor": (C.c_int, [_vp, _vp, _vp]),
    "kkt_solve": (C.c_int, [_vp, _vp, _vp, _vp]),
    "kkt_solve_transpose": (C.c_int, [_vp, _vp, _vp, _vp]),
    "kkt_refine": (C.c_int, [_vp, _vp, _vp, C.c_double, C.c_int, C.POINTER(RefineInfo), _vp]),
    "kkt_refine_transpose": (C.c_int, [_vp, _vp, _vp, C.c_double, C.c_int, C.POINTER(RefineInfo), _vp]),
    "kkt_adjoint_gather": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "kkt_status_sync": (C.c_int, [_vp, _vp, _ip]),
    "kkt_get_stats": (C.c_int, [_vp, C.POINTER(Stats)]),
    "kkt_export_symbolic": (C.c_int, [_vp, _ip, _ip, _ip, _ip, _ip]),
    "kkt_export_factors": (C.c_int, [_vp, _vp, _vp]),
    "kkt_export_scaling": (C.c_int, [_vp, _vp, _vp]),
    "kkt_export_trace": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_ulonglong), C.c_longlong,
                                   C.POINTER(C.c_longlong)]),
    "kkt_batch_refactor": (C.c_int, [_vp, C.c_int, _vp, _vp]),
    "kkt_batch_solve": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp]),
    "kkt_batch_solve_transpose": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp]),
    "kkt_batch_refine": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_double, C.c_int, C.POINTER(C.c_double),
                                   C.POINTER(C.c_int), _vp]),
    "kkt_batch_refine_transpose": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_double, C.c_int,
                                             C.POINTER(C.c_double), C.POINTER(C.c_int), _vp]),
    "kkt_batch_export_factors": (C.c_int, [_vp, C.c_int, _vp, _vp]),
    "kkt_queue_create": (C.c_int, [C.POINTER(_vp), C.c_int, C.POINTER(_vp)]),
    "kkt_queue_destroy": (None, [_vp]),
    "kkt_queue_set_launch": (C.c_int, [_vp, C.c_int, C.c_int]),
    "kkt_queue_set_tiles": (C.c_int, [_vp, C.c_int]),
    "kkt_queue_run": (C.c_int, [_vp, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp), C.c_int, _vp, _vp]),
    "kkt_queue_solve_transpose": (C.c_int, [_vp, C.POINTER(_vp), C.POINTER(_vp), _vp]),
    "kkt_queue_status_sync": (C.c_int, [_vp, _vp, _ip]),
    "kkt_scaled_residual_noalloc": (C.c_int, [C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "kkt_probe_fma_tflops": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_double)]),
    "kkt_inertia": (C.c_int, [_vp, _vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "kkt_solve_jacobi": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int, _vp]),
    "kkt_analyze_values": (C.c_int, [C.c_int, _ip, _ip, C.POINTER(C.c_double), C.POINTER(Options),
                                     C.POINTER(_vp)]),
    "kkt_export_row_perm": (C.c_int, [_vp, _ip]),
    "kkt_export_dense_rows": (C.c_int, [_vp, _ip]),
    "kkt_save_analysis": (C.c_int, [_vp, _vp, C.c_size_t, C.POINTER(C.c_size_t)]),
    "kkt_load_analysis": (C.c_int, [_vp, C.c_size_t, C.POINTER(Options), C.POINTER(_vp)]),
}

_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libkkt.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                _build.build()
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library not built: {path}")
            L = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


class KKTError(RuntimeError):
    def __init__(self, status, where):
        L = load(False)
        msg = L.kkt_status_string(status).decode()
        detail = L.kkt_last_error().decode()
        super().__init__(f"{where}: {msg} ({status})" + (f": {detail}" if detail else ""))
        self.status = status


def check(status, where, allow=()):
    if status != KKT_OK and status not in allow:
        raise KKTError(status, where)
    return status
