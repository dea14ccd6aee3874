"""ctypes binding of libmg.so: the entry points of include/mg.h under the same
names.  Argument marshalling only: every step of a setup or a solve runs in the
library's CUDA kernels.  There is no fallback: if libmg.so is missing or cannot
be loaded, loading raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmg.so")

MG_OK, MG_EINVAL, MG_ENOMEM, MG_ECUDA, MG_ENOTCONV, MG_EBUDGET, MG_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
MG_COARSE_DR_PROJ, MG_COARSE_CGNE = 0, 1
MG_FP64, MG_MIXED, MG_MIXED_BF16, MG_MIXED_FP16 = 0, 1, 2, 3
MG_F64, MG_F32, MG_BF16, MG_F16 = 0, 1, 2, 3
MG_METHOD_MG, MG_METHOD_FINE_DEFLATION, MG_METHOD_FINE_CGNE = 0, 1, 2

STATUS_NAMES = {0: "MG_OK", -1: "MG_EINVAL", -2: "MG_ENOMEM", -3: "MG_ECUDA", -4: "MG_ENOTCONV",
                -5: "MG_EBUDGET", -6: "MG_ETIMEOUT"}


class MGParams(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int), ("block", ctypes.c_int), ("nvec", ctypes.c_int),
        ("smooth_steps", ctypes.c_int), ("fgmres_m", ctypes.c_int), ("max_outer", ctypes.c_int),
        ("coarse_solver", ctypes.c_int), ("dr_m", ctypes.c_int), ("dr_k", ctypes.c_int),
        ("dr_max_cycles", ctypes.c_int), ("dr_stall_cycles", ctypes.c_int), ("proj_max_cycles", ctypes.c_int),
        ("cgne_max_iters", ctypes.c_int), ("nullvec_max_iters", ctypes.c_int),
        ("nullvec_tol", ctypes.c_double), ("coarse_tol_first", ctypes.c_double),
        ("coarse_tol_rest", ctypes.c_double), ("precision", ctypes.c_int), ("seed", ctypes.c_ulonglong),
        ("method", ctypes.c_int), ("parallel", ctypes.c_int), ("partial_tol", ctypes.c_double),
        ("coarse_tol_partial", ctypes.c_double), ("partial_max_iters", ctypes.c_int), ("pair_rhs", ctypes.c_int),
        ("vcycle_graph", ctypes.c_int), ("coarse_half", ctypes.c_int),
        ("coarse_dcgs2", ctypes.c_int), ("rhs_block", ctypes.c_int), ("lowrank_hops", ctypes.c_int),
        ("autotune", ctypes.c_int), ("coarse_mma", ctypes.c_int),
    ]


class MGSolveStats(ctypes.Structure):
    _fields_ = [
        ("mvps", ctypes.c_longlong * 3), ("fine_equiv_mvps", ctypes.c_double), ("outer_iters", ctypes.c_int),
        ("coarse_solves", ctypes.c_int), ("coarse_iters", ctypes.c_longlong), ("dr_solves", ctypes.c_int),
    ]


class MGRequest(ctypes.Structure):
    _fields_ = [
        ("key", ctypes.c_ulonglong), ("gauge", ctypes.c_void_p), ("L_x", ctypes.c_int), ("L_t", ctypes.c_int),
        ("m0", ctypes.c_double), ("starts0", ctypes.c_void_p), ("starts1", ctypes.c_void_p),
        ("b", ctypes.c_void_p), ("x", ctypes.c_void_p), ("nrhs", ctypes.c_int), ("tol", ctypes.c_double),
    ]


class MGServerInfo(ctypes.Structure):
    _fields_ = [
        ("resident_keys", ctypes.c_int), ("device_bytes", ctypes.c_ulonglong), ("evictions", ctypes.c_longlong),
        ("cold_starts", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("queued_items", ctypes.c_longlong),
        ("batches", ctypes.c_longlong), ("max_batch", ctypes.c_int), ("demand_bytes", ctypes.c_ulonglong),
    ]


class MGCoarseInfo(ctypes.Structure):
    _fields_ = [
        ("ctas", ctypes.c_int), ("sites_per_cta", ctypes.c_int), ("dataflow", ctypes.c_int), ("dcgs2", ctypes.c_int),
        ("half_operator", ctypes.c_int), ("shared_blocks", ctypes.c_int), ("paired", ctypes.c_int),
        ("cycles", ctypes.c_longlong), ("timeouts", ctypes.c_longlong), ("tensor_apply", ctypes.c_int),
    ]


MG_COARSE_PROBE_TIMEOUT = 1

_lib = None

# every symbol declared in include/mg.h
SYMBOLS = ("mg_default_params", "mg_setup", "mg_setup_from_vectors", "mg_solve", "mg_reset_deflation",
           "mg_destroy", "mg_last_error", "mg_apply", "mg_restrict", "mg_prolong", "mg_get_stencil",
           "mg_get_prolongator", "mg_get_deflation", "mg_level_shape", "mg_stencil_info", "mg_launch_shape",
           "mg_set_launch_shape",
           "mg_wilson_apply", "mg_timing_enable", "mg_timing_read", "mg_kernel_launches", "mg_server_create",
           "mg_server_submit",
           "mg_server_wait", "mg_server_poll", "mg_server_stats", "mg_server_destroy", "mg_wilson_residual_noalloc",
           "mg_set_deflation", "mg_coarse_solve", "mg_apply_block")


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libmg.so (raises if it is missing: there is no CPU fallback)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"{p} is missing: build it with paper_1912_02868_gb300.build()")
    lib = ctypes.CDLL(p)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "mg_default_params": (i, [ctypes.POINTER(MGParams)]),
        "mg_setup": (i, [vp, i, i, d, i, i, ctypes.POINTER(MGParams), vp, vp, vp, ctypes.POINTER(vp)]),
        "mg_setup_from_vectors": (i, [vp, i, i, d, i, i, ctypes.POINTER(MGParams), vp, vp, vp, ctypes.POINTER(vp)]),
        "mg_solve": (i, [vp, vp, vp, i, d, vp, ctypes.POINTER(i), ctypes.POINTER(d), ctypes.POINTER(MGSolveStats)]),
        "mg_reset_deflation": (i, [vp]),
        "mg_destroy": (i, [vp]),
        "mg_last_error": (ctypes.c_char_p, []),
        "mg_apply": (i, [vp, i, i, i, vp, vp, vp]),
        "mg_restrict": (i, [vp, i, i, vp, vp, vp]),
        "mg_prolong": (i, [vp, i, i, vp, vp, vp]),
        "mg_get_stencil": (i, [vp, i, vp]),
        "mg_get_prolongator": (i, [vp, i, vp]),
        "mg_get_deflation": (i, [vp, vp, vp, ctypes.POINTER(i)]),
        "mg_level_shape": (i, [vp, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]),
        "mg_stencil_info": (i, [vp, i, ctypes.POINTER(i), ctypes.POINTER(ctypes.c_double)]),
        "mg_launch_shape": (i, [vp, i, i, ctypes.POINTER(i), ctypes.POINTER(ctypes.c_double)]),
        "mg_set_launch_shape": (i, [vp, i, i, i]),
        "mg_wilson_apply": (i, [vp, i, i, d, i, i, vp, vp, vp]),
        "mg_timing_enable": (i, [vp, i, i]),
        "mg_timing_read": (i, [vp, i, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_longlong)]),
        "mg_kernel_launches": (ctypes.c_ulonglong, []),
        "mg_server_create": (i, [ctypes.POINTER(MGParams), ctypes.c_ulonglong, i, ctypes.POINTER(vp)]),
        "mg_server_submit": (i, [vp, ctypes.POINTER(MGRequest), ctypes.POINTER(ctypes.c_ulonglong)]),
        "mg_server_wait": (i, [vp, ctypes.c_ulonglong, ctypes.POINTER(i), ctypes.POINTER(d), ctypes.POINTER(d)]),
        "mg_server_poll": (i, [vp, ctypes.c_ulonglong, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(d),
                               ctypes.POINTER(d)]),
        "mg_server_stats": (i, [vp, ctypes.POINTER(MGServerInfo)]),
        "mg_set_deflation": (i, [vp, vp, vp, i]),
        "mg_apply_block": (i, [vp, i, i, i, vp, vp, vp]),
        "mg_coarse_solve": (i, [vp, i, i, vp, vp, d, i, ctypes.c_longlong, vp, ctypes.POINTER(ctypes.c_longlong),
                                ctypes.POINTER(i), ctypes.POINTER(MGCoarseInfo)]),
        "mg_server_destroy": (i, [vp]),
        "mg_wilson_residual_noalloc": (i, [vp, i, i, d, vp, vp, vp, ctypes.POINTER(d), vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = lib
    return lib


class MGError(RuntimeError):
    def __init__(self, status, where):
        msg = load().mg_last_error()
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg.decode() if msg else ''}")
        self.status = status


def check(status, where, allow=(MG_OK,)):
    if status not in allow:
        raise MGError(status, where)
    return status
