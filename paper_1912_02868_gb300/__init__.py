"""GB300-native deflated multigrid solver for the 2D Schwinger-model Wilson-Dirac
operator (Whyte, Wilcox, Morgan, arXiv:1912.02868).

The solver is the C ABI of libmg.so (include/mg.h); this package is a thin
binding with the same names.  Arrays may be torch tensors (CUDA or pinned host)
or numpy arrays (host); they are passed to the library by pointer.  Complex
arrays are complex128 (complex64 for the FP32 operator-level calls).
"""
from __future__ import annotations

import atexit
import ctypes
import sys
import weakref

import numpy as np

from . import _lib
from ._lib import (MG_COARSE_CGNE, MG_COARSE_DR_PROJ, MG_F32, MG_F64, MG_BF16, MG_F16, MG_FP64, MG_MIXED,  # noqa: F401
                   MG_MIXED_BF16, MG_MIXED_FP16, MG_OK,
                   MG_METHOD_MG, MG_METHOD_FINE_DEFLATION, MG_METHOD_FINE_CGNE,
                   MG_ENOTCONV, MG_ETIMEOUT, MG_COARSE_PROBE_TIMEOUT, MGError, MGParams, MGSolveStats, load)

__all__ = ["build", "default_params", "mg_setup", "mg_setup_from_vectors", "mg_solve", "mg_destroy",
           "mg_reset_deflation", "mg_apply", "mg_restrict", "mg_prolong", "mg_get_stencil",
           "mg_get_prolongator", "mg_get_deflation", "mg_level_shape", "mg_stencil_info", "mg_launch_shape",
           "mg_set_launch_shape", "mg_wilson_apply", "mg_timing_enable",
           "mg_timing_read", "mg_kernel_launches", "mg_wilson_residual_noalloc", "mg_set_deflation",
           "mg_coarse_solve", "mg_apply_block", "Handle"]


def build(force: bool = False) -> str:
    from .nvcc_build import build as _build
    return _build(force=force)


def _ptr(a):
    """Data pointer of a torch tensor / numpy array (must be contiguous), or None."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"cannot pass {type(a)} as a pointer")


def _stream(stream, *arrays):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    for a in arrays:
        if hasattr(a, "is_cuda") and a.is_cuda:
            import torch
            return torch.cuda.current_stream(a.device).cuda_stream
    return None


def default_params(**overrides) -> MGParams:
    p = MGParams()
    _lib.check(load().mg_default_params(ctypes.byref(p)), "mg_default_params")
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


# Handles and servers not yet closed.  An exit hook closes them, servers first
# (their workers solve on handles they own), while the interpreter and the CUDA
# runtime are still whole: exit hooks run before the interpreter tears its
# modules down and before the C runtime's static destructors.  A destructor that
# runs during interpreter finalization does not call into the library.
_live = weakref.WeakSet()


def _close_live():
    for o in sorted(list(_live), key=lambda o: 0 if isinstance(o, Server) else 1):
        try:
            o.close()
        except Exception:
            pass


atexit.register(_close_live)


class Handle:
    """Owner of an mg_handle; mg_destroy runs on close(), at garbage collection
    or at interpreter exit."""

    def __init__(self, ptr: int, Lx: int, Lt: int, params: MGParams):
        self.ptr = ptr
        self.Lx, self.Lt = Lx, Lt
        self.params = params
        _live.add(self)

    def close(self):
        if self.ptr:
            load().mg_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def mg_setup(gauge, Lx, Lt, m0, nvec=12, block=4, params=None, starts0=None, starts1=None, stream=None) -> Handle:
    p = params or default_params()
    out = ctypes.c_void_p()
    st = load().mg_setup(_ptr(gauge), Lx, Lt, float(m0), nvec, block, ctypes.byref(p), _ptr(starts0),
                         _ptr(starts1), _stream(stream, gauge), ctypes.byref(out))
    _lib.check(st, "mg_setup")
    return Handle(out.value, Lx, Lt, p)


def mg_setup_from_vectors(gauge, Lx, Lt, m0, nullvecs0, nullvecs1, nvec=12, block=4, params=None,
                          stream=None) -> Handle:
    p = params or default_params()
    out = ctypes.c_void_p()
    st = load().mg_setup_from_vectors(_ptr(gauge), Lx, Lt, float(m0), nvec, block, ctypes.byref(p),
                                      _ptr(nullvecs0), _ptr(nullvecs1), _stream(stream, gauge), ctypes.byref(out))
    _lib.check(st, "mg_setup_from_vectors")
    return Handle(out.value, Lx, Lt, p)


def mg_solve(h: Handle, b, x, nrhs, tol, stream=None, allow_notconv=False):
    """Returns (status, iters[nrhs], relres[nrhs], stats dict)."""
    iters = (ctypes.c_int * max(nrhs, 1))()
    relres = (ctypes.c_double * max(nrhs, 1))()
    stats = MGSolveStats()
    st = load().mg_solve(h.ptr, _ptr(b), _ptr(x), nrhs, float(tol), _stream(stream, b, x), iters, relres,
                         ctypes.byref(stats))
    _lib.check(st, "mg_solve", allow=(MG_OK, MG_ENOTCONV) if allow_notconv else (MG_OK,))
    sd = {"mvps": list(stats.mvps), "fine_equiv_mvps": stats.fine_equiv_mvps, "outer_iters": stats.outer_iters,
          "coarse_solves": stats.coarse_solves, "coarse_iters": stats.coarse_iters, "dr_solves": stats.dr_solves}
    return st, list(iters)[:nrhs], list(relres)[:nrhs], sd


def mg_destroy(h: Handle):
    h.close()


def mg_reset_deflation(h: Handle):
    _lib.check(load().mg_reset_deflation(h.ptr), "mg_reset_deflation")


def mg_apply(h: Handle, level, x, y, dagger=False, precision=MG_F64, stream=None):
    _lib.check(load().mg_apply(h.ptr, level, int(dagger), precision, _ptr(x), _ptr(y), _stream(stream, x)),
               "mg_apply")


def mg_apply_block(h: Handle, level, x, y, nrhs, precision=MG_BF16, stream=None):
    """y[r] = D^ x[r] on grid 1 or 2 for nrhs (a multiple of 8) complex64 vectors, tensor cores."""
    _lib.check(load().mg_apply_block(h.ptr, level, precision, nrhs, _ptr(x), _ptr(y), _stream(stream, x)),
               "mg_apply_block")


def mg_restrict(h: Handle, level, fine, coarse, precision=MG_F64, stream=None):
    _lib.check(load().mg_restrict(h.ptr, level, precision, _ptr(fine), _ptr(coarse), _stream(stream, fine)),
               "mg_restrict")


def mg_prolong(h: Handle, level, coarse, fine, precision=MG_F64, stream=None):
    _lib.check(load().mg_prolong(h.ptr, level, precision, _ptr(coarse), _ptr(fine), _stream(stream, coarse)),
               "mg_prolong")


def mg_level_shape(h: Handle, level):
    nx, nt, dof = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _lib.check(load().mg_level_shape(h.ptr, level, ctypes.byref(nx), ctypes.byref(nt), ctypes.byref(dof)),
               "mg_level_shape")
    return nx.value, nt.value, dof.value


def mg_stencil_info(h: Handle, level):
    """(factored, max_rel_err): whether `level` applies rank-4 hop factors."""
    f, e = ctypes.c_int(), ctypes.c_double()
    _lib.check(load().mg_stencil_info(h.ptr, level, ctypes.byref(f), ctypes.byref(e)), "mg_stencil_info")
    return bool(f.value), e.value


def mg_launch_shape(h: Handle, level, precision=MG_F32):
    """(shape, us_chosen, us_builtin): the launch shape the set-up's autotuner chose
    for `level`'s apply in `precision` (0 = the built-in shape) and the times of one
    apply with it and with the built-in shape."""
    sh, us = ctypes.c_int(), (ctypes.c_double * 2)()
    _lib.check(load().mg_launch_shape(h.ptr, level, precision, ctypes.byref(sh), us), "mg_launch_shape")
    return sh.value, us[0], us[1]


def mg_set_launch_shape(h: Handle, level, precision, shape):
    """Pin the launch shape of `level`'s apply in `precision` (0 = built-in)."""
    _lib.check(load().mg_set_launch_shape(h.ptr, level, precision, shape), "mg_set_launch_shape")


def mg_get_stencil(h: Handle, level) -> np.ndarray:
    nx, nt, dof = mg_level_shape(h, level)
    out = np.empty((nt, nx, 5, dof, dof), dtype=np.complex128)
    _lib.check(load().mg_get_stencil(h.ptr, level, _ptr(out)), "mg_get_stencil")
    return out


def mg_get_prolongator(h: Handle, level) -> np.ndarray:
    nxc, ntc, _ = mg_level_shape(h, level + 1)
    hh = 1 if level == 0 else 12
    out = np.empty((ntc, nxc, 2, 12, 16, hh), dtype=np.complex128)
    _lib.check(load().mg_get_prolongator(h.ptr, level, _ptr(out)), "mg_get_prolongator")
    return out


def mg_get_deflation(h: Handle):
    """(W complex128[k+1][n2], H complex128[k+1][k]) or (None, None) before the first coarse solve."""
    k = ctypes.c_int()
    lib = load()
    _lib.check(lib.mg_get_deflation(h.ptr, None, None, ctypes.byref(k)), "mg_get_deflation")
    if k.value == 0:
        return None, None
    nx, nt, dof = mg_level_shape(h, 2)
    W = np.empty((k.value + 1, nx * nt * dof), dtype=np.complex128)
    Hm = np.empty((k.value + 1, k.value), dtype=np.complex128)
    _lib.check(lib.mg_get_deflation(h.ptr, _ptr(W), _ptr(Hm), ctypes.byref(k)), "mg_get_deflation")
    return W, Hm


def mg_set_deflation(h: Handle, W, Hm):
    """Load a deflation space: W complex128[k+1][n2] rows, Hm complex128[k+1][k] (host or device)."""
    k = int(Hm.shape[1])
    _lib.check(load().mg_set_deflation(h.ptr, _ptr(W), _ptr(Hm), k), "mg_set_deflation")


def mg_coarse_solve(h: Handle, b, x, tol, precision=MG_F64, nrhs=1, flags=0, spin=0, stream=None,
                    allow=(MG_OK,)):
    """One projected coarse solve (device b, x [nrhs][n2]).  Returns
    (status, iters[nrhs], converged[nrhs], info dict)."""
    iters = (ctypes.c_longlong * nrhs)()
    conv = (ctypes.c_int * nrhs)()
    info = _lib.MGCoarseInfo()
    st = load().mg_coarse_solve(h.ptr, precision, nrhs, _ptr(b), _ptr(x), float(tol), int(flags), int(spin),
                                _stream(stream, b, x), iters, conv, ctypes.byref(info))
    _lib.check(st, "mg_coarse_solve", allow=allow)
    return st, list(iters), [bool(c) for c in conv], {f: getattr(info, f) for f, _ in info._fields_}


def mg_wilson_apply(gauge, Lx, Lt, m0, x, y, dagger=False, precision=MG_F64, stream=None):
    _lib.check(load().mg_wilson_apply(_ptr(gauge), Lx, Lt, float(m0), int(dagger), precision, _ptr(x), _ptr(y),
                                      _stream(stream, x)), "mg_wilson_apply")


def mg_wilson_residual_noalloc(gauge, Lx, Lt, m0, b, x, r, stream=None):
    """r = b - D x on the device; returns (||b - D x||, ||b||).  Allocates no device memory."""
    norms = (ctypes.c_double * 2)()
    _lib.check(load().mg_wilson_residual_noalloc(_ptr(gauge), Lx, Lt, float(m0), _ptr(b), _ptr(x), _ptr(r), norms,
                                                 _stream(stream, b)), "mg_wilson_residual_noalloc")
    return norms[0], norms[1]


def mg_timing_enable(h: Handle, level, enable=True):
    _lib.check(load().mg_timing_enable(h.ptr, level, int(enable)), "mg_timing_enable")


def mg_timing_read(h: Handle, level):
    """(total milliseconds, number of applies) of the timed applies on `level`."""
    ms, n = ctypes.c_double(), ctypes.c_longlong()
    _lib.check(load().mg_timing_read(h.ptr, level, ctypes.byref(ms), ctypes.byref(n)), "mg_timing_read")
    return ms.value, n.value


def mg_kernel_launches() -> int:
    return int(load().mg_kernel_launches())


class Server:
    """Continuous-batching solve server (mg_server_*): requests over many operators
    (keys) share the GPU; hierarchies are cached under an HBM byte budget."""

    def __init__(self, params=None, hbm_budget_bytes=0, workers=8):
        self.params = params or default_params()
        out = ctypes.c_void_p()
        _lib.check(load().mg_server_create(ctypes.byref(self.params), int(hbm_budget_bytes), int(workers),
                                           ctypes.byref(out)), "mg_server_create")
        self.ptr = out.value
        _live.add(self)
        self._keep = {}

    def submit(self, key, gauge, Lx, Lt, m0, b, x, nrhs, tol, starts0=None, starts1=None) -> int:
        r = _lib.MGRequest(key=int(key), gauge=_ptr(gauge), L_x=Lx, L_t=Lt, m0=float(m0), starts0=_ptr(starts0),
                           starts1=_ptr(starts1), b=_ptr(b), x=_ptr(x), nrhs=int(nrhs), tol=float(tol))
        t = ctypes.c_ulonglong()
        _lib.check(load().mg_server_submit(self.ptr, ctypes.byref(r), ctypes.byref(t)), "mg_server_submit")
        self._keep[t.value] = (gauge, b, x, starts0, starts1)  # the arrays must outlive the request
        return t.value

    def wait(self, ticket, nrhs, allow_notconv=False):
        """(status, iters[nrhs], relres[nrhs], latency seconds)"""
        it = (ctypes.c_int * nrhs)()
        rr = (ctypes.c_double * nrhs)()
        lat = ctypes.c_double()
        st = load().mg_server_wait(self.ptr, int(ticket), it, rr, ctypes.byref(lat))
        self._keep.pop(ticket, None)
        _lib.check(st, "mg_server_wait", allow=(MG_OK, MG_ENOTCONV) if allow_notconv else (MG_OK,))
        return st, list(it), list(rr), lat.value

    def poll(self, ticket, nrhs, allow_notconv=False):
        """None while the request runs; then (status, iters, relres, latency) as wait()."""
        done = ctypes.c_int()
        it = (ctypes.c_int * nrhs)()
        rr = (ctypes.c_double * nrhs)()
        lat = ctypes.c_double()
        st = load().mg_server_poll(self.ptr, int(ticket), ctypes.byref(done), it, rr, ctypes.byref(lat))
        if st == MG_OK and not done.value:
            return None
        self._keep.pop(ticket, None)
        _lib.check(st, "mg_server_poll", allow=(MG_OK, MG_ENOTCONV) if allow_notconv else (MG_OK,))
        return st, list(it), list(rr), lat.value

    def stats(self) -> dict:
        info = _lib.MGServerInfo()
        _lib.check(load().mg_server_stats(self.ptr, ctypes.byref(info)), "mg_server_stats")
        return {f: getattr(info, f) for f, _ in info._fields_}

    def close(self):
        if self.ptr:
            load().mg_server_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
