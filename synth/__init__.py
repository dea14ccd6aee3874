"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module holds no arithmetic of the solver.  It makes:

* quenched U(1) gauge fields at beta = 6.0 from a deterministic heatbath
  (``heatbath.c``), standing in for the paper's QCDLAB configurations
  (Section 2, "Methods": 10 configurations per lattice size at beta = 6.0);
  ``heatbath_gpu.cu`` is the same generator on the GPU, bit-identical to it,
  for the large lattices a benchmark needs in seconds;
* complex-Gaussian right-hand sides and null-vector start vectors
  (E|z|^2 = 1, i.e. real and imaginary parts each N(0, 1/2));
* Z(4) noise (the paper's right-hand sides, Section 2) as an option;
* the tuned bare mass m0 per configuration, read from ``m0_table.json``
  (written by ``oracle/tune_m0.py``; it puts the smallest real part of the
  spectrum of D at 1e-3).

Gauge layout: complex128[L_t][L_x][2], mu = 0 is x, mu = 1 is t.
Spinor layout: complex128[L_t][L_x][2] (site = x + L_x t, spin fastest).
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_heatbath.so")
_SRC = os.path.join(_HERE, "heatbath.c")
_SO_GPU = os.path.join(_HERE, "_heatbath_gpu.so")
_SRC_GPU = os.path.join(_HERE, "heatbath_gpu.cu")
_lock = threading.Lock()
_lib = None
_lib_gpu = None

BETA = 6.0


def build(force: bool = False) -> str:
    """Compile the heatbath library in place (gcc, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def build_gpu(force: bool = False) -> str | None:
    """Compile the GPU heatbath in place (nvcc, sm_103a, no FMA contraction);
    None when no CUDA toolkit is installed."""
    cc = _nvcc()
    if cc is None:
        return None
    if force or not os.path.exists(_SO_GPU) or os.path.getmtime(_SO_GPU) < os.path.getmtime(_SRC_GPU):
        tmp = _SO_GPU + f".{os.getpid()}.tmp"
        cmd = [cc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-fmad=false", "-shared",
               "-Xcompiler", "-fPIC", _SRC_GPU, "-o", tmp, "-lcudart"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO_GPU)
    return _SO_GPU


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            lib.synth_heatbath.restype = ctypes.c_int
            lib.synth_heatbath.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_int, ctypes.c_uint64, ctypes.c_int]
            lib.synth_vonmises.restype = ctypes.c_int
            lib.synth_vonmises.argtypes = [ctypes.c_double, ctypes.c_long, ctypes.c_uint64, ctypes.c_void_p]
            lib.synth_exp.restype = ctypes.c_double
            lib.synth_exp.argtypes = [ctypes.c_double]
            _lib = lib
    return _lib


def _load_gpu():
    global _lib_gpu
    with _lock:
        if _lib_gpu is None:
            if build_gpu() is None:
                raise RuntimeError("the GPU heatbath needs the CUDA toolkit (nvcc)")
            lib = ctypes.CDLL(_SO_GPU)
            lib.synth_heatbath_gpu.restype = ctypes.c_int
            lib.synth_heatbath_gpu.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                               ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p]
            _lib_gpu = lib
    return _lib_gpu


def heatbath_gpu(Lx: int, Lt: int, beta: float, sweeps: int, seed: int) -> np.ndarray:
    """heatbath() computed on the current CUDA device; bit-identical result."""
    import torch
    U = torch.empty((Lt, Lx, 2), dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream()
    rc = _load_gpu().synth_heatbath_gpu(U.data_ptr(), Lx, Lt, float(beta), int(sweeps),
                                        int(seed) & (2**64 - 1), ctypes.c_void_p(stream.cuda_stream))
    if rc != 0:
        raise RuntimeError(f"GPU heatbath failed ({rc}) for Lx={Lx} Lt={Lt} beta={beta} sweeps={sweeps}")
    return U.cpu().numpy()


def default_sweeps(L: int) -> int:
    """1000 thermalisation sweeps, 2000 at 1024^2 and above."""
    return 2000 if L >= 1024 else 1000


def gauge_seed(L: int, config: int) -> int:
    return 1000 * L + config


def heatbath(Lx: int, Lt: int, beta: float, sweeps: int, seed: int, nthreads: int | None = None) -> np.ndarray:
    """Thermalised field (the result does not depend on the thread count)."""
    if nthreads is None:
        # small lattices: one thread (a parallel sub-sweep of a few hundred links costs more than it saves)
        nthreads = 1 if Lx * Lt <= 64 * 64 else min(os.cpu_count() or 1, 16)
    U = np.empty((Lt, Lx, 2), dtype=np.complex128)
    rc = _load().synth_heatbath(U.ctypes.data, Lx, Lt, float(beta), int(sweeps), int(seed) & (2**64 - 1),
                                int(nthreads))
    if rc != 0:
        raise ValueError(f"heatbath rejected Lx={Lx} Lt={Lt} beta={beta} sweeps={sweeps}")
    return U


_CACHE_DIR = os.path.join(_HERE, "_cache")


def gauge_field(L: int, config: int, sweeps: int | None = None, beta: float = BETA,
                cache: bool = True, gpu: bool = False) -> np.ndarray:
    """Configuration `config` of the L x L pool (seed 1000 L + config); with
    gpu=True a field not in the cache is generated on the current CUDA device
    (the same bits)."""
    sweeps = default_sweeps(L) if sweeps is None else sweeps
    path = os.path.join(_CACHE_DIR, f"gauge_L{L}_c{config}_s{sweeps}_b{beta:g}.npy")
    if cache and os.path.exists(path):
        return np.load(path)
    if gpu:
        U = heatbath_gpu(L, L, beta, sweeps, gauge_seed(L, config))
    else:
        U = heatbath(L, L, beta, sweeps, gauge_seed(L, config))
    if cache:
        os.makedirs(_CACHE_DIR, exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp.npy"
        np.save(tmp, U)
        os.replace(tmp, path)
    return U


def fingerprint(U: np.ndarray) -> str:
    """Short hash of the exact bytes of a field (checks cross-machine identity)."""
    return hashlib.sha256(np.ascontiguousarray(U).tobytes()).hexdigest()[:16]


def vonmises(kappa: float, n: int, seed: int) -> np.ndarray:
    out = np.empty((n, 2), dtype=np.float64)
    _load().synth_vonmises(float(kappa), int(n), int(seed), out.ctypes.data)
    return out


def det_exp(x: float) -> float:
    return _load().synth_exp(float(x))


def _rng(*key: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(k) for k in key])))


def complex_gaussian(shape, *key: int) -> np.ndarray:
    """Complex Gaussian with E|z|^2 = 1, seeded by the integer tuple `key`."""
    g = _rng(*key)
    re = g.standard_normal(shape)
    im = g.standard_normal(shape)
    return (re + 1j * im) * np.sqrt(0.5)


def z4_noise(shape, *key: int) -> np.ndarray:
    """Z(4) noise: entries uniform over {1, i, -1, -i} (Section 2)."""
    k = _rng(*key).integers(0, 4, size=shape)
    return (1j ** k).astype(np.complex128)


_TAG_RHS = 0x5248  # "RH"
_TAG_NULL = 0x4E56  # "NV"


def rhs(L: int, config: int, index: int, nrhs: int = 1) -> np.ndarray:
    """nrhs right-hand sides, complex128[nrhs][L][L][2], seed (L, config, index + i)."""
    return np.stack([complex_gaussian((L, L, 2), _TAG_RHS, L, config, index + i) for i in range(nrhs)])


def nullvec_starts(L: int, config: int, level: int, nvec: int, n: int) -> np.ndarray:
    """Random start vectors x_i of the near-null-vector solves, complex128[nvec][n]."""
    return np.stack([complex_gaussian((n,), _TAG_NULL, L, config, level, i) for i in range(nvec)])


_M0_TABLE = os.path.join(_HERE, "m0_table.json")


def m0_table() -> dict:
    with open(_M0_TABLE) as f:
        return json.load(f)


def m0_for(L: int, config: int) -> float:
    """Tuned bare mass of configuration (L, config)."""
    t = m0_table()
    key = f"{L}:{config}"
    if key not in t["entries"]:
        raise KeyError(f"no tuned m0 for L={L} config={config}; run oracle/tune_m0.py")
    return float(t["entries"][key]["m0"])


def check_fingerprint(L: int, config: int, U: np.ndarray) -> bool:
    """True when U is bit-identical to the field m0 was tuned on."""
    t = m0_table()
    e = t["entries"].get(f"{L}:{config}")
    return e is not None and e.get("fingerprint") == fingerprint(U)
