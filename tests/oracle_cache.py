"""Oracle results shared by the GPU parity tests of one pytest process: the
hierarchy of a synthetic configuration (from the oracle's own near-null
vectors) and a GMRES-DR deflation space of its coarsest operator.  Everything
here comes from oracle/ and synth/ only."""
import functools

import numpy as np

import synth
from oracle import hierarchy, krylov


@functools.lru_cache(maxsize=4)
def hier(L, c=0):
    U = synth.gauge_field(L, c)
    m0 = synth.m0_for(L, c)
    h = hierarchy.build(U, m0, synth.nullvec_starts(L, c, 0, 12, L * L * 2),
                        synth.nullvec_starts(L, c, 1, 12, (L // 4) ** 2 * 24))
    return U, m0, h


def coarse_op(h, rounded=None):
    """v -> D^^ v on the coarsest grid (flat vectors); `rounded` replaces the stencil."""
    A2 = h.A2 if rounded is None else rounded
    from oracle import dirac
    shape = h.shapes[2]
    return lambda v: dirac.stencil_apply(A2, v.reshape(shape)).ravel()


@functools.lru_cache(maxsize=4)
def coarse_deflation(L, c=0, m=30, k=10, tol=1e-14):
    """GMRES-DR(m,k) on the coarsest system with a seeded right-hand side: the
    deflation space (W, H_k) of Section 2, built by the oracle."""
    U, m0, h = hier(L, c)
    f = synth.complex_gaussian((h.size(2),), 7000 + L, c)
    _, info, defl = krylov.gmres_dr(coarse_op(h), f, m, k, tol)
    return defl


def fp16(a):
    """each part of a complex array rounded once to FP16 (round to nearest)"""
    return a.real.astype(np.float16).astype(np.float64) + 1j * a.imag.astype(np.float16).astype(np.float64)
