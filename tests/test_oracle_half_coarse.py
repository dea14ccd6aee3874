"""Why the mixed path may stream the coarsest operator in FP16 (oracle only, no
GPU): with the deflation space built by GMRES-DR on the exact operator, the
later GMRES-Proj coarse solves run on a copy whose entries are rounded to FP16
(each part rounded once from FP64).  MG-FGMRES then needs the same outer
iterations as with the exact operator, and about the same coarse iterations.
(Rounding a 24x24 block entry of size <= 1 to FP16 errs by at most 2^-12,
far below the 1e-2 to 1e-8 coarse tolerances.)
"""
import copy

import numpy as np

import synth
from oracle import hierarchy, krylov, mg as omg


class _ProjOnRounded(omg.MGSolver):
    def __init__(self, hier, rounded):
        super().__init__(hier, omg.Params())
        self.rounded = rounded

    def coarse_solve(self, f):
        if self.deflation is None:
            return super().coarse_solve(f)
        shape = self.h.shapes[2]
        A2 = self.counter.wrap(2, lambda v: self.rounded.apply(2, v.reshape(shape)).ravel())
        x, info = krylov.gmres_proj(A2, f, self.deflation, self.p.dr_m, self.p.coarse_tol_rest,
                                    self.p.proj_max_cycles)
        self.coarse_solves.append(("proj", info.iters))
        return x


def _fp16(a):
    return a.real.astype(np.float16).astype(np.float64) + 1j * a.imag.astype(np.float16).astype(np.float64)


def test_fp16_coarse_operator_keeps_outer_iterations():
    L = 32
    U = synth.gauge_field(L, 0)
    m0 = synth.m0_for(L, 0)
    h = hierarchy.build(U, m0, synth.nullvec_starts(L, 0, 0, 12, L * L * 2),
                        synth.nullvec_starts(L, 0, 1, 12, (L // 4) ** 2 * 24))
    hr = copy.copy(h)
    hr.A2 = _fp16(h.A2)
    err = np.abs(hr.A2 - h.A2).max()
    assert 0 < err <= 2.0 ** -12 * max(1.0, np.abs(h.A2).max())
    B = synth.rhs(L, 0, 0, nrhs=3)
    exact, rounded = omg.MGSolver(h, omg.Params()), _ProjOnRounded(h, hr)
    for i in range(3):
        _, ie = exact.solve(B[i], 1e-8)
        _, ir = rounded.solve(B[i], 1e-8)
        assert ie.iters == ir.iters
        assert ir.relres <= 1e-8
    ce = sum(c[1] for c in exact.coarse_solves[1:])
    cr = sum(c[1] for c in rounded.coarse_solves[1:])
    assert abs(cr - ce) <= 0.02 * ce
