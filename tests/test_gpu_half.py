"""The FP16 copy of the coarsest operator (mg_params.coarse_half, the mixed
default): the GMRES-Proj cluster kernels stream it instead of the FP32 copy
and multiply in FP32.

* with it on and off, every solve meets its true-residual tolerance
  (recomputed with the oracle's FP64 D), the outer iteration counts agree
  within one, and the coarse iteration totals within 2%;
* the two paths are different arithmetic (the solutions are not bitwise
  equal), so the FP16 operator is the one in use.
"""
import numpy as np
import pytest

import synth
from oracle import dirac
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mgmod(cuda_lib):
    import paper_1912_02868_gb300 as mg
    return mg


@pytest.mark.parametrize("L,c", [(64, 2), (256, 0)])
def test_half_coarse_operator(mgmod, L, c):
    import torch
    U = synth.gauge_field(L, c)
    m0 = synth.m0_for(L, c)
    B = synth.rhs(L, c, 0, nrhs=3)
    out = {}
    for half in (0, 1):
        g = mgmod.mg_setup(dev(U), L, L, m0,
                           params=mgmod.default_params(precision=mgmod.MG_MIXED, coarse_half=half),
                           starts0=dev(synth.nullvec_starts(L, c, 0, 12, L * L * 2)),
                           starts1=dev(synth.nullvec_starts(L, c, 1, 12, (L // 4) ** 2 * 24)))
        try:
            X = torch.zeros(B.shape, dtype=torch.complex128, device="cuda")
            st, iters, relres, stats = mgmod.mg_solve(g, dev(B), X, 3, 1e-8)
            out[half] = (host(X), iters, stats)
        finally:
            g.close()
        for i in range(3):
            r = dirac.wilson(U, out[half][0][i], m0) - B[i]
            assert np.linalg.norm(r) <= 1.0001e-8 * np.linalg.norm(B[i])
    (x0, it0, s0), (x1, it1, s1) = out[0], out[1]
    assert all(abs(a - b) <= 1 for a, b in zip(it0, it1))
    assert abs(s1["coarse_iters"] - s0["coarse_iters"]) <= 0.02 * s0["coarse_iters"]
    assert not np.array_equal(x0, x1)
