"""GPU parity of the partial intermediate solve (Section 2 variant) against the
FP64 oracle, through the C ABI (mg_params.partial_tol = 0.2).

* FP64, identical prolongators: the solve reaches its true-residual tolerance;
  against a sparse direct solve the error is <= kappa * tol; the outer
  iteration count is the oracle's to within one.  (The coarse solves stop at
  1e-2 and the intermediate solves at 0.2, so iterates of two implementations
  need not agree to rounding: where a threshold falls between two steps, the
  preconditioner outputs differ at the level of that threshold.  The bound is
  therefore the direct solve's, not bit-for-bit agreement with the oracle.)
* the deflation space is built once (one GMRES-DR solve) and reused;
* mixed precision: true residual <= 1e-8, fewer outer iterations and less
  coarse work than the V-cycle on the same system.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import dirac, hierarchy, mg as omg
from gpu_util import dev, host, rel2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mgmod(cuda_lib):
    import paper_1912_02868_gb300 as mg
    return mg


def _hier(L, cfg=0):
    U = synth.gauge_field(L, cfg)
    m0 = synth.m0_for(L, cfg)
    h = hierarchy.build(U, m0, synth.nullvec_starts(L, cfg, 0, 12, L * L * 2),
                        synth.nullvec_starts(L, cfg, 1, 12, (L // 4) ** 2 * 24))
    return U, m0, h


def _kappa(A):
    Ad = A.toarray()
    return np.linalg.norm(Ad, 2) / np.linalg.svd(Ad, compute_uv=False)[-1]


@pytest.mark.parametrize("L", [16, 32])
def test_partial_fp64_parity(mgmod, L):
    import torch
    U, m0, h = _hier(L)
    tol = 1e-10
    b = synth.rhs(L, 0, 0)[0]
    osol = omg.MGSolver(h, omg.Params(partial_tol=0.2))
    xo, info_o = osol.solve(b, tol)
    p = mgmod.default_params(partial_tol=0.2)
    g = mgmod.mg_setup_from_vectors(dev(U), L, L, m0, dev(h.nullvecs[0]), dev(h.nullvecs[1]), params=p)
    try:
        x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
        st, iters, relres, stats = mgmod.mg_solve(g, dev(b), x, 1, tol)
        xg = host(x)
        # a second right-hand side reuses the deflation space
        b2 = synth.rhs(L, 0, 1)[0]
        x2 = torch.zeros(b2.shape, dtype=torch.complex128, device="cuda")
        st2, iters2, relres2, stats2 = mgmod.mg_solve(g, dev(b2), x2, 1, tol)
    finally:
        g.close()
    A = dirac.stencil_sparse(dirac.wilson_stencil(U, m0)).tocsc()
    xs = spla.splu(A).solve(b.ravel())
    assert relres[0] <= tol
    assert np.linalg.norm(dirac.wilson(U, xg, m0) - b) <= 1.0001 * tol * np.linalg.norm(b)
    assert rel2(xg, xs) <= _kappa(A) * tol
    assert abs(iters[0] - info_o.iters) <= 1
    assert stats["dr_solves"] == 1 and stats2["dr_solves"] == 0 and relres2[0] <= tol


def test_partial_mixed_64(mgmod):
    import torch
    L = 64
    U = synth.gauge_field(L, 0)
    m0 = synth.m0_for(L, 0)
    starts = dict(starts0=dev(synth.nullvec_starts(L, 0, 0, 12, L * L * 2)),
                  starts1=dev(synth.nullvec_starts(L, 0, 1, 12, (L // 4) ** 2 * 24)))
    B = synth.rhs(L, 0, 0, nrhs=2)
    out = {}
    for name, pt in (("vcycle", 0.0), ("partial", 0.2)):
        g = mgmod.mg_setup(dev(U), L, L, m0, params=mgmod.default_params(precision=mgmod.MG_MIXED, partial_tol=pt),
                           **starts)
        try:
            X = torch.zeros(B.shape, dtype=torch.complex128, device="cuda")
            st, iters, relres, stats = mgmod.mg_solve(g, dev(B), X, 2, 1e-8)
            Xh = host(X)
        finally:
            g.close()
        for i in range(2):
            assert relres[i] <= 1e-8
            assert np.linalg.norm(dirac.wilson(U, Xh[i], m0) - B[i]) <= 1.0001e-8 * np.linalg.norm(B[i])
        out[name] = (sum(iters), stats["coarse_iters"])
    assert out["partial"][0] < out["vcycle"][0]
    assert out["partial"][1] < out["vcycle"][1]
