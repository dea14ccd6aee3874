"""Lockstep pairs of right-hand sides (mg_params.pair_rhs): two solve contexts
advance together and their coarsest GMRES-Proj solves run in one cluster kernel
that streams the coarse operator once for both.  Each right-hand side goes
through the operations of a separate solve, so against solving the right-hand
sides one by one (odd counts leave one right-hand side to a plain solve) the
solutions agree to rounding and the outer iteration counts are equal.  The two
cluster kernels are compiled separately, so the compiler may contract a few
products differently; where a coarse stopping test then lands within rounding
of its threshold, a coarse solve takes a step more or less, so the coarse step
totals agree to 0.1%.  The paired kernel applies the coarse operator with FP32
FMAs, so both sides run with coarse_mma = 0 (singles would otherwise use the
tensor-core apply, which rounds differently).
"""
import numpy as np
import pytest

import synth
from oracle import dirac
from gpu_util import dev, host, rel2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mgmod(cuda_lib):
    import paper_1912_02868_gb300 as mg
    return mg


@pytest.mark.parametrize("L,nrhs,par", [(256, 5, 2), (64, 4, 2), (128, 6, 3)])
def test_pairs_equal_sequential(mgmod, L, nrhs, par):
    import torch
    c = 1
    U = synth.gauge_field(L, c)
    m0 = synth.m0_for(L, c)
    starts = dict(starts0=dev(synth.nullvec_starts(L, c, 0, 12, L * L * 2)),
                  starts1=dev(synth.nullvec_starts(L, c, 1, 12, (L // 4) ** 2 * 24)))
    B = synth.rhs(L, c, 0, nrhs=nrhs)
    out = {}
    for mode, over in (("seq", dict(parallel=1)), ("pairs", dict(parallel=par, pair_rhs=1))):
        g = mgmod.mg_setup(dev(U), L, L, m0,
                           params=mgmod.default_params(precision=mgmod.MG_MIXED, coarse_mma=0, **over), **starts)
        try:
            X = torch.zeros(B.shape, dtype=torch.complex128, device="cuda")
            st, iters, relres, stats = mgmod.mg_solve(g, dev(B), X, nrhs, 1e-8)
            out[mode] = (host(X), list(iters), list(relres), stats)
        finally:
            g.close()
    Xs, its, rrs, sts = out["seq"]
    Xp, itp, rrp, stp = out["pairs"]
    assert itp == its
    for i in range(nrhs):
        assert rrp[i] <= 1e-8
        assert np.linalg.norm(dirac.wilson(U, Xp[i], m0) - B[i]) <= 1.0001e-8 * np.linalg.norm(B[i])
        assert rel2(Xp[i], Xs[i]) <= 1e-12
    assert stp["dr_solves"] == sts["dr_solves"] == 1
    assert abs(stp["coarse_iters"] - sts["coarse_iters"]) <= 1e-3 * sts["coarse_iters"] + 1
    assert stp["outer_iters"] == sts["outer_iters"]
