"""The intermediate grid with rank-4 hop factors (mg_params.lowrank_hops).

Every hop block of D^ = P^+ D P sums four boundary-site terms, each with a
rank-1 spin projector (Section 2's operator), so it has rank <= 4 (the oracle
pins this).  The library factors each dense block at set-up and applies the
factors.  Checks, on handles built from the same near-null vectors with and
without the factors:

* the factors are in use, and reproduce every block to rounding (the largest
  relative Frobenius error is reported by mg_stencil_info);
* the factored apply, D^ and D^+, against the oracle's dense stencil: 1e-12
  relative in FP64 and 2e-6 in FP32 (max norm), and against the dense handle;
* a whole FP64 solve takes the same outer iterations and agrees with the dense
  handle's solution to 1e-10.
"""
import numpy as np
import pytest

import synth
from oracle import dirac
import oracle_cache as oc
from gpu_util import dev, host, rel, rel2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mgmod(cuda_lib):
    import paper_1912_02868_gb300 as mg
    return mg


def _pair(mgmod, L, **params):
    U, m0, h = oc.hier(L)
    hs = []
    for lr in (1, 0):
        p = mgmod.default_params(lowrank_hops=lr, **params)
        hs.append(mgmod.mg_setup_from_vectors(dev(U), L, L, m0, dev(h.nullvecs[0]), dev(h.nullvecs[1]), params=p))
    return hs[0], hs[1], U, m0, h


@pytest.mark.parametrize("L", [64, 256])
def test_factored_intermediate_stencil(mgmod, L):
    import torch
    g, gd, U, m0, h = _pair(mgmod, L, precision=mgmod.MG_MIXED)
    try:
        fac, err = mgmod.mg_stencil_info(g, 1)
        assert fac and err <= 1e-13, err
        assert mgmod.mg_stencil_info(gd, 1) == (False, 0.0)
        assert mgmod.mg_stencil_info(g, 2)[0] is False  # the coarsest grid stays dense
        shape = h.shapes[1]
        xv = synth.complex_gaussian(shape, 9900 + L)
        for dagger in (False, True):
            ref = (h.apply_dagger if dagger else h.apply)(1, xv)
            for prec, dt, tol in ((mgmod.MG_F64, torch.complex128, 1e-12), (mgmod.MG_F32, torch.complex64, 2e-6)):
                y = torch.zeros(shape, dtype=dt, device="cuda")
                yd = torch.zeros_like(y)
                mgmod.mg_apply(g, 1, dev(xv, dt), y, dagger=dagger, precision=prec)
                mgmod.mg_apply(gd, 1, dev(xv, dt), yd, dagger=dagger, precision=prec)
                assert rel(host(y), ref) <= tol, (dagger, prec)
                assert rel(host(y), host(yd)) <= tol, (dagger, prec)
    finally:
        g.close()
        gd.close()


def test_factored_solve_matches_dense(mgmod):
    import torch
    L = 128
    g, gd, U, m0, h = _pair(mgmod, L)
    try:
        b = synth.rhs(L, 0, 5)[0]
        x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
        xd = torch.zeros_like(x)
        _, it, rr, _ = mgmod.mg_solve(g, dev(b), x, 1, 1e-10)
        _, itd, rrd, _ = mgmod.mg_solve(gd, dev(b), xd, 1, 1e-10)
        assert it == itd and rr[0] <= 1e-10 and rrd[0] <= 1e-10
        assert rel2(host(x), host(xd)) <= 1e-10
        r = np.linalg.norm(dirac.wilson(U, host(x), m0) - b) / np.linalg.norm(b)
        assert r <= 1.0001e-10
    finally:
        g.close()
        gd.close()
