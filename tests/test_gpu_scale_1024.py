"""The scale-up configuration at full size: 1024^2 lattice (2000 heatbath sweeps,
m0 tuned to min Re lambda = 1e-3), hierarchy 1024^2 x 2 -> 256^2 x 24 -> 64^2 x 24,
GMRES-DR(40,16) / GMRES-Proj(40,16) on the coarsest grid, mixed precision, several
right-hand sides solved together.

The oracle cannot follow a solve of this size step by step, so the check is the
property that defines a solution: the true residual, recomputed here with the
oracle's FP64 Wilson operator, meets the tolerance for every right-hand side.
The coarse grid here is 16 times the 256^2 one, so it runs the general path of
the coarse cluster kernel (basis in global memory, staged neighbour rows).  The
lockstep block solve with FP16 tensor-core block products runs 16 right-hand
sides; its coarse Arnoldi steps take the three-kernel form (the chunked grid
does not fit the resident cooperative launch).  The field comes from the GPU
heatbath, bit-identical to the host generator (its fingerprint is checked).
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


def test_scale_1024_mixed_dr40_16(mgmod):
    import torch
    L = 1024
    U = synth.gauge_field(L, 0, gpu=True)
    assert synth.check_fingerprint(L, 0, U)
    m0 = synth.m0_for(L, 0)
    p = mgmod.default_params(precision=mgmod.MG_MIXED, dr_m=40, dr_k=16, parallel=4)
    g = mgmod.mg_setup(dev(U), L, L, m0, params=p)
    try:
        B = synth.rhs(L, 0, 0, nrhs=4)
        X = torch.zeros(B.shape, dtype=torch.complex128, device="cuda")
        st, iters, relres, stats = mgmod.mg_solve(g, dev(B), X, 4, 1e-8)
        Xh = host(X)
        W, Hk = mgmod.mg_get_deflation(g)
    finally:
        g.close()
    assert stats["dr_solves"] == 1 and Hk.shape == (17, 16)
    for i in range(4):
        assert relres[i] <= 1e-8
        r = dirac.wilson(U, Xh[i], m0) - B[i]
        assert np.linalg.norm(r) <= 1.0001e-8 * np.linalg.norm(B[i])


def test_scale_1024_block_fp16_16rhs(mgmod):
    import torch
    L, nrhs = 1024, 16
    U = synth.gauge_field(L, 0, gpu=True)
    assert synth.check_fingerprint(L, 0, U)
    m0 = synth.m0_for(L, 0)
    p = mgmod.default_params(precision=mgmod.MG_MIXED_FP16, dr_m=40, dr_k=16)
    g = mgmod.mg_setup(dev(U), L, L, m0, params=p)
    try:
        B = synth.rhs(L, 0, 100, nrhs=nrhs)
        X = torch.zeros(B.shape, dtype=torch.complex128, device="cuda")
        st, iters, relres, stats = mgmod.mg_solve(g, dev(B), X, nrhs, 1e-8)
        Xh = host(X)
    finally:
        g.close()
    assert stats["dr_solves"] == 1
    for i in range(nrhs):
        assert relres[i] <= 1e-8
        r = dirac.wilson(U, Xh[i], m0) - B[i]
        assert np.linalg.norm(r) <= 1.0001e-8 * np.linalg.norm(B[i]), i
