"""GPU parity of the operator kernels against the FP64 oracle, through the C ABI.

Per apply the FP64 kernels must agree with the oracle to <= 1e-12 relative
(max norm); the FP32 kernels to <= 2e-6 (single-precision rounding of sums of
at most 5 x 24 terms of unit-size magnitude).  Sizes span several CTAs and a
ragged tail (48 x 32, 80 x 16), the bench lattice 256^2, and 1024^2.
"""
import numpy as np
import pytest

import synth
from oracle import dirac, hierarchy
from gpu_util import dev, host, rel

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_TOL = 2e-6


@pytest.fixture(scope="module")
def mgmod(cuda_lib):
    import paper_1912_02868_gb300 as mg
    return mg


def _field(Lx, Lt, seed):
    if Lx == Lt and Lx in (16, 32, 64, 256):
        return synth.gauge_field(Lx, 0)
    return synth.heatbath(Lx, Lt, 6.0, 200, seed)


@pytest.mark.parametrize("Lx,Lt", [(16, 16), (48, 32), (80, 16), (64, 64), (256, 256), (1024, 1024), (6, 4)])
@pytest.mark.parametrize("dagger", [False, True])
def test_wilson_apply_parity(mgmod, Lx, Lt, dagger):
    import torch
    U = _field(Lx, Lt, 3) if Lx * Lt <= 256 * 256 else np.exp(2j * np.pi * synth.complex_gaussian((Lt, Lx, 2), 4).real)
    m0 = -0.07
    psi = synth.complex_gaussian((Lt, Lx, 2), 5)
    ref = (dirac.wilson_dagger if dagger else dirac.wilson)(U, psi, m0)
    y = torch.empty(psi.shape, dtype=torch.complex128, device="cuda")
    mgmod.mg_wilson_apply(dev(U), Lx, Lt, m0, dev(psi), y, dagger=dagger)
    assert rel(host(y), ref) <= F64_TOL
    y32 = torch.empty(psi.shape, dtype=torch.complex64, device="cuda")
    mgmod.mg_wilson_apply(dev(U, torch.complex64), Lx, Lt, m0, dev(psi, torch.complex64), y32, dagger=dagger,
                          precision=mgmod.MG_F32)
    assert rel(host(y32), ref) <= F32_TOL


def _oracle_hierarchy(Lx, Lt, cfg=0):
    if Lx == Lt:
        U = synth.gauge_field(Lx, cfg)
        m0 = synth.m0_for(Lx, cfg)
    else:
        U = synth.heatbath(Lx, Lt, 6.0, 300, 41)
        m0 = -0.07
    s0 = synth.complex_gaussian((12, Lt, Lx, 2), 7, Lx, Lt)
    s1 = synth.complex_gaussian((12, Lt // 4, Lx // 4, 24), 8, Lx, Lt)
    return U, m0, hierarchy.build(U, m0, s0, s1)


@pytest.fixture(scope="module", params=[(16, 16), (32, 32), (48, 32), (64, 64)])
def pair(request, mgmod):
    """The oracle hierarchy and the GPU hierarchy built from the same near-null vectors."""
    Lx, Lt = request.param
    U, m0, h = _oracle_hierarchy(Lx, Lt)
    g = mgmod.mg_setup_from_vectors(dev(U), Lx, Lt, m0, dev(h.nullvecs[0]), dev(h.nullvecs[1]))
    yield Lx, Lt, U, m0, h, g
    g.close()


def test_prolongator_parity(mgmod, pair):
    Lx, Lt, U, m0, h, g = pair
    assert rel(mgmod.mg_get_prolongator(g, 0), h.Q0) <= F64_TOL
    assert rel(mgmod.mg_get_prolongator(g, 1), h.Q1) <= 1e-11


def test_galerkin_parity(mgmod, pair):
    Lx, Lt, U, m0, h, g = pair
    assert rel(mgmod.mg_get_stencil(g, 1), h.A1) <= F64_TOL
    assert rel(mgmod.mg_get_stencil(g, 2), h.A2) <= 1e-11


@pytest.mark.parametrize("level", [0, 1, 2])
@pytest.mark.parametrize("dagger", [False, True])
def test_level_apply_parity(mgmod, pair, level, dagger):
    import torch
    Lx, Lt, U, m0, h, g = pair
    v = synth.complex_gaussian(h.shapes[level], 9, level)
    ref = (h.apply_dagger if dagger else h.apply)(level, v)
    y = torch.empty(v.shape, dtype=torch.complex128, device="cuda")
    mgmod.mg_apply(g, level, dev(v), y, dagger=dagger)
    assert rel(host(y), ref) <= F64_TOL
    y32 = torch.empty(v.shape, dtype=torch.complex64, device="cuda")
    mgmod.mg_apply(g, level, dev(v, torch.complex64), y32, dagger=dagger, precision=mgmod.MG_F32)
    assert rel(host(y32), ref) <= F32_TOL


@pytest.mark.parametrize("level", [0, 1])
def test_transfer_parity(mgmod, pair, level):
    import torch
    Lx, Lt, U, m0, h, g = pair
    v = synth.complex_gaussian(h.shapes[level], 10, level)
    vc = synth.complex_gaussian(h.shapes[level + 1], 11, level)
    out_c = torch.empty(vc.shape, dtype=torch.complex128, device="cuda")
    mgmod.mg_restrict(g, level, dev(v), out_c)
    assert rel(host(out_c), h.restrict(level, v)) <= F64_TOL
    out_f = torch.empty(v.shape, dtype=torch.complex128, device="cuda")
    mgmod.mg_prolong(g, level, dev(vc), out_f)
    assert rel(host(out_f), h.prolong(level, vc)) <= F64_TOL
    out_c32 = torch.empty(vc.shape, dtype=torch.complex64, device="cuda")
    mgmod.mg_restrict(g, level, dev(v, torch.complex64), out_c32, precision=mgmod.MG_F32)
    assert rel(host(out_c32), h.restrict(level, v)) <= F32_TOL


def test_gpu_setup_at_bench_size_properties(mgmod):
    """256^2, near-null vectors solved on the GPU: P^+P = I, sigma3^-hermitian
    stencils, and the Galerkin kernel equals the oracle's Galerkin product of
    the GPU's own prolongator (every coarse site compared)."""
    L = 256
    U = synth.gauge_field(L, 0)
    m0 = synth.m0_for(L, 0)
    g = mgmod.mg_setup(dev(U), L, L, m0, starts0=dev(synth.nullvec_starts(L, 0, 0, 12, L * L * 2)),
                       starts1=dev(synth.nullvec_starts(L, 0, 1, 12, (L // 4) ** 2 * 24)))
    try:
        Q0 = mgmod.mg_get_prolongator(g, 0)
        Q1 = mgmod.mg_get_prolongator(g, 1)
        # single-pass modified Gram-Schmidt keeps orthogonality to ~eps * cond(block);
        # the 16 x 12 and 192 x 12 blocks at 256^2 reach ~1e-12
        for Q, tol in ((Q0, 1e-11), (Q1, 1e-11)):
            G = np.einsum("tzcjla,tzcila->tzcji", np.conj(Q), Q)
            assert np.abs(G - np.eye(12)).max() < tol
        A1 = mgmod.mg_get_stencil(g, 1)
        A2 = mgmod.mg_get_stencil(g, 2)
        assert rel(A1, hierarchy.galerkin(dirac.wilson_stencil(U, m0), Q0)) <= F64_TOL
        assert rel(A2, hierarchy.galerkin(A1, Q1)) <= F64_TOL
        # sigma3^-hermiticity: A[s, +mu]^+ = s3 A[s + mu, -mu] s3, A[s, self]^+ = s3 A[s, self] s3
        s3 = np.concatenate([np.ones(12), -np.ones(12)])
        for A in (A1, A2):
            Ad = np.conj(np.swapaxes(A, -1, -2))
            S = s3[:, None] * A * s3[None, :]
            assert np.abs(Ad[:, :, 0] - S[:, :, 0]).max() < 1e-12
            assert np.abs(Ad[:, :, 1] - np.roll(S[:, :, 2], -1, axis=1)).max() < 1e-12
            assert np.abs(Ad[:, :, 3] - np.roll(S[:, :, 4], -1, axis=0)).max() < 1e-12
    finally:
        g.close()


def test_invalid_arguments_are_errors(mgmod):
    import torch
    U = synth.gauge_field(16, 0)
    with pytest.raises(mgmod.MGError):
        mgmod.mg_setup(dev(U), 24, 16, 0.0)  # 24 is not a multiple of 16
    with pytest.raises(mgmod.MGError):
        mgmod.mg_setup(dev(U), 16, 16, 0.0, nvec=8)
    with pytest.raises(mgmod.MGError):
        mgmod.mg_setup(dev(U), 16, 16, float("nan"))
    p = mgmod.default_params(dr_k=40)
    with pytest.raises(mgmod.MGError):
        mgmod.mg_setup(dev(U), 16, 16, 0.0, params=p)
    x = torch.zeros((16, 16, 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(mgmod.MGError):
        mgmod.mg_wilson_apply(dev(U), 16, 16, 0.0, x, x)  # aliasing
