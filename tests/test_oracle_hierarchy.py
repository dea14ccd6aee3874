"""Pins of the oracle's multigrid set-up (Section 2, first paragraph), CPU only.

* P^+ P = I (local orthonormalisation) and sigma_3 P = P sigma3^ (chirality kept);
* range(P) does not depend on the Gram-Schmidt variant or on the global
  orthonormalisation (compared through the projector P P^+);
* D^ = P^+ D P against the product of explicitly assembled dense matrices, on
  both coarsenings;
* sigma3^-hermiticity of D^; every intermediate-grid hop block has rank <= 4
  (four face sites, each a rank-one spin projector);
* the near-null vectors satisfy the stopping rule of their CG solve.
"""
import numpy as np
import pytest

import synth
from oracle import dirac, hierarchy


@pytest.fixture(scope="module")
def small():
    L = 16
    U = synth.gauge_field(L, 0, cache=False)
    m0 = synth.m0_for(L, 0)
    s0 = synth.nullvec_starts(L, 0, 0, 12, L * L * 2)
    s1 = synth.nullvec_starts(L, 0, 1, 12, (L // 4) ** 2 * 24)
    h = hierarchy.build(U, m0, s0, s1)
    return L, U, m0, h


def test_prolongator_orthonormal_and_chiral(small):
    L, U, m0, h = small
    for Q, shape in ((h.Q0, (L, L, 2)), (h.Q1, h.shapes[1])):
        P = hierarchy.dense_prolongator(Q, shape)
        assert np.abs(P.conj().T @ P - np.eye(P.shape[1])).max() < 1e-13
        dof = shape[-1]
        s3 = np.tile(np.concatenate([np.ones(dof // 2), -np.ones(dof // 2)]), shape[0] * shape[1])
        nc = P.shape[1]
        s3c = np.tile(np.concatenate([np.ones(12), -np.ones(12)]), nc // 24)
        assert np.abs(s3[:, None] * P - P * s3c[None, :]).max() < 1e-14
        # restriction undoes prolongation
        vc = synth.complex_gaussian((nc,), 17)
        cs = h.shapes[1] if Q is h.Q0 else h.shapes[2]
        back = hierarchy.restrict(Q, hierarchy.prolong(Q, vc.reshape(cs)))
        assert np.abs(back.ravel() - vc).max() < 1e-13


def test_range_independent_of_gram_schmidt(small):
    L, U, m0, h = small
    nv = h.nullvecs[0]
    Pa = hierarchy.dense_prolongator(h.Q0, (L, L, 2))
    # no global orthonormalisation, Householder QR per block instead of MGS
    blocks = hierarchy.local_blocks(nv)
    Qb = np.empty_like(blocks)
    for idx in np.ndindex(blocks.shape[:3]):
        M = blocks[idx].reshape(12, -1).T
        Qb[idx] = np.linalg.qr(M)[0].T.reshape(blocks[idx].shape)
    Pb = hierarchy.dense_prolongator(Qb, (L, L, 2))
    assert np.abs(Pa @ Pa.conj().T - Pb @ Pb.conj().T).max() < 1e-12


def test_galerkin_equals_dense_product(small):
    L, U, m0, h = small
    D = dirac.dense_from_apply(lambda v: dirac.wilson(U, v, m0), (L, L, 2))
    P = hierarchy.dense_prolongator(h.Q0, (L, L, 2))
    D1 = dirac.dense_from_apply(lambda v: dirac.stencil_apply(h.A1, v), h.shapes[1])
    assert np.abs(P.conj().T @ D @ P - D1).max() < 1e-13
    P1 = hierarchy.dense_prolongator(h.Q1, h.shapes[1])
    D2 = dirac.dense_from_apply(lambda v: dirac.stencil_apply(h.A2, v), h.shapes[2])
    assert np.abs(P1.conj().T @ D1 @ P1 - D2).max() < 1e-13


def test_galerkin_on_rectangular_lattice():
    Lx, Lt = 32, 16
    U = synth.heatbath(Lx, Lt, 6.0, 100, 77)
    m0 = -0.06
    s0 = synth.complex_gaussian((12, Lt, Lx, 2), 1)
    s1 = synth.complex_gaussian((12, Lt // 4, Lx // 4, 24), 2)
    h = hierarchy.build(U, m0, s0, s1)
    D = dirac.dense_from_apply(lambda v: dirac.wilson(U, v, m0), (Lt, Lx, 2))
    P = hierarchy.dense_prolongator(h.Q0, (Lt, Lx, 2))
    D1 = dirac.dense_from_apply(lambda v: dirac.stencil_apply(h.A1, v), h.shapes[1])
    assert np.abs(P.conj().T @ D @ P - D1).max() < 1e-13
    P1 = hierarchy.dense_prolongator(h.Q1, h.shapes[1])
    D2 = dirac.dense_from_apply(lambda v: dirac.stencil_apply(h.A2, v), h.shapes[2])
    assert np.abs(P1.conj().T @ D1 @ P1 - D2).max() < 1e-13


def test_coarse_sigma3_hermiticity_and_hop_rank(small):
    L, U, m0, h = small
    for A in (h.A1, h.A2):
        M = dirac.dense_from_apply(lambda v: dirac.stencil_apply(A, v), A.shape[:2] + (24,))
        s3 = np.tile(np.concatenate([np.ones(12), -np.ones(12)]), A.shape[0] * A.shape[1])
        assert np.abs(M.conj().T - s3[:, None] * M * s3[None, :]).max() < 1e-13
        Md = dirac.dense_from_apply(lambda v: dirac.stencil_dagger_sigma(A, v), A.shape[:2] + (24,))
        assert np.abs(Md - M.conj().T).max() < 1e-13
    sv = np.linalg.svd(h.A1[:, :, 1:], compute_uv=False)
    assert np.all(sv[..., 4] < 1e-12 * sv[..., 0])
    assert np.all(sv[..., 3] > 1e-8 * sv[..., 0])


def test_nullvector_solve_meets_its_tolerance(small):
    L, U, m0, h = small
    s0 = synth.nullvec_starts(L, 0, 0, 12, L * L * 2).reshape(12, L, L, 2)
    psi = h.nullvecs[0]
    e = psi - s0
    for i in range(12):
        Ax = dirac.wilson(U, dirac.wilson_dagger(U, s0[i], m0), m0)
        r = -Ax - dirac.wilson(U, dirac.wilson_dagger(U, e[i], m0), m0)
        assert np.linalg.norm(r) <= 1e-4 * np.linalg.norm(Ax) * (1 + 1e-6)
    # the near-null vectors are dominated by low modes: ||D psi|| / ||psi|| far below ||D x|| / ||x||
    for i in range(12):
        q_psi = np.linalg.norm(dirac.wilson(U, psi[i], m0)) / np.linalg.norm(psi[i])
        q_x = np.linalg.norm(dirac.wilson(U, s0[i], m0)) / np.linalg.norm(s0[i])
        assert q_psi < 0.3 * q_x


def test_rank_deficient_block_is_an_error():
    L = 16
    v = synth.complex_gaussian((12, L, L, 2), 3)
    blocks = hierarchy.local_blocks(v)
    hierarchy.local_orthonormalise(blocks)  # full rank: fine
    blocks[1, 2, 0, 5] = 2.0 * blocks[1, 2, 0, 4]  # one block, one chirality loses rank
    with pytest.raises(ValueError):
        hierarchy.local_orthonormalise(blocks)
