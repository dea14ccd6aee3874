"""Pins of the oracle's Krylov solvers (Section 2, second paragraph), CPU only.

Each solver is checked against dense linear algebra on small systems:
* GMRES(2) smoother = the minimum-residual vector of span{f, A f}, and its
  Arnoldi-relation residual = f - A x;
* FGMRES with M = I is GMRES: equal to the dense minimum-residual solution over
  the Krylov space; with an exact preconditioner it converges in one step;
* GMRES-DR: the first cycle is GMRES(m); m >= n solves exactly; the exported
  space satisfies A V_k = V_{k+1} H_k with orthonormal V_{k+1}; its Ritz values
  approach the eigenvalues of smallest modulus (dense eig);
* GMRES-Proj: the projection is the dense minimum-residual solution over
  span(V_k); with an exact invariant subspace containing b it solves at once;
* CGNE against dense LU.
"""
import numpy as np
import pytest

import synth
from oracle import dirac, hierarchy, krylov


@pytest.fixture(scope="module")
def coarse32():
    """Coarse operator (2^2 x 24 = 96) and intermediate (8^2 x 24) of a 32^2 hierarchy."""
    L = 32
    U = synth.gauge_field(L, 0, cache=False)
    m0 = synth.m0_for(L, 0)
    h = hierarchy.build(U, m0, synth.nullvec_starts(L, 0, 0, 12, L * L * 2),
                        synth.nullvec_starts(L, 0, 1, 12, (L // 4) ** 2 * 24))
    A2 = dirac.dense_from_apply(lambda v: dirac.stencil_apply(h.A2, v), h.shapes[2])
    A1 = dirac.dense_from_apply(lambda v: dirac.stencil_apply(h.A1, v), h.shapes[1])
    return A1, A2


def test_smoother_is_min_residual_on_two_dim_krylov_space(coarse32):
    A1, _ = coarse32
    f = synth.complex_gaussian((A1.shape[0],), 5)
    x, r = krylov.smoother(lambda v: A1 @ v, f, 2)
    K = np.stack([f, A1 @ f], axis=1)
    y = np.linalg.lstsq(A1 @ K, f, rcond=None)[0]
    xd = K @ y
    assert np.linalg.norm(x - xd) <= 1e-12 * np.linalg.norm(xd)
    assert np.linalg.norm(r - (f - A1 @ x)) <= 1e-12 * np.linalg.norm(f)
    assert np.linalg.norm(r) < np.linalg.norm(f)


def test_fgmres_identity_preconditioner_is_gmres(coarse32):
    A1, _ = coarse32
    n = A1.shape[0]
    b = synth.complex_gaussian((n,), 6)
    for j in (1, 3, 6):
        x, info = krylov.fgmres(lambda v: A1 @ v, b, lambda v: v, 1e-30, m=8, max_iters=j)
        K = np.stack([np.linalg.matrix_power(A1, i) @ b for i in range(j)], axis=1)
        Qk = np.linalg.qr(K)[0]
        xd = Qk @ np.linalg.lstsq(A1 @ Qk, b, rcond=None)[0]
        assert info.iters == j
        assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)


def test_fgmres_exact_preconditioner_one_step(coarse32):
    A1, _ = coarse32
    b = synth.complex_gaussian((A1.shape[0],), 7)
    Ainv = np.linalg.inv(A1)
    x, info = krylov.fgmres(lambda v: A1 @ v, b, lambda v: Ainv @ v, 1e-10, m=8)
    assert info.converged and info.iters == 1
    assert np.linalg.norm(x - np.linalg.solve(A1, b)) <= 1e-9 * np.linalg.norm(x)


def test_fgmres_restarted_solution_matches_lu(coarse32):
    _, A2 = coarse32
    A = A2 + 0.3 * np.eye(A2.shape[0])  # shifted away from critical mass: restarts converge quickly
    b = synth.complex_gaussian((A.shape[0],), 8)
    x, info = krylov.fgmres(lambda v: A @ v, b, lambda v: v, 1e-10, m=8, max_iters=2000)
    xs = np.linalg.solve(A, b)
    kappa = np.linalg.cond(A)
    assert info.converged and info.relres <= 1e-10
    assert np.linalg.norm(x - xs) <= kappa * 1e-10 * np.linalg.norm(xs)


def test_gmres_dr_first_cycle_is_gmres(coarse32):
    _, A2 = coarse32
    b = synth.complex_gaussian((A2.shape[0],), 9)
    m = 20
    x, info, _ = krylov.gmres_dr(lambda v: A2 @ v, b, m, 5, 1e-30, max_cycles=1)
    # orthonormal basis of the Krylov space by modified Gram-Schmidt (not the oracle's CGS2)
    Qk = np.zeros((A2.shape[0], m), dtype=np.complex128)
    Qk[:, 0] = b / np.linalg.norm(b)
    for j in range(1, m):
        w = A2 @ Qk[:, j - 1]
        for i in range(j):
            w = w - np.vdot(Qk[:, i], w) * Qk[:, i]
        Qk[:, j] = w / np.linalg.norm(w)
    xd = Qk @ np.linalg.lstsq(A2 @ Qk, b, rcond=None)[0]
    assert info.iters == m
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


def test_gmres_dr_exact_when_m_at_least_n():
    n = 24
    A = np.eye(n) * 2 + synth.complex_gaussian((n, n), 10) * 0.3
    b = synth.complex_gaussian((n,), 11)
    x, info, defl = krylov.gmres_dr(lambda v: A @ v, b, 30, 10, 1e-13)
    assert info.converged and info.cycles == 1
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-11 * np.linalg.norm(x)


def test_gmres_dr_deflation_space_relations_and_eigenvalues(coarse32):
    _, A2 = coarse32
    n = A2.shape[0]
    b = synth.complex_gaussian((n,), 12)
    m, k = 30, 10
    x, info, defl = krylov.gmres_dr(lambda v: A2 @ v, b, m, k, 1e-14, max_cycles=200)
    assert np.linalg.norm(A2 @ x - b) <= 1e-10 * np.linalg.norm(b)
    W = defl.W.T  # columns
    Hk = defl.Hk
    assert np.abs(W.conj().T @ W - np.eye(k + 1)).max() < 1e-12
    assert np.linalg.norm(A2 @ W[:, :k] - W @ Hk) <= 1e-10 * np.linalg.norm(A2, 2)
    lam = np.linalg.eigvals(A2)
    small = np.sort(np.abs(lam))[:4]
    ritz = np.sort(np.abs(np.linalg.eigvals(Hk[:k, :k])))[:4]
    # the lowest modes, which GMRES-DR deflates, are found to good accuracy
    assert np.allclose(ritz, small, rtol=1e-4)


def test_harmonic_ritz_with_full_space_gives_eigenvalues():
    n = 12
    A = np.diag(np.arange(1, n + 1).astype(complex)) + 0.1 * np.triu(synth.complex_gaussian((n, n), 13), 1)
    b = synth.complex_gaussian((n,), 14)
    V = np.zeros((n + 1, n), dtype=np.complex128)
    H = np.zeros((n + 1, n), dtype=np.complex128)
    V[0] = b / np.linalg.norm(b)
    for j in range(n):
        h, w = krylov.cgs2(V[: j + 1], A @ V[j])
        H[: j + 1, j] = h
        H[j + 1, j] = np.linalg.norm(w)
        if j + 1 < n:
            V[j + 1] = w / H[j + 1, j]
    theta, _ = krylov.harmonic_ritz(H, n, 4)
    assert np.allclose(np.sort(np.abs(theta)), [1, 2, 3, 4], atol=1e-8)


def test_gmres_proj_projection_is_min_residual(coarse32):
    _, A2 = coarse32
    n = A2.shape[0]
    _, _, defl = krylov.gmres_dr(lambda v: A2 @ v, synth.complex_gaussian((n,), 15), 30, 10, 1e-12)
    b = synth.complex_gaussian((n,), 16)
    Wk = defl.W[: defl.k].T
    d, _ = krylov.lsq(defl.Hk, defl.W.conj() @ b)
    dd = np.linalg.lstsq(A2 @ Wk, b, rcond=None)[0]
    assert np.linalg.norm(Wk @ d - Wk @ dd) <= 1e-9 * np.linalg.norm(Wk @ dd)
    x, info = krylov.gmres_proj(lambda v: A2 @ v, b, defl, 30, 1e-10)
    assert info.converged
    assert np.linalg.norm(A2 @ x - b) <= 1.01e-10 * np.linalg.norm(b)


def test_gmres_proj_exact_invariant_subspace_one_step(coarse32):
    _, A2 = coarse32
    n = A2.shape[0]
    k = 6
    lam, X = np.linalg.eig(A2)
    idx = np.argsort(np.abs(lam))[:k]
    Qk = np.linalg.qr(X[:, idx])[0]
    extra = synth.complex_gaussian((n,), 18)
    extra -= Qk @ (Qk.conj().T @ extra)
    W = np.concatenate([Qk, (extra / np.linalg.norm(extra))[:, None]], axis=1)
    Hk = W.conj().T @ A2 @ Qk
    defl = krylov.Deflation(W.T.copy(), Hk)
    b = Qk @ synth.complex_gaussian((k,), 19)
    x, info = krylov.gmres_proj(lambda v: A2 @ v, b, defl, 30, 1e-10)
    assert info.converged and info.iters == 0
    assert np.linalg.norm(A2 @ x - b) <= 1e-12 * np.linalg.norm(b)


def test_cgne_matches_lu(coarse32):
    _, A2 = coarse32
    b = synth.complex_gaussian((A2.shape[0],), 20)
    x, info = krylov.cgne(lambda v: A2 @ v, lambda v: A2.conj().T @ v, b, 1e-11)
    xs = np.linalg.solve(A2, b)
    assert info.converged
    assert np.linalg.norm(x - xs) <= np.linalg.cond(A2) * 1e-11 * np.linalg.norm(xs)
