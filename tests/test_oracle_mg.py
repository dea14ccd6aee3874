"""Pins of the oracle's whole solve (Section 2) and of the Mvps count (Section 3, Eq. 1).

* deflated MG-FGMRES reaches the requested true residual and agrees with a
  direct sparse LU solve to within kappa * tol;
* the CGNE comparison arm solves the same system;
* the deflation space is built by the first coarse solve and reused (GMRES-Proj)
  by every later coarse solve, also for a second right-hand side;
* Eq. 1's dimension ratios n_int / n_fine = 0.75 and n_coarse / n_fine = 3/64;
* the partial intermediate solve (Section 2's variant): each intermediate solve
  meets ||f - P^+ D P x|| <= 0.2 ||f|| with the product of independently
  assembled dense matrices; the whole solve still agrees with a direct solve;
  and the coarse tolerances follow the schedule: 1e-8 within a right-hand
  side's first outer iteration (GMRES-DR first), 1e-2 after it.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import dirac, hierarchy, mg


def _setup(L, c=0):
    U = synth.gauge_field(L, c, cache=False)
    m0 = synth.m0_for(L, c)
    h = hierarchy.build(U, m0, synth.nullvec_starts(L, c, 0, 12, L * L * 2),
                        synth.nullvec_starts(L, c, 1, 12, (L // 4) ** 2 * 24))
    return U, m0, h


@pytest.fixture(scope="module")
def h16():
    return _setup(16)


def _direct(U, m0, b):
    A = dirac.stencil_sparse(dirac.wilson_stencil(U, m0)).tocsc()
    return spla.splu(A).solve(b.ravel()), A


def test_deflated_mg_solve_matches_direct(h16):
    U, m0, h = h16
    b = synth.rhs(16, 0, 0)[0]
    s = mg.MGSolver(h)
    x, info = s.solve(b, 1e-10)
    xs, A = _direct(U, m0, b)
    assert info.converged and info.relres <= 1e-10
    assert np.linalg.norm(A @ x.ravel() - b.ravel()) <= 1e-10 * np.linalg.norm(b)
    smin = np.linalg.svd(A.toarray(), compute_uv=False)[-1]
    kappa = np.linalg.norm(A.toarray(), 2) / smin
    assert np.linalg.norm(x.ravel() - xs) <= kappa * 1e-10 * np.linalg.norm(xs)
    kinds = [k for k, _ in s.coarse_solves]
    assert kinds[0] == "dr" and all(k == "proj" for k in kinds[1:])
    # a second right-hand side reuses the deflation space: no GMRES-DR
    n_before = len(kinds)
    x2, info2 = s.solve(synth.rhs(16, 0, 1)[0], 1e-10)
    assert info2.converged
    assert all(k == "proj" for k, _ in s.coarse_solves[n_before:])


def test_cgne_arm_solves(h16):
    U, m0, h = h16
    b = synth.rhs(16, 0, 2)[0]
    s = mg.MGSolver(h, mg.Params(coarse="cgne"))
    x, info = s.solve(b, 1e-9)
    assert info.converged
    assert np.linalg.norm(dirac.wilson(U, x, m0) - b) <= 1e-9 * np.linalg.norm(b)
    assert all(k == "cgne" for k, _ in s.coarse_solves)


def test_deflation_lowers_coarse_work():
    # Section 3: deflation cuts the coarse operator applications per outer iteration
    U, m0, h = _setup(32)
    b = synth.rhs(32, 0, 0)[0]
    sd = mg.MGSolver(h)
    sd.solve(b, 1e-8)
    sd.counter.mvps = [0, 0, 0]
    sd.coarse_solves = []
    _, info_d = sd.solve(synth.rhs(32, 0, 1)[0], 1e-8)  # GMRES-Proj only
    sc = mg.MGSolver(h, mg.Params(coarse="cgne"))
    _, info_c = sc.solve(synth.rhs(32, 0, 1)[0], 1e-8)
    per_outer_d = sd.counter.mvps[2] / max(info_d.iters, 1)
    per_outer_c = sc.counter.mvps[2] / max(info_c.iters, 1)
    assert per_outer_d < per_outer_c


def test_fine_equivalent_mvps_ratios():
    U = np.ones((64, 64, 2), dtype=np.complex128)
    Q0 = np.zeros((16, 16, 2, 12, 16, 1), dtype=np.complex128)
    A1 = np.zeros((16, 16, 5, 24, 24), dtype=np.complex128)
    Q1 = np.zeros((4, 4, 2, 12, 16, 12), dtype=np.complex128)
    A2 = np.zeros((4, 4, 5, 24, 24), dtype=np.complex128)
    h = hierarchy.Hierarchy(U, 0.0, Q0, A1, Q1, A2)
    assert h.size(1) / h.size(0) == 0.75
    assert h.size(2) / h.size(0) == 3 / 64
    s = mg.MGSolver(h)
    s.counter.mvps = [10, 100, 1000]
    assert s.fine_equivalent_mvps() == 10 + 75 + 1000 * 3 / 64


def test_partial_intermediate_solve(h16):
    U, m0, h = h16
    L = 16
    # dense P^+ D P, assembled from the fine operator and the prolongator matrix
    D = dirac.dense_from_apply(lambda v: dirac.wilson(U, v, m0), (L, L, 2))
    P = hierarchy.dense_prolongator(h.Q0, (L, L, 2))
    A1 = P.conj().T @ D @ P
    s = mg.MGSolver(h, mg.Params(partial_tol=0.2))
    b = synth.rhs(16, 0, 3)[0]
    x, info = s.solve(b, 1e-10)
    xs, A = _direct(U, m0, b)
    assert info.converged and np.linalg.norm(A @ x.ravel() - b.ravel()) <= 1e-10 * np.linalg.norm(b)
    smin = np.linalg.svd(A.toarray(), compute_uv=False)[-1]
    kappa = np.linalg.norm(A.toarray(), 2) / smin
    assert np.linalg.norm(x.ravel() - xs) <= kappa * 1e-10 * np.linalg.norm(xs)
    assert s.partial_solves and all(rr <= 0.2 for _, rr in s.partial_solves)
    # one intermediate solve by itself, checked with the dense operator
    f = synth.complex_gaussian((A1.shape[0],), 7, 3)
    x1 = s.partial_solve(f)
    assert np.linalg.norm(f - A1 @ x1) <= 0.2 * np.linalg.norm(f)
    # tolerance schedule of the coarse solves
    kinds = [k for k, _ in s.coarse_solves]
    assert kinds[0] == "dr" and s.coarse_tols[0] == 1e-8
    assert 1e-2 in s.coarse_tols
    first_loose = s.coarse_tols.index(1e-2)
    assert all(t == 1e-8 for t in s.coarse_tols[:first_loose])
    assert all(t == 1e-2 for t in s.coarse_tols[first_loose:])
    # a second right-hand side: projected solves only, 1e-8 again in its first outer iteration
    n0 = len(s.coarse_tols)
    x2, info2 = s.solve(synth.rhs(16, 0, 4)[0], 1e-10)
    assert info2.converged
    assert all(k == "proj" for k, _ in s.coarse_solves[n0:])
    assert s.coarse_tols[n0] == 1e-8 and s.coarse_tols[-1] == 1e-2
