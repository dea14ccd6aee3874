"""Pins of the oracle's V-cycle and two-grid cycle (Section 2) and of its m0 search.

The outer solver is flexible, so a V-cycle with a missing, misplaced or
misdirected step still converges; these checks fix the cycle itself:

* operator applications per grid in one cycle: on a grid that smooths,
  GMRES(2) pre-smoothing (2), the residual after the correction (1) and
  GMRES(2) post-smoothing (2), i.e. 5, plus exactly one coarsest solve;
* with the coarsest solve replaced by an exact dense solve, one V-cycle equals
  the same steps written with dense matrices assembled independently of the
  oracle's stencils (dense D, dense prolongators, D^ = P^+ D P, and GMRES(2)
  as the minimum residual over span{f, A f});
* the leftmost eigenvalues found by shift-invert Arnoldi (the m0 search)
  against a dense eigendecomposition of D(0), and the tabulated m0 placing the
  smallest real part of the spectrum of D(m0) at 1e-3.
"""
import numpy as np
import pytest

import synth
from oracle import dirac, hierarchy, mg, tune_m0


def _setup(L, c=0):
    U = synth.gauge_field(L, c, cache=False)
    m0 = synth.m0_for(L, c)
    h = hierarchy.build(U, m0, synth.nullvec_starts(L, c, 0, 12, L * L * 2),
                        synth.nullvec_starts(L, c, 1, 12, (L // 4) ** 2 * 24))
    return U, m0, h


@pytest.fixture(scope="module")
def h16():
    return _setup(16)


@pytest.fixture(scope="module")
def dense16(h16):
    U, m0, h = h16
    L = 16
    D0 = dirac.dense_from_apply(lambda v: dirac.wilson(U, v, m0), (L, L, 2))
    P0 = hierarchy.dense_prolongator(h.Q0, (L, L, 2))
    D1 = P0.conj().T @ D0 @ P0
    P1 = hierarchy.dense_prolongator(h.Q1, h.shapes[1])
    D2 = P1.conj().T @ D1 @ P1
    return D0, P0, D1, P1, D2


def _gmres2_dense(A, f):
    """GMRES(2) from zero: x = argmin over span{f, A f} of ||f - A x||."""
    K = np.stack([f, A @ f], axis=1)
    c = np.linalg.lstsq(A @ K, f, rcond=None)[0]
    return K @ c


def _vcycle_dense(D, P, f, level, drop_post=False):
    """x = S(f); r = f - A x; x += P (next grid on P^+ r); r = f - A x; x += S(r)."""
    A = D[level]
    x = _gmres2_dense(A, f)
    r = f - A @ x
    rc = P[level].conj().T @ r
    ec = np.linalg.solve(D[2], rc) if level == 1 else _vcycle_dense(D, P, rc, 1, drop_post)
    x = x + P[level] @ ec
    if drop_post:
        return x
    r = f - A @ x
    return x + _gmres2_dense(A, r)


def _exact_coarse(s, D2):
    def solve(f):
        s.coarse_solves.append(("exact", 0))
        return np.linalg.solve(D2, f)
    s.coarse_solve = solve


def test_vcycle_operator_applications_per_grid(h16):
    U, m0, h = h16
    s = mg.MGSolver(h)
    f = synth.complex_gaussian((h.size(0),), 31, 0)
    s.vcycle(0, f)  # the first coarse solve builds the deflation space (GMRES-DR)
    for trial in range(2):
        s.counter.mvps = [0, 0, 0]
        n_before = len(s.coarse_solves)
        s.vcycle(0, synth.complex_gaussian((h.size(0),), 31, 1 + trial))
        new = s.coarse_solves[n_before:]
        assert len(new) == 1 and new[0][0] == "proj"
        assert s.counter.mvps[0] == 2 + 1 + 2
        assert s.counter.mvps[1] == 2 + 1 + 2
        assert s.counter.mvps[2] == new[0][1]  # every coarse application is a GMRES-Proj step
    # the two-grid cycle of the intermediate grid: 5 intermediate applications, one coarse solve
    s.counter.mvps = [0, 0, 0]
    n_before = len(s.coarse_solves)
    s.twogrid(synth.complex_gaussian((h.size(1),), 31, 9))
    assert s.counter.mvps[0] == 0 and s.counter.mvps[1] == 5
    assert len(s.coarse_solves) == n_before + 1


def test_vcycle_equals_dense_steps(h16, dense16):
    U, m0, h = h16
    D0, P0, D1, P1, D2 = dense16
    s = mg.MGSolver(h)
    _exact_coarse(s, D2)
    for seed in range(3):
        f = synth.complex_gaussian((h.size(0),), 41, seed)
        x = s.vcycle(0, f)
        xd = _vcycle_dense((D0, D1, D2), (P0, P1), f, 0)
        assert np.linalg.norm(x - xd) <= 1e-11 * np.linalg.norm(xd)
    # the comparison resolves single steps: the same cycle without its
    # post-smoothers is far from the oracle's output
    x_nopost = _vcycle_dense((D0, D1, D2), (P0, P1), f, 0, drop_post=True)
    assert np.linalg.norm(x - x_nopost) > 1e-3 * np.linalg.norm(xd)


def test_twogrid_equals_dense_steps(h16, dense16):
    U, m0, h = h16
    D0, P0, D1, P1, D2 = dense16
    s = mg.MGSolver(h)
    _exact_coarse(s, D2)
    f = synth.complex_gaussian((h.size(1),), 43, 0)
    x = s.twogrid(f)
    xd = _vcycle_dense((D0, D1, D2), (P0, P1), f, 1)
    assert np.linalg.norm(x - xd) <= 1e-11 * np.linalg.norm(xd)


def test_vcycle_with_exact_coarse_solve_reduces_error(h16, dense16):
    # a correct two-level correction with an exact coarsest solve contracts the
    # error of a random f: ||f - D0 x|| well below ||f||
    U, m0, h = h16
    D0, P0, D1, P1, D2 = dense16
    s = mg.MGSolver(h)
    _exact_coarse(s, D2)
    f = synth.complex_gaussian((h.size(0),), 47, 0)
    x = s.vcycle(0, f)
    assert np.linalg.norm(f - D0 @ x) < 0.5 * np.linalg.norm(f)


@pytest.mark.parametrize("L", [16, 32])
def test_leftmost_eigs_match_dense_spectrum(L):
    U = synth.gauge_field(L, 0, cache=False)
    D = dirac.dense_from_apply(lambda v: dirac.wilson(U, v, 0.0), (L, L, 2))
    ev = np.linalg.eigvals(D)
    got = tune_m0.leftmost_eigs(U)
    # the leftmost eigenvalue is found, and every returned value is an eigenvalue
    assert abs(np.min(got.real) - np.min(ev.real)) <= 1e-9
    for lam in got:
        assert np.min(np.abs(ev - lam)) <= 1e-8
    # the tabulated m0 puts the smallest real part of the spectrum of D(m0) at 1e-3
    m0 = synth.m0_for(L, 0)
    assert abs(np.min(ev.real) + m0 - tune_m0.TARGET) <= 1e-9
