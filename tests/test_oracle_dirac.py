"""Pins of the oracle's Wilson-Dirac operator and stencils (CPU only).

Each check is fixed by the mathematics of the operator of Section 2, not by
re-typing the oracle's formula:
* free field (U = 1): the spectrum is known in closed form in momentum space
  with antiperiodic t momenta p_t = 2 pi (n + 1/2) / L;
* sigma3-hermiticity D^+ = sigma_3 D sigma_3;
* gauge covariance: U_mu(s) -> g(s) U_mu(s) g(s+mu)^*, psi -> g psi;
* the hop structure: every off-diagonal spin block has rank one.
"""
import numpy as np
import pytest

import synth
from oracle import dirac


def free_field_spectrum(Lx, Lt, m0):
    px = 2 * np.pi * np.arange(Lx) / Lx
    pt = 2 * np.pi * (np.arange(Lt) + 0.5) / Lt
    PT, PX = np.meshgrid(pt, px, indexing="ij")
    re = m0 + (1 - np.cos(PX)) + (1 - np.cos(PT))
    im = np.sqrt(np.sin(PX) ** 2 + np.sin(PT) ** 2)
    return np.concatenate([(re + 1j * im).ravel(), (re - 1j * im).ravel()])


def _match_spectra(a, b):
    """max distance between two multisets of complex numbers (greedy on sorted keys)."""
    a = np.sort_complex(np.round(a, 9))
    b = np.sort_complex(np.round(b, 9))
    return np.max(np.abs(a - b))


@pytest.mark.parametrize("Lx,Lt,m0", [(4, 4, 0.0), (6, 6, 0.1), (8, 6, -0.3), (12, 8, 0.05)])
def test_free_field_spectrum_closed_form(Lx, Lt, m0):
    U = np.ones((Lt, Lx, 2), dtype=np.complex128)
    D = dirac.dense_from_apply(lambda v: dirac.wilson(U, v, m0), (Lt, Lx, 2))
    ev = np.linalg.eigvals(D)
    assert _match_spectra(ev, free_field_spectrum(Lx, Lt, m0)) < 1e-9


def test_free_field_detects_periodic_t():
    # the same closed form with periodic t momenta must NOT match (the pin sees the boundary)
    L, m0 = 6, 0.1
    U = np.ones((L, L, 2), dtype=np.complex128)
    D = dirac.dense_from_apply(lambda v: dirac.wilson(U, v, m0), (L, L, 2))
    ev = np.linalg.eigvals(D)
    px = 2 * np.pi * np.arange(L) / L
    PT, PX = np.meshgrid(px, px, indexing="ij")
    re = m0 + (1 - np.cos(PX)) + (1 - np.cos(PT))
    im = np.sqrt(np.sin(PX) ** 2 + np.sin(PT) ** 2)
    wrong = np.concatenate([(re + 1j * im).ravel(), (re - 1j * im).ravel()])
    assert _match_spectra(ev, wrong) > 1e-3


def test_sigma3_hermiticity():
    U = synth.heatbath(8, 8, 6.0, 50, 11)
    m0 = -0.07
    D = dirac.dense_from_apply(lambda v: dirac.wilson(U, v, m0), (8, 8, 2))
    S3 = np.kron(np.eye(64), np.diag([1.0, -1.0]))
    assert np.abs(D.conj().T - S3 @ D @ S3).max() < 1e-14
    Dd = dirac.dense_from_apply(lambda v: dirac.wilson_dagger(U, v, m0), (8, 8, 2))
    assert np.abs(Dd - D.conj().T).max() < 1e-14
    # D itself is not hermitian on a non-trivial field
    assert np.abs(D.conj().T - D).max() > 1e-2


def test_gauge_covariance():
    L, m0 = 8, 0.2
    U = synth.heatbath(L, L, 6.0, 30, 5)
    g = np.exp(1j * synth.complex_gaussian((L, L), 99).real * 3.0)
    Ug = np.empty_like(U)
    Ug[:, :, 0] = g * U[:, :, 0] * np.conj(np.roll(g, -1, axis=1))
    Ug[:, :, 1] = g * U[:, :, 1] * np.conj(np.roll(g, -1, axis=0))
    psi = synth.complex_gaussian((L, L, 2), 3)
    lhs = dirac.wilson(Ug, g[..., None] * psi, m0)
    rhs = g[..., None] * dirac.wilson(U, psi, m0)
    assert np.abs(lhs - rhs).max() < 1e-13


def test_stencil_form_equals_operator_and_hops_rank_one():
    L, m0 = 8, -0.05
    U = synth.heatbath(L, L, 6.0, 30, 7)
    A = dirac.wilson_stencil(U, m0)
    psi = synth.complex_gaussian((3, L, L, 2), 4)
    assert np.abs(dirac.stencil_apply(A, psi) - dirac.wilson(U, psi, m0)).max() < 1e-14
    for d in range(1, 5):
        s = np.linalg.svd(A[:, :, d], compute_uv=False)
        assert np.all(s[..., 1] < 1e-14) and np.all(np.abs(s[..., 0] - 1.0) < 1e-14)


def test_sparse_matrix_matches_apply():
    L, m0 = 8, 0.1
    U = synth.heatbath(L, L, 6.0, 20, 2)
    M = dirac.stencil_sparse(dirac.wilson_stencil(U, m0))
    psi = synth.complex_gaussian((L, L, 2), 8)
    assert np.abs(M @ psi.ravel() - dirac.wilson(U, psi, m0).ravel()).max() < 1e-14
