"""Oracle: the 2D Wilson-Dirac operator and the coarse block stencils (FP64).

Test infrastructure only (see ``oracle/__init__.py``).

The paper (Section 2) works with the Wilson-Dirac operator of the 2D lattice
Schwinger model on quenched U(1) fields, periodic in x and antiperiodic for the
fermion in t:

    (D psi)(s) = (m0 + 2) psi(s)
               - 1/2 sum_mu [ (1 - sigma_mu) U_mu(s) psi(s + mu)
                            + (1 + sigma_mu) U_mu(s - mu)^* psi(s - mu) ]

with sigma_1 (x) = [[0,1],[1,0]], sigma_2 (t) = [[0,-i],[i,0]]; a hop across
t = L_t - 1 <-> 0 carries a factor -1.  Its adjoint follows from
sigma3-hermiticity, D^+ = sigma_3 D sigma_3 (used by the null-vector normal
equations DD^+ of Section 2 and by CGNE).

Arrays: U complex128[L_t][L_x][2] (mu = 0: x, 1: t); psi complex128[...,L_t,L_x,2].
Coarse stencils (the Galerkin operators D^ = P^+ D P of Section 2) are stored
as A complex128[N_t][N_x][5][n][n] with directions (self, +x, -x, +t, -t):

    (A v)(s) = sum_d A[s, d] v(nbr(s, d)),  nbr(s, +x) = s + x^ (periodic).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

SIGMA1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
SIGMA2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
SIGMA3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
ID2 = np.eye(2, dtype=np.complex128)

# direction order of every stencil: self, +x, -x, +t, -t
DIRS = ("self", "+x", "-x", "+t", "-t")


def _spin(M, v):
    """Apply a 2x2 spin matrix M to the last axis of v."""
    return np.einsum("ab,...b->...a", M, v)


def _t_signs(Lt):
    """Antiperiodic fermion boundary in t: forward hop from t = L_t-1 and
    backward hop from t = 0 cross the boundary and pick up -1."""
    fwd = np.ones(Lt)
    bwd = np.ones(Lt)
    fwd[Lt - 1] = -1.0
    bwd[0] = -1.0
    return fwd[:, None, None], bwd[:, None, None]


def wilson(U, psi, m0):
    """D psi, written term by term from the definition in the module docstring."""
    Lt, Lx = U.shape[:2]
    out = (m0 + 2.0) * psi
    # x direction (axis -2 of psi), periodic
    Ux = U[:, :, 0][..., None]
    Ux_back = np.conj(np.roll(U[:, :, 0], 1, axis=1))[..., None]  # U_x(s - x^)^*
    fwd = Ux * np.roll(psi, -1, axis=-2)  # U_x(s) psi(s + x^)
    bwd = Ux_back * np.roll(psi, 1, axis=-2)  # U_x(s - x^)^* psi(s - x^)
    out = out - 0.5 * (_spin(ID2 - SIGMA1, fwd) + _spin(ID2 + SIGMA1, bwd))
    # t direction (axis -3 of psi), antiperiodic
    sf, sb = _t_signs(Lt)
    Ut = U[:, :, 1][..., None]
    Ut_back = np.conj(np.roll(U[:, :, 1], 1, axis=0))[..., None]  # U_t(s - t^)^*
    fwd = sf * Ut * np.roll(psi, -1, axis=-3)
    bwd = sb * Ut_back * np.roll(psi, 1, axis=-3)
    out = out - 0.5 * (_spin(ID2 - SIGMA2, fwd) + _spin(ID2 + SIGMA2, bwd))
    return out


def gamma5(psi):
    """sigma_3 on the spin index (the 2D gamma_5)."""
    out = psi.copy()
    out[..., 1] *= -1.0
    return out


def wilson_dagger(U, psi, m0):
    """D^+ psi = sigma_3 D sigma_3 psi (sigma3-hermiticity)."""
    return gamma5(wilson(U, gamma5(psi), m0))


def wilson_stencil(U, m0):
    """The same operator as 5 spin blocks per site, in the stencil layout.

    A[s, +x] = -1/2 (1 - sigma_1) U_x(s)      acting on psi(s + x^), etc.
    Antiperiodic signs are folded into the t blocks.
    """
    Lt, Lx = U.shape[:2]
    A = np.zeros((Lt, Lx, 5, 2, 2), dtype=np.complex128)
    A[:, :, 0] = (m0 + 2.0) * ID2
    sf, sb = _t_signs(Lt)
    Ux = U[:, :, 0]
    Ut = U[:, :, 1]
    A[:, :, 1] = -0.5 * Ux[..., None, None] * (ID2 - SIGMA1)
    A[:, :, 2] = -0.5 * np.conj(np.roll(Ux, 1, axis=1))[..., None, None] * (ID2 + SIGMA1)
    A[:, :, 3] = -0.5 * (sf[..., None] * Ut[..., None, None]) * (ID2 - SIGMA2)
    A[:, :, 4] = -0.5 * (sb[..., None] * np.conj(np.roll(Ut, 1, axis=0))[..., None, None]) * (ID2 + SIGMA2)
    return A


def neighbour(v, d, axes=(-3, -2)):
    """v(nbr(s, d)) for every site s; the sites of v lie on axes = (t, x)."""
    ta, xa = axes
    if d == 0:
        return v
    if d == 1:
        return np.roll(v, -1, axis=xa)
    if d == 2:
        return np.roll(v, 1, axis=xa)
    if d == 3:
        return np.roll(v, -1, axis=ta)
    return np.roll(v, 1, axis=ta)


def stencil_apply(A, v):
    """(A v)(s) = sum_d A[s, d] v(nbr(s, d)); v complex[..., N_t, N_x, n].

    Each term is a batch of per-site matrix-vector products (numpy matmul)."""
    Nt, Nx, _, n, _ = A.shape
    lead = v.shape[:-3]
    nb_ = int(np.prod(lead)) if lead else 1
    out = np.zeros((Nt * Nx, n, nb_), dtype=np.complex128)
    for d in range(5):
        x = neighbour(v, d).reshape(nb_, Nt * Nx, n).transpose(1, 2, 0)  # [site][l][batch]
        out = out + np.matmul(A[:, :, d].reshape(Nt * Nx, n, n), x)
    return out.transpose(2, 0, 1).reshape(lead + (Nt, Nx, n))


def stencil_dagger_sigma(A, v):
    """sigma3-hat A sigma3-hat v with sigma3-hat = diag(+1 x n/2, -1 x n/2):
    the adjoint of a Galerkin operator (D^^+ = s3^ D^ s3^, Section 2)."""
    n = A.shape[-1]
    s = np.concatenate([np.ones(n // 2), -np.ones(n // 2)])
    return s * stencil_apply(A, s * v)


def stencil_sparse(A):
    """Sparse CSR matrix of a stencil, site index x + N_x t, dof fastest."""
    Nt, Nx, _, n, _ = A.shape
    t, x = np.meshgrid(np.arange(Nt), np.arange(Nx), indexing="ij")
    site = (x + Nx * t).ravel()
    nbrs = [site,
            ((x + 1) % Nx + Nx * t).ravel(),
            ((x - 1) % Nx + Nx * t).ravel(),
            (x + Nx * ((t + 1) % Nt)).ravel(),
            (x + Nx * ((t - 1) % Nt)).ravel()]
    rows, cols, vals = [], [], []
    k = np.arange(n)
    for d in range(5):
        blk = A[:, :, d].reshape(-1, n, n)
        r = (site[:, None, None] * n + k[None, :, None]) + 0 * k[None, None, :]
        c = (nbrs[d][:, None, None] * n + k[None, None, :]) + 0 * k[None, :, None]
        rows.append(r.ravel())
        cols.append(c.ravel())
        vals.append(blk.ravel())
    N = Nt * Nx * n
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))


def dense_from_apply(apply, shape):
    """Dense matrix of a linear map on complex arrays of the given shape (tiny cases)."""
    n = int(np.prod(shape))
    M = np.zeros((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1.0
        M[:, j] = apply(e.reshape(shape)).ravel()
    return M
