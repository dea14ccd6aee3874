"""Oracle: the adaptive multigrid set-up (FP64), Section 2, first paragraph.

Test infrastructure only (see ``oracle/__init__.py``).

The paper builds each coarser grid as follows:

1. near-null vectors: from random x, solve  A A^+ e = -A A^+ x  to relative
   tolerance 1e-4 and set psi = x + e (12 vectors);
2. global orthonormalisation of the 12 vectors;
3. chiral doubling with the projectors (1 +/- sigma_3)/2;
4. local 4^2 blocking and local orthonormalisation -> the columns of P;
5. Galerkin operator  A^ = P^+ A P;
and then repeats 1-5 on A^ to build the coarsest operator.

Readings where the paper is silent:
* the near-null solver is CG on A A^+ (Hermitian positive definite), stopped on
  the recursive residual ||r|| <= tol ||A A^+ x||;
* Gram-Schmidt is modified Gram-Schmidt in vector order, globally and locally;
* coarse dof index k = 12 c + j (chirality c, vector j);
* the intermediate grid's chirality is sigma3^ = P^+ sigma_3 P = diag(+1 x 12,
  -1 x 12) and its adjoint is A^+ = sigma3^ A sigma3^; the repeat uses both;
* a local column whose norm after orthogonalisation falls below 1e-12 of its
  norm before is a rank deficiency and is an error (no column is dropped).

Prolongator layout Q[B_t][B_x][c][j][l][a]: block B, chirality c, vector j,
site l = lx + 4 lt inside the 4x4 block, dof a of chirality c at that site
(1 dof on the fine grid, 12 on the intermediate grid).
"""
from __future__ import annotations

import numpy as np

from . import dirac

BLOCK = 4


def cg_normal(apply_A, apply_Ad, x0s, tol, maxiter=100000):
    """Near-null vectors: for each row x of x0s solve A A^+ e = -A A^+ x by CG
    from e = 0 until ||r|| <= tol ||A A^+ x||; return psi = x + e and the
    iteration counts.  apply_* act on arrays with the vectors on axis 0."""
    X = np.array(x0s, dtype=np.complex128)
    nv = X.shape[0]
    flat = X.reshape(nv, -1)
    AAd = lambda v: apply_A(apply_Ad(v.reshape(X.shape))).reshape(nv, -1)
    b = -AAd(flat)
    e = np.zeros_like(flat)
    r = b.copy()
    p = r.copy()
    rr = np.einsum("ij,ij->i", r.conj(), r).real
    bnorm = np.sqrt(np.einsum("ij,ij->i", b.conj(), b).real)
    active = np.sqrt(rr) > tol * bnorm
    iters = np.zeros(nv, dtype=int)
    it = 0
    while active.any() and it < maxiter:
        q = AAd(p)
        pq = np.einsum("ij,ij->i", p.conj(), q).real
        alpha = np.where(active, rr / np.where(active, pq, 1.0), 0.0)
        e = e + alpha[:, None] * p
        r = r - alpha[:, None] * q
        rr_new = np.einsum("ij,ij->i", r.conj(), r).real
        beta = np.where(active, rr_new / np.where(active, rr, 1.0), 0.0)
        p = np.where(active[:, None], r + beta[:, None] * p, p)
        rr = np.where(active, rr_new, rr)
        iters = iters + active
        active = active & (np.sqrt(rr) > tol * bnorm)
        it += 1
    return (flat + e).reshape(X.shape), iters


def mgs_rows(V):
    """Modified Gram-Schmidt of the rows of V (in row order)."""
    V = np.array(V, dtype=np.complex128)
    for j in range(V.shape[0]):
        for i in range(j):
            V[j] = V[j] - np.vdot(V[i], V[j]) * V[i]
        V[j] = V[j] / np.linalg.norm(V[j])
    return V


def local_blocks(vecs, block=BLOCK):
    """Split vectors complex[nv][N_t][N_x][n] into complex[B_t][B_x][2][nv][16][n/2]:
    chirality c keeps dofs c*n/2 .. (c+1)*n/2 - 1 (chiral doubling)."""
    nv, Nt, Nx, n = vecs.shape
    h = n // 2
    v = vecs.reshape(nv, Nt // block, block, Nx // block, block, 2, h)
    # -> [Bt][Bx][c][j][lt][lx][a]
    v = v.transpose(1, 3, 5, 0, 2, 4, 6)
    return v.reshape(Nt // block, Nx // block, 2, nv, block * block, h)


def local_orthonormalise(blocks, rank_tol=1e-12):
    """MGS over the vector index j inside every (block, chirality)."""
    Q = np.array(blocks, dtype=np.complex128)
    nv = Q.shape[3]
    for j in range(nv):
        before = np.sqrt(np.sum(np.abs(Q[:, :, :, j]) ** 2, axis=(-2, -1)))
        for i in range(j):
            ov = np.sum(np.conj(Q[:, :, :, i]) * Q[:, :, :, j], axis=(-2, -1))
            Q[:, :, :, j] = Q[:, :, :, j] - ov[..., None, None] * Q[:, :, :, i]
        nrm = np.sqrt(np.sum(np.abs(Q[:, :, :, j]) ** 2, axis=(-2, -1)))
        if np.any(nrm <= rank_tol * before):
            raise ValueError("rank-deficient local block in the prolongator")
        Q[:, :, :, j] = Q[:, :, :, j] / nrm[..., None, None]
    return Q


def prolongator(nullvecs, block=BLOCK):
    """Steps 2-4: global MGS, chiral doubling, local blocking + local MGS.
    nullvecs complex[nv][N_t][N_x][n] -> Q (layout in the module docstring)."""
    nv = nullvecs.shape[0]
    G = mgs_rows(nullvecs.reshape(nv, -1)).reshape(nullvecs.shape)
    return local_orthonormalise(local_blocks(G, block))


def restrict(Q, v, block=BLOCK):
    """v^ = P^+ v:  v^[B, 12c + j] = sum_{l,a} conj(Q[B,c,j,l,a]) v[s(B,l), c h + a]."""
    Bt, Bx, _, nv, _, h = Q.shape
    lead = v.shape[:-3]
    b = len(lead)
    w = v.reshape(lead + (Bt, block, Bx, block, 2, h))  # [..., Bt, lt, Bx, lx, c, a]
    w = w.transpose(tuple(range(b)) + tuple(b + i for i in (0, 2, 4, 1, 3, 5)))  # [..., Bt, Bx, c, lt, lx, a]
    w = w.reshape(lead + (Bt, Bx, 2, block * block, h))
    out = np.einsum("tzcjla,...tzcla->...tzcj", np.conj(Q), w)
    return out.reshape(lead + (Bt, Bx, 2 * nv))


def prolong(Q, vc, block=BLOCK):
    """v = P v^:  v[s(B,l), c h + a] = sum_j Q[B,c,j,l,a] v^[B, 12c + j]."""
    Bt, Bx, _, nv, L2, h = Q.shape
    lead = vc.shape[:-3]
    w = vc.reshape(lead + (Bt, Bx, 2, nv))
    f = np.einsum("tzcjla,...tzcj->...tzcla", Q, w)  # [..., Bt, Bx, c, l, a]
    b = len(lead)
    f = f.reshape(lead + (Bt, Bx, 2, block, block, h))  # l = lx + 4 lt -> (lt, lx)
    f = f.transpose(tuple(range(b)) + tuple(b + i for i in (0, 3, 1, 4, 2, 5)))  # [..., Bt, lt, Bx, lx, c, a]
    return f.reshape(lead + (Bt * block, Bx * block, 2 * h))


def site_matrices(Q, block=BLOCK):
    """P restricted to each finer site: complex[N_t][N_x][n][2 nv] with
    P_s[c h + a, 12 c + j] = Q[B(s), c, j, l(s), a]."""
    Bt, Bx, _, nv, _, h = Q.shape
    Ps = np.zeros((Bt, Bx, block * block, 2 * h, 2 * nv), dtype=np.complex128)
    for c in range(2):
        # Q[..., c, j, l, a] -> [..., l, a, j]
        Ps[:, :, :, c * h:(c + 1) * h, c * nv:(c + 1) * nv] = np.transpose(Q[:, :, c], (0, 1, 3, 4, 2))
    Ps = Ps.reshape(Bt, Bx, block, block, 2 * h, 2 * nv)  # l -> (lt, lx)
    Ps = Ps.transpose(0, 2, 1, 3, 4, 5)
    return Ps.reshape(Bt * block, Bx * block, 2 * h, 2 * nv)


def galerkin(A, Q, block=BLOCK):
    """Step 5: the coarse stencil of P^+ A P from a finer stencil A.

    A finer term A[s, d] v(nbr(s, d)) lands in coarse block B(s); it stays in the
    coarse 'self' entry unless the hop leaves the block through its face (local
    coordinate block-1 for +x/+t, 0 for -x/-t), in which case it lands in the
    coarse entry of the same direction:
        Ac[B, dir] += P_s^+ A[s, d] P_{nbr(s, d)}.
    """
    Nt, Nx = A.shape[:2]
    Bt, Bx = Nt // block, Nx // block
    Ps = site_matrices(Q, block)
    nc = Ps.shape[-1]
    Ac = np.zeros((Bt, Bx, 5, nc, nc), dtype=np.complex128)
    t, x = np.meshgrid(np.arange(Nt), np.arange(Nx), indexing="ij")
    lx, lt = x % block, t % block
    cross = {1: lx == block - 1, 2: lx == 0, 3: lt == block - 1, 4: lt == 0}
    for d in range(5):
        # left[s] = P_s^+ A[s, d]  (nc x n),  right[s] = P_nbr(s,d)  (n x nc)
        left = np.einsum("tzak,tzab->tzkb", np.conj(Ps), A[:, :, d])
        right = dirac.neighbour(Ps, d, axes=(0, 1))
        n = right.shape[-2]
        R = right.reshape(Bt, block, Bx, block, n, nc).transpose(0, 2, 1, 3, 4, 5).reshape(Bt, Bx, -1, nc)
        mask_out = cross[d] if d else np.zeros_like(lx, dtype=bool)
        for dest, m in ((0, ~mask_out), (d, mask_out)):
            if not m.any():
                continue
            # sum over the block's sites s (and the dof index) of P_s^+ A[s, d] P_nbr(s,d)
            Lm = (left * m[..., None, None]).reshape(Bt, block, Bx, block, nc, n)
            Lm = Lm.transpose(0, 2, 4, 1, 3, 5).reshape(Bt, Bx, nc, -1)
            Ac[:, :, dest] += np.matmul(Lm, R)
    return Ac


def dense_prolongator(Q, fine_shape, block=BLOCK):
    """Dense P (n_fine x n_coarse), columns = prolong(unit vectors) (tiny cases)."""
    Bt, Bx, _, nv, _, _ = Q.shape
    nc = Bt * Bx * 2 * nv
    P = np.zeros((int(np.prod(fine_shape)), nc), dtype=np.complex128)
    for j in range(nc):
        e = np.zeros(nc, dtype=np.complex128)
        e[j] = 1.0
        P[:, j] = prolong(Q, e.reshape(Bt, Bx, 2 * nv), block).ravel()
    return P


class Hierarchy:
    """Three-grid hierarchy: fine Wilson operator, intermediate and coarse stencils.

    levels[0] = (None) fine grid: U, m0
    A1, Q0 : intermediate stencil and fine -> intermediate prolongator
    A2, Q1 : coarse stencil and intermediate -> coarse prolongator
    """

    def __init__(self, U, m0, Q0, A1, Q1, A2, null_iters=None):
        self.U = U
        self.m0 = m0
        self.Q0, self.A1, self.Q1, self.A2 = Q0, A1, Q1, A2
        self.null_iters = null_iters
        L_t, L_x = U.shape[:2]
        self.shapes = [(L_t, L_x, 2), A1.shape[:2] + (A1.shape[-1],), A2.shape[:2] + (A2.shape[-1],)]

    # operator applies on arrays of the level's shape (leading batch axes allowed)
    def apply(self, level, v):
        if level == 0:
            return dirac.wilson(self.U, v, self.m0)
        return dirac.stencil_apply(self.A1 if level == 1 else self.A2, v)

    def apply_dagger(self, level, v):
        if level == 0:
            return dirac.wilson_dagger(self.U, v, self.m0)
        return dirac.stencil_dagger_sigma(self.A1 if level == 1 else self.A2, v)

    def restrict(self, level, v):
        return restrict(self.Q0 if level == 0 else self.Q1, v)

    def prolong(self, level, vc):
        return prolong(self.Q0 if level == 0 else self.Q1, vc)

    def size(self, level):
        return int(np.prod(self.shapes[level]))


def nullvectors_level(apply, apply_dag, starts, tol):
    return cg_normal(apply, apply_dag, starts, tol)


def build(U, m0, starts0, starts1=None, nvec=12, tol=1e-4, nullvecs0=None, nullvecs1=None):
    """Full set-up.  starts0/starts1: random start vectors for the near-null
    solves on the fine and intermediate grids (complex[nv][n]); alternatively
    pass the near-null vectors themselves (nullvecs0/1, complex[nv][...])."""
    Lt, Lx = U.shape[:2]
    sh0 = (Lt, Lx, 2)
    it0 = it1 = None
    if nullvecs0 is None:
        nullvecs0, it0 = cg_normal(lambda v: dirac.wilson(U, v, m0), lambda v: dirac.wilson_dagger(U, v, m0),
                                   np.asarray(starts0).reshape((-1,) + sh0), tol)
    Q0 = prolongator(np.asarray(nullvecs0).reshape((-1,) + sh0))
    A1 = galerkin(dirac.wilson_stencil(U, m0), Q0)
    sh1 = A1.shape[:2] + (A1.shape[-1],)
    if nullvecs1 is None:
        nullvecs1, it1 = cg_normal(lambda v: dirac.stencil_apply(A1, v),
                                   lambda v: dirac.stencil_dagger_sigma(A1, v),
                                   np.asarray(starts1).reshape((-1,) + sh1), tol)
    Q1 = prolongator(np.asarray(nullvecs1).reshape((-1,) + sh1))
    A2 = galerkin(A1, Q1)
    h = Hierarchy(U, m0, Q0, A1, Q1, A2, null_iters=(it0, it1))
    h.nullvecs = (np.asarray(nullvecs0).reshape((-1,) + sh0), np.asarray(nullvecs1).reshape((-1,) + sh1))
    return h
