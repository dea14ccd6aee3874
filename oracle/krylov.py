"""Oracle: the Krylov solvers of the method (FP64), Section 2, second paragraph.

Test infrastructure only (see ``oracle/__init__.py``).

All vectors are flat complex128 arrays; operators are callables v -> A v.
Every Arnoldi process orthogonalises by classical Gram-Schmidt applied twice
(CGS2); every small least-squares problem min ||c - H d|| is solved with
numpy.linalg.lstsq (a library primitive), so the residual estimate after each
step is the plain definition  min_d ||c - H_j d||.

* arnoldi_run      - Arnoldi steps of one (F)GMRES cycle with per-step stopping
* smoother         - GMRES(2) from a zero guess (pre/post smoother, Section 2)
* fgmres           - FGMRES(m) [Saad 1993], right preconditioned, flexible,
                     convergence on the true residual ||b - A x|| / ||b||
* gmres_dr         - GMRES-DR(m,k) [Morgan 2002]: solves and deflates at once
* gmres_proj       - GMRES-Proj(m,k) [Morgan & Wilcox]: minres projection over
                     the deflation space alternating with GMRES(m-k) cycles
* cgne             - CG on A A^+ y = b, x = A^+ y (the undeflated comparison)

Readings where the paper is silent: the GMRES-Proj cycle length is m - k; a
GMRES-DR solve also ends after `stall` cycles without 0.1% progress or
`max_cycles` cycles, and always exports the deflation space (V_{k+1}, H_k) of
its last cycle (restarting that cycle once more when it ended early); the
restart's new right-hand side is c = P_{k+1}^+ rho; a zero Krylov vector
(exact breakdown) ends a cycle early.
"""
from __future__ import annotations

import numpy as np


def _norm(v):
    return float(np.sqrt(np.vdot(v, v).real))


def cgs2(V, w):
    """Orthogonalise w against the rows of V twice; return (h, w)."""
    h = V.conj() @ w
    w = w - V.T @ h
    h2 = V.conj() @ w
    w = w - V.T @ h2
    return h + h2, w


def lsq(H, c):
    """d = argmin ||c - H d|| and the residual vector rho = c - H d."""
    d = np.linalg.lstsq(H, c, rcond=None)[0]
    return d, c - H @ d


class Counter:
    """Operator applications per level (the Mvps of Section 3, Eq. 1)."""

    def __init__(self, nlevels=3):
        self.mvps = [0] * nlevels

    def wrap(self, level, apply):
        def f(v):
            self.mvps[level] += 1
            return apply(v)
        return f


def arnoldi_run(A, V, H, j0, jmax, c, tol_abs, precond=None, Z=None):
    """Arnoldi steps j0..jmax-1 on rows of V (V[j0] given), stopping as soon as
    min ||c - H_j d|| <= tol_abs.  Returns (j_end, d, rho, converged)."""
    j_end = j0
    d = np.zeros(0, dtype=np.complex128)
    rho = c[: j0 + 1].copy()
    conv = False
    for j in range(j0, jmax):
        z = V[j] if precond is None else precond(V[j])
        if Z is not None:
            Z[j] = z
        w = A(z)
        h, w = cgs2(V[: j + 1], w)
        H[: j + 1, j] = h
        hn = _norm(w)
        H[j + 1, j] = hn
        j_end = j + 1
        if hn > 0.0:
            V[j + 1] = w / hn
        d, rho = lsq(H[: j + 2, : j + 1], c[: j + 2])
        if _norm(rho) <= tol_abs or hn == 0.0:
            conv = _norm(rho) <= tol_abs
            break
    return j_end, d, rho, conv


def smoother(A, f, steps=2):
    """GMRES(steps) from x = 0 on A x = f.  Returns (x, r) with the new residual
    r = f - A x taken from the Arnoldi relation r = V_{steps+1}(beta e1 - H d)."""
    n = f.shape[0]
    beta = _norm(f)
    if beta == 0.0:
        return np.zeros_like(f), np.zeros_like(f)
    V = np.zeros((steps + 1, n), dtype=np.complex128)
    H = np.zeros((steps + 1, steps), dtype=np.complex128)
    V[0] = f / beta
    c = np.zeros(steps + 1, dtype=np.complex128)
    c[0] = beta
    for j in range(steps):
        w = A(V[j])
        h, w = cgs2(V[: j + 1], w)
        H[: j + 1, j] = h
        H[j + 1, j] = _norm(w)
        V[j + 1] = w / H[j + 1, j]
    d, rho = lsq(H, c)
    return V[:steps].T @ d, V.T @ rho


class SolveInfo:
    def __init__(self):
        self.iters = 0
        self.cycles = 0
        self.converged = False
        self.relres = np.inf
        self.history = []


def fgmres(A, b, M, tol, m=8, max_iters=1000, x0=None):
    """FGMRES(m): flexible right-preconditioned GMRES with restarts every m steps.

    z_j = M(v_j), A z_j = V_{j+1} H_j (flexible Arnoldi), x = x0 + Z_j d.
    A cycle stops early when min ||beta e1 - H_j d|| <= tol ||b||; after every
    cycle the true residual b - A x is recomputed (FP64) and decides convergence.
    """
    n = b.shape[0]
    nb = _norm(b)
    info = SolveInfo()
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    r = b - A(x) if x0 is not None else b.copy()
    if nb == 0.0:
        info.converged, info.relres = True, 0.0
        return x, info
    while True:
        beta = _norm(r)
        V = np.zeros((m + 1, n), dtype=np.complex128)
        Z = np.zeros((m, n), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        c = np.zeros(m + 1, dtype=np.complex128)
        c[0] = beta
        V[0] = r / beta
        jmax = min(m, max_iters - info.iters)
        j_end, d, rho, _ = arnoldi_run(A, V, H, 0, jmax, c, tol * nb, precond=M, Z=Z)
        info.iters += j_end
        info.cycles += 1
        x = x + Z[:j_end].T @ d
        r = b - A(x)
        info.relres = _norm(r) / nb
        info.history.append(info.relres)
        if info.relres <= tol:
            info.converged = True
            return x, info
        if info.iters >= max_iters:
            return x, info


class Deflation:
    """A deflation space (V_{k+1}, H_k) with A V_k = V_{k+1} H_k."""

    def __init__(self, W, Hk):
        self.W = W  # rows: k+1 orthonormal vectors
        self.Hk = Hk  # (k+1) x k
        self.k = Hk.shape[1]


def harmonic_ritz(H, j, k):
    """The k harmonic Ritz vectors of smallest |theta| of the j-step Arnoldi
    matrix H ((j+1) x j):  (H_j + |h_{j+1,j}|^2 H_j^{-H} e_j e_j^T) g = theta g.
    Ties in |theta| keep the lower index (stable sort)."""
    Hj = H[:j, :j]
    h = H[j, j - 1]
    ej = np.zeros(j, dtype=np.complex128)
    ej[j - 1] = 1.0
    f = np.linalg.solve(Hj.conj().T, ej)
    T = Hj.copy()
    T[:, j - 1] = T[:, j - 1] + abs(h) ** 2 * f
    theta, G = np.linalg.eig(T)
    order = np.argsort(np.abs(theta), kind="stable")[:k]
    return theta[order], G[:, order]


def dr_restart(V, H, j, k, rho):
    """GMRES-DR restart from a j-step cycle (rows V[0..j], H (j+1) x j) with LS
    residual rho (length j+1).  Returns (V_{k+1}, H_k, c) for the next cycle."""
    _, G = harmonic_ritz(H, j, k)
    P = np.zeros((j + 1, k + 1), dtype=np.complex128)
    P[:j, :k] = np.linalg.qr(G)[0]
    # append rho orthonormalised against the first k columns (twice)
    w = rho.copy()
    for _ in range(2):
        w = w - P[:, :k] @ (P[:, :k].conj().T @ w)
    P[:, k] = w / _norm(w)
    Vk1 = P.T @ V[: j + 1]  # new basis rows: V_{k+1} = V_{j+1} P
    Hk = P.conj().T @ H[: j + 1, :j] @ P[:j, :k]
    c = P.conj().T @ rho  # the residual V_{j+1} rho lies in span(V_{k+1})
    # reorthogonalise the last basis vector against the first k
    v = Vk1[k]
    v = v - Vk1[:k].T @ (Vk1[:k].conj() @ v)
    Vk1[k] = v / _norm(v)
    return Vk1, Hk, c


def gmres_dr(A, b, m, k, tol, max_cycles=100, stall=2):
    """GMRES-DR(m,k) from x = 0.  Returns (x, info, Deflation)."""
    n = b.shape[0]
    nb = _norm(b)
    info = SolveInfo()
    x = np.zeros(n, dtype=np.complex128)
    V = np.zeros((m + 1, n), dtype=np.complex128)
    H = np.zeros((m + 1, m), dtype=np.complex128)
    c = np.zeros(m + 1, dtype=np.complex128)
    c[0] = nb
    V[0] = b / nb
    j0 = 0
    defl = None
    best = np.inf
    stalled = 0
    while True:
        j_end, d, rho, conv = arnoldi_run(A, V, H, j0, m, c, tol * nb)
        info.iters += j_end - j0
        info.cycles += 1
        x = x + V[:j_end].T @ d
        res = _norm(rho)
        info.history.append(res / nb)
        stalled = stalled + 1 if res >= best * (1.0 - 1e-3) else 0
        best = min(best, res)
        done = conv or info.cycles >= max_cycles or stalled >= stall or j_end < m and not conv
        kk = min(k, j_end - 1)
        if kk >= 1:
            Vk1, Hk, cn = dr_restart(V, H, j_end, kk, rho)
            defl = Deflation(Vk1, Hk)
        else:
            defl = Deflation(V[: j_end + 1].copy(), H[: j_end + 1, :j_end].copy())
        if done:
            info.converged = conv
            info.relres = res / nb
            return x, info, defl
        V[:] = 0.0
        H[:] = 0.0
        c[:] = 0.0
        V[: kk + 1] = Vk1
        H[: kk + 1, :kk] = Hk
        c[: kk + 1] = cn
        j0 = kk


def gmres_proj(A, b, defl, m, tol, max_cycles=1000):
    """GMRES-Proj(m,k) from x = 0 with deflation space defl = (W = V_{k+1}, H_k):
    repeat { d = argmin ||W^+ r - H_k d||; x += V_k d; r -= W H_k d;
             one GMRES(m - k) cycle from r } until ||r|| <= tol ||b||."""
    n = b.shape[0]
    nb = _norm(b)
    info = SolveInfo()
    x = np.zeros(n, dtype=np.complex128)
    r = b.copy()
    W, Hk, k = defl.W, defl.Hk, defl.k
    ms = max(m - k, 1)
    while True:
        d, _ = lsq(Hk, W.conj() @ r)
        x = x + W[:k].T @ d
        r = r - W.T @ (Hk @ d)
        res = _norm(r)
        if res <= tol * nb:
            info.converged, info.relres = True, res / nb
            return x, info
        V = np.zeros((ms + 1, n), dtype=np.complex128)
        H = np.zeros((ms + 1, ms), dtype=np.complex128)
        c = np.zeros(ms + 1, dtype=np.complex128)
        c[0] = res
        V[0] = r / res
        j_end, dd, rho, conv = arnoldi_run(A, V, H, 0, ms, c, tol * nb)
        info.iters += j_end
        info.cycles += 1
        x = x + V[:j_end].T @ dd
        r = V[: j_end + 1].T @ rho
        info.history.append(_norm(rho) / nb)
        if conv or info.cycles >= max_cycles:
            info.converged, info.relres = conv, _norm(rho) / nb
            return x, info


def cgne(A, Ad, b, tol, max_iters=100000):
    """CG on A A^+ y = b (Hermitian positive definite), x = A^+ y; stops on the
    recursive residual ||b - A A^+ y|| <= tol ||b||."""
    nb = _norm(b)
    info = SolveInfo()
    y = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = np.vdot(r, r).real
    while np.sqrt(rr) > tol * nb and info.iters < max_iters:
        q = A(Ad(p))
        alpha = rr / np.vdot(p, q).real
        y = y + alpha * p
        r = r - alpha * q
        rr_new = np.vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
        info.iters += 1
    info.converged = np.sqrt(rr) <= tol * nb
    info.relres = np.sqrt(rr) / nb
    return Ad(y), info
