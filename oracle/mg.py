"""Oracle: the three-grid V-cycle and the deflated MG-FGMRES solve (FP64).

Test infrastructure only (see ``oracle/__init__.py``).

Section 2: FGMRES(8) is the outer solver; the preconditioner is a multigrid
cycle with two iterations of GMRES as pre- and post-smoother on the fine and
intermediate grids; the coarsest grid is solved with GMRES-DR(m,k) at the first
outer iteration (which also yields the deflation space) and with
GMRES-Proj(m,k) at every later outer iteration and for every later right-hand
side (the space is kept).  The comparison arm solves the coarsest grid with
CGNE at every outer iteration.  Section 3, Eq. 1, counts the cost in fine
equivalent matrix-vector products:
    Mvps = fine + (n_int / n_fine) int + (n_coarse / n_fine) coarse.

V-cycle on level l with right-hand side f (reading of Section 2):
    x = S(f)                      GMRES(2) from 0; r from the Arnoldi relation
    x += P (cycle or solve on level l+1 with P^+ r)
    r = f - A x                   (one operator application)
    x += S(r)

Partial intermediate solve (Section 2, the variant with a partial solve on the
intermediate grid).  The cycle on the intermediate grid is replaced by a solve
of the intermediate system to relative residual 0.2.  Readings (the solver is
not named in the paper):
  * the solve is FGMRES(m) on the intermediate operator, with the same m as the
    outer solver, preconditioned by the two-grid cycle above (smoothing on the
    intermediate grid, coarse solve, smoothing);
  * coarse solves inside the first outer iteration of a right-hand side go to
    1e-8 (the first one of all by GMRES-DR, which builds the deflation space);
    every later coarse solve is a projected solve to 1e-2.
"""
from __future__ import annotations

import numpy as np

from . import krylov


class Params:
    def __init__(self, fgmres_m=8, smooth_steps=2, coarse="dr_proj", dr_m=30, dr_k=10,
                 coarse_tol_first=1e-14, coarse_tol_rest=1e-8, dr_max_cycles=100, max_outer=500,
                 proj_max_cycles=1000, partial_tol=None, coarse_tol_partial=1e-2, partial_max_iters=200):
        self.fgmres_m = fgmres_m
        self.smooth_steps = smooth_steps
        self.coarse = coarse  # "dr_proj" | "cgne"
        self.dr_m, self.dr_k = dr_m, dr_k
        self.coarse_tol_first = coarse_tol_first
        self.coarse_tol_rest = coarse_tol_rest
        self.dr_max_cycles = dr_max_cycles
        self.max_outer = max_outer
        self.proj_max_cycles = proj_max_cycles
        self.partial_tol = partial_tol  # None: V-cycle; else the intermediate partial solve's tolerance
        self.coarse_tol_partial = coarse_tol_partial
        self.partial_max_iters = partial_max_iters


class MGSolver:
    """Deflated MG-FGMRES on an oracle Hierarchy.  The coarse deflation space
    is built by the first coarse solve and then kept for all later solves."""

    def __init__(self, hier, params=None):
        self.h = hier
        self.p = params or Params()
        self.counter = krylov.Counter(3)
        self.deflation = None
        self.coarse_solves = []  # (kind, iters) per coarse solve
        self.coarse_tols = []    # tolerance of each coarse solve
        self.partial_solves = []  # (iters, relres) per intermediate partial solve
        self._precond_calls = 0  # preconditioner applications in the current solve

    def _op(self, level):
        shape = self.h.shapes[level]
        f = lambda v: self.h.apply(level, v.reshape(shape)).ravel()
        return self.counter.wrap(level, f)

    def _op_dag(self, level):
        shape = self.h.shapes[level]
        f = lambda v: self.h.apply_dagger(level, v.reshape(shape)).ravel()
        return self.counter.wrap(level, f)

    def coarse_solve(self, f):
        p = self.p
        A2 = self._op(2)
        if p.coarse == "cgne":
            x, info = krylov.cgne(A2, self._op_dag(2), f, p.coarse_tol_rest)
            self.coarse_solves.append(("cgne", info.iters))
            self.coarse_tols.append(p.coarse_tol_rest)
            return x
        if p.partial_tol is None:
            tol_dr, tol_proj = p.coarse_tol_first, p.coarse_tol_rest
        else:  # first outer iteration of this right-hand side: 1e-8, later 1e-2
            tol_dr = p.coarse_tol_rest
            tol_proj = p.coarse_tol_rest if self._precond_calls <= 1 else p.coarse_tol_partial
        if self.deflation is None:
            x, info, defl = krylov.gmres_dr(A2, f, p.dr_m, p.dr_k, tol_dr, p.dr_max_cycles)
            self.deflation = defl
            self.coarse_solves.append(("dr", info.iters))
            self.coarse_tols.append(tol_dr)
            return x
        x, info = krylov.gmres_proj(A2, f, self.deflation, p.dr_m, tol_proj, p.proj_max_cycles)
        self.coarse_solves.append(("proj", info.iters))
        self.coarse_tols.append(tol_proj)
        return x

    def twogrid(self, f):
        """The cycle on the intermediate grid: smoothing there, coarse solve, smoothing."""
        A = self._op(1)
        shape = self.h.shapes[1]
        x, r = krylov.smoother(A, f, self.p.smooth_steps)
        ec = self.coarse_solve(self.h.restrict(1, r.reshape(shape)).ravel())
        x = x + self.h.prolong(1, ec.reshape(self.h.shapes[2])).ravel()
        r = f - A(x)
        e, _ = krylov.smoother(A, r, self.p.smooth_steps)
        return x + e

    def partial_solve(self, f):
        """Intermediate system solved to ||f - A x|| <= partial_tol ||f|| by FGMRES
        preconditioned with the two-grid cycle."""
        x, info = krylov.fgmres(self._op(1), f, self.twogrid, self.p.partial_tol, m=self.p.fgmres_m,
                                max_iters=self.p.partial_max_iters)
        self.partial_solves.append((info.iters, info.relres))
        return x

    def vcycle(self, level, f):
        if level == 2:
            return self.coarse_solve(f)
        if level == 1 and self.p.partial_tol is not None:
            return self.partial_solve(f)
        A = self._op(level)
        shape = self.h.shapes[level]
        x, r = krylov.smoother(A, f, self.p.smooth_steps)
        rc = self.h.restrict(level, r.reshape(shape)).ravel()
        ec = self.vcycle(level + 1, rc)
        x = x + self.h.prolong(level, ec.reshape(self.h.shapes[level + 1])).ravel()
        r = f - A(x)
        e, _ = krylov.smoother(A, r, self.p.smooth_steps)
        return x + e

    def solve(self, b, tol):
        """Solve D x = b (b complex[L_t][L_x][2]) to true relative residual tol."""
        shape = self.h.shapes[0]
        bf = np.asarray(b, dtype=np.complex128).ravel()
        self._precond_calls = 0

        def precond(v):
            self._precond_calls += 1
            return self.vcycle(0, v)

        x, info = krylov.fgmres(self._op(0), bf, precond, tol, m=self.p.fgmres_m, max_iters=self.p.max_outer)
        return x.reshape(shape), info

    def fine_equivalent_mvps(self):
        n = [self.h.size(l) for l in range(3)]
        m = self.counter.mvps
        return m[0] + n[1] / n[0] * m[1] + n[2] / n[0] * m[2]
