"""GPU parity of the whole solve (Section 2) against the FP64 oracle, through the C ABI.

* FP64 path, identical prolongators (mg_setup_from_vectors with the oracle's
  near-null vectors): the same algorithm step by step, so the solutions agree to
  <= 1e-10 relative and the outer iteration counts to within one;
* every solve meets its tolerance on the true residual recomputed here with the
  oracle's operator; against a sparse direct solve the error is <= kappa * tol;
* mixed precision (FP32 V-cycle, FP64 outer): true residual <= 1e-8, and, run to
  tol = 1e-7 / kappa, solution error <= 1e-7;
* the deflation space exported by the GPU satisfies A W_k = W H_k and spans the
  oracle's space; the CGNE arm; host buffers (the end-to-end path); edge cases.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import dirac, hierarchy, mg as omg
from gpu_util import dev, host, rel2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mgmod(cuda_lib):
    import paper_1912_02868_gb300 as mg
    return mg


def _hier(L, cfg=0):
    U = synth.gauge_field(L, cfg)
    m0 = synth.m0_for(L, cfg)
    h = hierarchy.build(U, m0, synth.nullvec_starts(L, cfg, 0, 12, L * L * 2),
                        synth.nullvec_starts(L, cfg, 1, 12, (L // 4) ** 2 * 24))
    return U, m0, h


@pytest.fixture(scope="module", params=[16, 32, 64])
def case(request, mgmod):
    L = request.param
    U, m0, h = _hier(L)
    A = dirac.stencil_sparse(dirac.wilson_stencil(U, m0)).tocsc()
    lu = spla.splu(A)
    return L, U, m0, h, A, lu


def _true_relres(U, m0, x, b):
    return np.linalg.norm(dirac.wilson(U, x.reshape(b.shape), m0) - b) / np.linalg.norm(b)


def _kappa_bound(A, lu):
    # ||A^{-1}|| by a few steps of power iteration on A^{-H} A^{-1}
    v = synth.complex_gaussian((A.shape[0],), 99)
    for _ in range(30):
        v = lu.solve(lu.solve(v), trans="H")
        v /= np.linalg.norm(v)
    inv_norm = np.sqrt(np.linalg.norm(lu.solve(lu.solve(v), trans="H")))
    return 4.0 * inv_norm  # ||A|| <= 4 for |U| = 1 and |m0| small


def test_fp64_solve_parity_with_oracle(mgmod, case):
    L, U, m0, h, A, lu = case
    tol = 1e-10
    b = synth.rhs(L, 0, 0)[0]
    osol = omg.MGSolver(h)
    xo, info_o = osol.solve(b, tol)
    g = mgmod.mg_setup_from_vectors(dev(U), L, L, m0, dev(h.nullvecs[0]), dev(h.nullvecs[1]))
    try:
        import torch
        x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
        st, iters, relres, stats = mgmod.mg_solve(g, dev(b), x, 1, tol)
        xg = host(x)
    finally:
        g.close()
    assert relres[0] <= tol
    assert _true_relres(U, m0, xg, b) <= tol * 1.0001
    assert abs(iters[0] - info_o.iters) <= 1
    assert rel2(xg, xo) <= 1e-10
    xs = lu.solve(b.ravel())
    assert rel2(xg, xs) <= _kappa_bound(A, lu) * tol
    assert stats["dr_solves"] == 1 and stats["coarse_solves"] == iters[0]


def test_deflation_space_parity(mgmod, case):
    L, U, m0, h, A, lu = case
    b = synth.rhs(L, 0, 0)[0]
    osol = omg.MGSolver(h)
    osol.solve(b, 1e-8)
    g = mgmod.mg_setup_from_vectors(dev(U), L, L, m0, dev(h.nullvecs[0]), dev(h.nullvecs[1]))
    try:
        import torch
        x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
        mgmod.mg_solve(g, dev(b), x, 1, 1e-8)
        W, Hk = mgmod.mg_get_deflation(g)
    finally:
        g.close()
    Wo = osol.deflation.W
    k = Hk.shape[1]
    assert k == osol.deflation.k
    A2 = dirac.dense_from_apply(lambda v: dirac.stencil_apply(h.A2, v), h.shapes[2])
    Wc = W.T
    assert np.abs(Wc.conj().T @ Wc - np.eye(k + 1)).max() < 1e-12
    assert np.linalg.norm(A2 @ Wc[:, :k] - Wc @ Hk) <= 1e-10 * np.linalg.norm(A2, 2)
    # Ritz values of the space (unique even when the kept set is not): the k of
    # smallest modulus, compared as moduli because sigma3^-hermiticity makes the
    # spectrum closed under conjugation, so |theta| ties come in exact pairs
    rg = np.sort(np.abs(np.linalg.eigvals(Hk[:k, :k])))
    ro = np.sort(np.abs(np.linalg.eigvals(osol.deflation.Hk[:k, :k])))
    assert np.allclose(rg, ro, rtol=1e-6)
    # the same subspace as the oracle's (projectors) when the kept set is unique
    # (n_coarse > m: the solve restarts and the space is not an exact eigenspace
    # split inside a conjugate pair).  The GMRES-DR solve runs many restarts before
    # it stalls near 1e-14; rounding differences between the two implementations
    # move the not-yet-converged part of the space at the 1e-7 level.
    if A2.shape[0] > 30:
        Po = Wo.T @ Wo.conj()
        Pg = Wc @ Wc.conj().T
        assert np.abs(Po - Pg).max() < 1e-6


def test_second_rhs_reuses_deflation_and_multi_rhs(mgmod, case):
    L, U, m0, h, A, lu = case
    import torch
    g = mgmod.mg_setup_from_vectors(dev(U), L, L, m0, dev(h.nullvecs[0]), dev(h.nullvecs[1]))
    try:
        B = synth.rhs(L, 0, 0, nrhs=3)
        X = torch.zeros(B.shape, dtype=torch.complex128, device="cuda")
        st, iters, relres, stats = mgmod.mg_solve(g, dev(B), X, 3, 1e-8)
        assert stats["dr_solves"] == 1
        Xh = host(X)
        for i in range(3):
            assert relres[i] <= 1e-8
            assert _true_relres(U, m0, Xh[i], B[i]) <= 1.0001e-8
        # solving the second right-hand side alone, after the deflation space exists, gives the same x
        X1 = torch.zeros(B[1].shape, dtype=torch.complex128, device="cuda")
        st, it1, rr1, st1 = mgmod.mg_solve(g, dev(B[1]), X1, 1, 1e-8)
        assert st1["dr_solves"] == 0
        assert rel2(host(X1), Xh[1]) <= 1e-12
    finally:
        g.close()


def test_mixed_precision_solve(mgmod, case):
    L, U, m0, h, A, lu = case
    import torch
    p = mgmod.default_params(precision=mgmod.MG_MIXED)
    g = mgmod.mg_setup_from_vectors(dev(U), L, L, m0, dev(h.nullvecs[0]), dev(h.nullvecs[1]), params=p)
    try:
        b = synth.rhs(L, 0, 0)[0]
        x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
        st, iters, relres, stats = mgmod.mg_solve(g, dev(b), x, 1, 1e-8)
        assert relres[0] <= 1e-8
        assert _true_relres(U, m0, host(x), b) <= 1.0001e-8
        kappa = _kappa_bound(A, lu)
        tol = 1e-7 / kappa
        st, iters, relres, stats = mgmod.mg_solve(g, dev(b), x, 1, tol)
        xs = lu.solve(b.ravel())
        assert rel2(host(x), xs) <= 1e-7
    finally:
        g.close()


def test_cgne_arm(mgmod):
    import torch
    L = 32
    U, m0, h = _hier(L)
    p = mgmod.default_params(coarse_solver=mgmod.MG_COARSE_CGNE)
    g = mgmod.mg_setup_from_vectors(dev(U), L, L, m0, dev(h.nullvecs[0]), dev(h.nullvecs[1]), params=p)
    try:
        b = synth.rhs(L, 0, 0)[0]
        x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
        st, iters, relres, stats = mgmod.mg_solve(g, dev(b), x, 1, 1e-8)
        assert relres[0] <= 1e-8 and stats["dr_solves"] == 0
        assert _true_relres(U, m0, host(x), b) <= 1.0001e-8
        xo, info = omg.MGSolver(h, omg.Params(coarse="cgne")).solve(b, 1e-8)
        assert abs(iters[0] - info.iters) <= 1
    finally:
        g.close()


@pytest.mark.parametrize("L", [16, 32])
def test_fine_deflation_arm(mgmod, L):
    """Comparison arm without multigrid: GMRES-DR(30,10) on the fine operator for
    the first right-hand side, GMRES-Proj(30,10) for the next (Section 2), FP64,
    against the oracle's gmres_dr / gmres_proj on the same operator."""
    import torch
    from oracle import krylov
    U = synth.gauge_field(L, 0)
    m0 = synth.m0_for(L, 0)
    p = mgmod.default_params(method=mgmod.MG_METHOD_FINE_DEFLATION)
    g = mgmod.mg_setup(dev(U), L, L, m0, params=p)
    A = lambda v: dirac.wilson(U, v.reshape(L, L, 2), m0).ravel()
    try:
        b0, b1 = synth.rhs(L, 0, 0, nrhs=2)
        x = torch.zeros(b0.shape, dtype=torch.complex128, device="cuda")
        st, it0, rr0, s0 = mgmod.mg_solve(g, dev(b0), x, 1, 1e-8)
        xg0 = host(x)
        xo0, info0, defl = krylov.gmres_dr(A, b0.ravel(), 30, 10, 1e-8)
        assert s0["dr_solves"] == 1 and rr0[0] <= 1e-8
        assert _true_relres(U, m0, xg0, b0) <= 1.0001e-8
        assert abs(it0[0] - info0.iters) <= 2
        assert rel2(xg0, xo0) <= 1e-6
        st, it1, rr1, s1 = mgmod.mg_solve(g, dev(b1), x, 1, 1e-8)
        xo1, info1 = krylov.gmres_proj(A, b1.ravel(), defl, 30, 1e-8)
        assert s1["dr_solves"] == 0 and rr1[0] <= 1e-8
        assert _true_relres(U, m0, host(x), b1) <= 1.0001e-8
        assert abs(it1[0] - info1.iters) <= 2
    finally:
        g.close()


def test_host_buffers_end_to_end_and_edge_cases(mgmod):
    import torch
    L = 16
    U, m0, h = _hier(L)
    g = mgmod.mg_setup(U, L, L, m0, starts0=synth.nullvec_starts(L, 0, 0, 12, L * L * 2),
                       starts1=synth.nullvec_starts(L, 0, 1, 12, (L // 4) ** 2 * 24))
    try:
        b = synth.rhs(L, 0, 0, nrhs=2)
        x = np.zeros_like(b)
        st, iters, relres, stats = mgmod.mg_solve(g, b, x, 2, 1e-9)  # numpy (pageable host) buffers
        for i in range(2):
            assert _true_relres(U, m0, x[i], b[i]) <= 1.0001e-9
        bp = torch.from_numpy(b).pin_memory()
        xp = torch.zeros_like(bp).pin_memory()
        mgmod.mg_solve(g, bp, xp, 2, 1e-9)
        assert rel2(xp.numpy(), x) <= 1e-12
        # zero right-hand side: x = 0, relres 0, no iterations
        z = np.zeros((L, L, 2), dtype=np.complex128)
        xz = np.ones_like(z)
        st, iters, relres, _ = mgmod.mg_solve(g, z, xz, 1, 1e-9)
        assert iters[0] == 0 and relres[0] == 0.0 and not xz.any()
        # nrhs = 0 is a no-op
        mgmod.mg_solve(g, z, xz, 0, 1e-9)
        # an iteration limit that cannot be met reports MG_ENOTCONV
        g2 = mgmod.mg_setup(U, L, L, m0, params=mgmod.default_params(max_outer=1))
        try:
            st, iters, relres, _ = mgmod.mg_solve(g2, b[0].copy(), np.zeros_like(b[0]), 1, 1e-12, allow_notconv=True)
            assert st == mgmod.MG_ENOTCONV and iters[0] == 1 and relres[0] > 1e-12
        finally:
            g2.close()
    finally:
        g.close()


def test_bench_size_solve_meets_tolerance(mgmod):
    """256^2 (the bench lattice): the GPU set-up and solve, FP64 and mixed, checked
    by the true residual recomputed with the oracle's operator."""
    import torch
    L = 256
    U = synth.gauge_field(L, 0)
    m0 = synth.m0_for(L, 0)
    for prec in (mgmod.MG_FP64, mgmod.MG_MIXED):
        g = mgmod.mg_setup(dev(U), L, L, m0, params=mgmod.default_params(precision=prec),
                           starts0=dev(synth.nullvec_starts(L, 0, 0, 12, L * L * 2)),
                           starts1=dev(synth.nullvec_starts(L, 0, 1, 12, (L // 4) ** 2 * 24)))
        try:
            B = synth.rhs(L, 0, 0, nrhs=2)
            X = torch.zeros(B.shape, dtype=torch.complex128, device="cuda")
            st, iters, relres, stats = mgmod.mg_solve(g, dev(B), X, 2, 1e-8)
            Xh = host(X)
            for i in range(2):
                assert relres[i] <= 1e-8
                assert _true_relres(U, m0, Xh[i], B[i]) <= 1.0001e-8
        finally:
            g.close()


@pytest.mark.parametrize("L", [16, 32])
def test_fine_cgne_method(mgmod, L):
    """The plain comparison method without multigrid: CGNE on the fine operator
    (CG on D D^+ y = b, x = D^+ y), FP64, against the oracle's cgne: the same
    iteration count within 1%, the true residual at the tolerance, and the
    fine-operator count of Eq. 1 (two applies per step, one for x, one for the
    residual check)."""
    import torch
    from oracle import krylov
    U = synth.gauge_field(L, 0)
    m0 = synth.m0_for(L, 0)
    p = mgmod.default_params(method=mgmod.MG_METHOD_FINE_CGNE, precision=mgmod.MG_FP64)
    g = mgmod.mg_setup(dev(U), L, L, m0, params=p)
    A = lambda v: dirac.wilson(U, v.reshape(L, L, 2), m0).ravel()
    Ad = lambda v: dirac.wilson_dagger(U, v.reshape(L, L, 2), m0).ravel()
    try:
        b = synth.rhs(L, 0, 3)[0]
        x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
        # CG stops on its recursive residual, so the true one may sit a rounding above
        st, it, rr, stats = mgmod.mg_solve(g, dev(b), x, 1, 1e-8, allow_notconv=True)
        xo, info = krylov.cgne(A, Ad, b.ravel(), 1e-8)
        assert info.converged and rr[0] <= 1.05e-8
        assert _true_relres(U, m0, host(x), b) <= 1.05e-8
        assert abs(it[0] - info.iters) <= max(2, 0.01 * info.iters), (it[0], info.iters)
        assert stats["mvps"][0] == 2 * it[0] + 2 and stats["mvps"][1] == 0 and stats["mvps"][2] == 0
        assert rel2(host(x).ravel(), xo) <= 1e-5
    finally:
        g.close()


def test_nondeflated_partial_solve(mgmod):
    """Non-deflated MG with the partial intermediate solve: CGNE on the coarsest
    grid to 1e-8 in every outer iteration (Section 2: relaxing it like the
    deflated solve costs outer iterations), against the oracle with the same
    near-null vectors: outer counts within 1, the true residual at 1e-8, and
    every coarse solve a CGNE solve."""
    import torch
    L = 32
    U, m0, h = _hier(L)
    p = mgmod.default_params(coarse_solver=mgmod.MG_COARSE_CGNE, partial_tol=0.2)
    g = mgmod.mg_setup_from_vectors(dev(U), L, L, m0, dev(h.nullvecs[0]), dev(h.nullvecs[1]), params=p)
    try:
        b = synth.rhs(L, 0, 0)[0]
        x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
        st, iters, relres, stats = mgmod.mg_solve(g, dev(b), x, 1, 1e-8)
        assert relres[0] <= 1e-8 and stats["dr_solves"] == 0
        assert _true_relres(U, m0, host(x), b) <= 1.0001e-8
        solver = omg.MGSolver(h, omg.Params(coarse="cgne", partial_tol=0.2))
        xo, info = solver.solve(b, 1e-8)
        assert abs(iters[0] - info.iters) <= 1, (iters[0], info.iters)
        assert all(kind == "cgne" for kind, _ in solver.coarse_solves)
        assert all(t == 1e-8 for t in solver.coarse_tols)
    finally:
        g.close()
