"""GPU parity of the lockstep block solve (precision MG_MIXED_BF16 / MG_MIXED_FP16)
through the C ABI.

* Tensor-core block stencil (mg_apply_block): for blocks of 8..64 right-hand
  sides, against the oracle's stencil with the operator rounded once from FP64
  to BF16 / FP16 (each part round-to-nearest) and exact products: the FP32
  vectors enter as a high and a low 16-bit part, so the difference is the
  rounding of the vector's low part (<= 2^-18 relative for BF16, smaller for
  FP16) plus FP32 accumulation over 120 complex terms: max-norm <= 3e-5 (BF16)
  and 1e-5 (FP16) relative to the output's max.
* Batched coarse GMRES-Proj (mg_coarse_solve with MG_BF16 / MG_F16): each
  right-hand side against the oracle's GMRES-Proj (FP64) on the same rounded
  operator and the oracle's deflation space: Krylov step counts within 2%, the
  solutions within 1e-4 (the same algorithm in FP32 against FP64: measured
  1e-6 to 2e-5), and the true residual with the rounded operator no worse than
  the oracle's own (the projection step uses the deflation relation of the
  exact operator, so both level off near the operator's rounding, 1e-3 for
  FP16 and 1e-2 for BF16); a ragged block (not a multiple of 8).
* Whole block solve (mg_solve): every right-hand side meets the true FP64
  residual 1e-8 recomputed with the oracle's operator; outer counts close to
  the FP32 path's; run to 1e-7 / kappa, the solution is within 1e-7 of a sparse
  direct solve; a ragged block, host buffers, and a zero right-hand side.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import dirac, krylov
import oracle_cache as oc
from gpu_util import dev, host, rel, rel2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mgmod(cuda_lib):
    import paper_1912_02868_gb300 as mg
    return mg


def bf16(a):
    """a real FP64 array rounded once to BF16 (8 significant bits, round to nearest
    even on the FP64 significand), returned as FP64"""
    u = np.ascontiguousarray(a, dtype=np.float64).view(np.uint64).copy()
    u += np.uint64(0x00000FFFFFFFFFFF) + ((u >> np.uint64(45)) & np.uint64(1))
    u &= np.uint64(0xFFFFE00000000000)
    return u.view(np.float64)


def round16(A, fp16):
    if fp16:
        return oc.fp16(A)
    return bf16(A.real) + 1j * bf16(A.imag)


def _handle(mgmod, L, prec=None, defl=True):
    U, m0, h = oc.hier(L)
    p = mgmod.default_params(precision=prec if prec is not None else mgmod.MG_MIXED_BF16)
    g = mgmod.mg_setup_from_vectors(dev(U), L, L, m0, dev(h.nullvecs[0]), dev(h.nullvecs[1]), params=p)
    if defl:
        d = oc.coarse_deflation(L)
        mgmod.mg_set_deflation(g, d.W, d.Hk)
    return g, U, m0, h


@pytest.mark.parametrize("L,level,nrhs,fp16", [(64, 1, 8, False), (64, 2, 16, True), (256, 1, 64, False),
                                               (256, 2, 24, False), (256, 1, 16, True)])
def test_block_stencil_parity(mgmod, L, level, nrhs, fp16):
    import torch
    g, U, m0, h = _handle(mgmod, L, defl=False)
    try:
        A = h.A1 if level == 1 else h.A2
        shape = h.shapes[level]
        X = np.stack([synth.complex_gaussian(shape, 9100 + level, r) for r in range(nrhs)]).astype(np.complex64)
        Y = torch.zeros(X.shape, dtype=torch.complex64, device="cuda")
        mgmod.mg_apply_block(g, level, dev(X), Y, nrhs, mgmod.MG_F16 if fp16 else mgmod.MG_BF16)
        Yg = host(Y)
        Ar = round16(A, fp16)
        for r in range(nrhs):
            ref = dirac.stencil_apply(Ar, X[r].astype(np.complex128))
            assert rel(Yg[r], ref) <= (1e-5 if fp16 else 3e-5), r
    finally:
        g.close()


def _coarse_relres(A, x, b, shape):
    return np.linalg.norm(dirac.stencil_apply(A, x.reshape(shape)).ravel() - b) / np.linalg.norm(b)


def _kappa(A2):
    M = dirac.stencil_sparse(A2).tocsc()
    lu = spla.splu(M)
    v = synth.complex_gaussian((M.shape[0],), 99)
    for _ in range(30):
        v = lu.solve(lu.solve(v), trans="H")
        v /= np.linalg.norm(v)
    inv = np.sqrt(np.linalg.norm(lu.solve(lu.solve(v), trans="H")))
    u = synth.complex_gaussian((M.shape[0],), 98)
    for _ in range(30):
        u = M.conj().T @ (M @ u)
        u /= np.linalg.norm(u)
    return np.sqrt(np.linalg.norm(M.conj().T @ (M @ u))) * inv


@pytest.mark.parametrize("L,nrhs,fp16", [(64, 16, False), (256, 9, False), (256, 8, True)])
def test_block_coarse_solve_parity(mgmod, L, nrhs, fp16):
    import torch
    g, U, m0, h = _handle(mgmod, L)
    try:
        n2 = h.size(2)
        tol = 1e-5
        Bc = np.stack([synth.complex_gaussian((n2,), 9200 + L, r) for r in range(nrhs)])
        X = torch.zeros((nrhs, n2), dtype=torch.complex64, device="cuda")
        st, it, conv, info = mgmod.mg_coarse_solve(g, dev(Bc, torch.complex64), X, tol,
                                                   mgmod.MG_F16 if fp16 else mgmod.MG_BF16, nrhs=nrhs)
        Xg = host(X).astype(np.complex128)
        Ar = round16(h.A2, fp16)
        defl = oc.coarse_deflation(L)
        for r in range(nrhs):
            xo, io = krylov.gmres_proj(oc.coarse_op(h, Ar), Bc[r], defl, 30, tol)
            assert conv[r] and io.converged
            assert abs(it[r] - io.iters) <= max(2, 0.02 * io.iters), (r, it[r], io.iters)
            assert rel2(Xg[r], xo) <= 1e-4
            res_g = _coarse_relres(Ar, Xg[r], Bc[r], h.shapes[2])
            res_o = _coarse_relres(Ar, xo, Bc[r], h.shapes[2])
            assert res_g <= 1.5 * res_o + tol, (res_g, res_o)
    finally:
        g.close()


def _true_relres(U, m0, x, b):
    return np.linalg.norm(dirac.wilson(U, x.reshape(b.shape), m0) - b) / np.linalg.norm(b)


@pytest.mark.parametrize("L,nrhs,prec", [(64, 16, "bf16"), (64, 11, "fp16"), (256, 24, "bf16")])
def test_block_solve_meets_tolerance(mgmod, L, nrhs, prec):
    import torch
    p = mgmod.MG_MIXED_BF16 if prec == "bf16" else mgmod.MG_MIXED_FP16
    g, U, m0, h = _handle(mgmod, L, prec=p, defl=False)
    gm, _, _, _ = _handle(mgmod, L, prec=mgmod.MG_MIXED, defl=False)
    try:
        B = synth.rhs(L, 0, 0, nrhs=nrhs)
        X = torch.zeros(B.shape, dtype=torch.complex128, device="cuda")
        st, iters, relres, stats = mgmod.mg_solve(g, dev(B), X, nrhs, 1e-8)
        Xh = host(X)
        assert stats["dr_solves"] == 1  # right-hand side 0 builds the deflation space alone
        for i in range(nrhs):
            assert relres[i] <= 1e-8
            assert _true_relres(U, m0, Xh[i], B[i]) <= 1.0001e-8, i
        # the FP32 path (FP16-stored coarse operator, no tensor cores) on the same system
        Xm = torch.zeros(B.shape, dtype=torch.complex128, device="cuda")
        _, iters_m, _, _ = mgmod.mg_solve(gm, dev(B), Xm, nrhs, 1e-8)
        assert abs(np.mean(iters) - np.mean(iters_m)) <= 0.1 * np.mean(iters_m) + 1, (iters, iters_m)
        assert max(abs(a - b) for a, b in zip(iters, iters_m)) <= 3, (iters, iters_m)
    finally:
        g.close()
        gm.close()


def test_block_solve_accuracy_and_edge_cases(mgmod):
    import torch
    L = 64
    g, U, m0, h = _handle(mgmod, L, prec=mgmod.MG_MIXED_BF16, defl=False)
    try:
        A = dirac.stencil_sparse(dirac.wilson_stencil(U, m0)).tocsc()
        lu = spla.splu(A)
        v = synth.complex_gaussian((A.shape[0],), 99)
        for _ in range(30):
            v = lu.solve(lu.solve(v), trans="H")
            v /= np.linalg.norm(v)
        kappa = 4.0 * np.sqrt(np.linalg.norm(lu.solve(lu.solve(v), trans="H")))
        B = synth.rhs(L, 0, 0, nrhs=9)
        B[4] = 0.0  # a zero right-hand side inside the block
        X = np.zeros_like(B)  # host (pageable) buffers
        st, iters, relres, _ = mgmod.mg_solve(g, B, X, 9, 1e-7 / kappa)
        assert iters[4] == 0 and relres[4] == 0.0 and not X[4].any()
        for i in (0, 1, 5, 8):
            xs = lu.solve(B[i].ravel())
            assert rel2(X[i], xs) <= 1e-7, i
        # a limit that cannot be met is reported per right-hand side
        g2 = mgmod.mg_setup(dev(U), L, L, m0, params=mgmod.default_params(precision=mgmod.MG_MIXED_BF16, max_outer=8))
        try:
            Bt = torch.from_numpy(B[:3].copy()).cuda()
            Xt = torch.zeros_like(Bt)
            st, iters, relres, _ = mgmod.mg_solve(g2, Bt, Xt, 3, 1e-12, allow_notconv=True)
            assert st == mgmod.MG_ENOTCONV and all(rr > 1e-12 for rr in relres)
        finally:
            g2.close()
    finally:
        g.close()


def test_block_coarse_probe_times_out_and_handle_stays_usable(mgmod):
    """A tile-barrier wait of the batched cycle kernel that gives up (the probe: a
    word nothing writes) makes the coarse solve return MG_ETIMEOUT; the barrier
    state is reset, so the next solve is bitwise the one before the probe, and a
    whole block solve on the same handle still meets its tolerance."""
    import torch
    L, nrhs = 256, 16
    g, U, m0, h = _handle(mgmod, L)
    try:
        n2 = h.size(2)
        Bc = dev(np.stack([synth.complex_gaussian((n2,), 9300, r) for r in range(nrhs)]), torch.complex64)
        X0 = torch.zeros((nrhs, n2), dtype=torch.complex64, device="cuda")
        st0, it0, conv0, _ = mgmod.mg_coarse_solve(g, Bc, X0, 1e-5, mgmod.MG_BF16, nrhs=nrhs)
        assert st0 == mgmod.MG_OK and all(conv0)
        Xp = torch.zeros_like(X0)
        st, _, _, info = mgmod.mg_coarse_solve(g, Bc, Xp, 1e-5, mgmod.MG_BF16, nrhs=nrhs,
                                               flags=mgmod.MG_COARSE_PROBE_TIMEOUT, spin=64,
                                               allow=(mgmod.MG_ETIMEOUT,))
        assert st == mgmod.MG_ETIMEOUT and info["timeouts"] == 1
        X1 = torch.zeros_like(X0)
        st1, it1, _, info1 = mgmod.mg_coarse_solve(g, Bc, X1, 1e-5, mgmod.MG_BF16, nrhs=nrhs)
        assert st1 == mgmod.MG_OK and info1["timeouts"] == 0 and it1 == it0
        assert torch.equal(X0, X1)
        B = synth.rhs(L, 0, 40, nrhs=8)
        X = torch.zeros(B.shape, dtype=torch.complex128, device="cuda")
        _, iters, relres, _ = mgmod.mg_solve(g, dev(B), X, 8, 1e-8)
        Xh = host(X)
        for i in range(8):
            assert relres[i] <= 1e-8 and _true_relres(U, m0, Xh[i], B[i]) <= 1.0001e-8
    finally:
        g.close()
