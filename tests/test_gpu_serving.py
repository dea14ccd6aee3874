"""GPU tests of the batching and serving layers (through the C ABI).

* mg_solve with nrhs > 1 and parallel > 1 runs right-hand sides concurrently on
  solve contexts that share the hierarchy; every result equals the sequential
  solve of the same right-hand side (same deflation space, deterministic
  kernels) and meets the tolerance on the true residual;
* the server: each request's result is the same alone and in a mix of
  concurrent requests over several operators and lattice sizes, and meets the
  tolerance; an HBM budget that holds one hierarchy forces evictions without
  changing results.
"""
import numpy as np
import pytest

import synth
from oracle import dirac
from gpu_util import dev, host, rel2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mgmod(cuda_lib):
    import paper_1912_02868_gb300 as mg
    return mg


def _true_relres(U, m0, x, b):
    return np.linalg.norm(dirac.wilson(U, x.reshape(b.shape), m0) - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_parallel_multi_rhs_equals_sequential(mgmod, prec):
    import torch
    L = 64
    U = synth.gauge_field(L, 1)
    m0 = synth.m0_for(L, 1)
    precision = mgmod.MG_MIXED if prec == "mixed" else mgmod.MG_FP64
    starts = dict(starts0=dev(synth.nullvec_starts(L, 1, 0, 12, L * L * 2)),
                  starts1=dev(synth.nullvec_starts(L, 1, 1, 12, (L // 4) ** 2 * 24)))
    B = synth.rhs(L, 1, 0, nrhs=7)
    gs = mgmod.mg_setup(dev(U), L, L, m0, params=mgmod.default_params(precision=precision), **starts)
    gp = mgmod.mg_setup(dev(U), L, L, m0, params=mgmod.default_params(precision=precision, parallel=3), **starts)
    try:
        Xs = torch.zeros(B.shape, dtype=torch.complex128, device="cuda")
        Xp = torch.zeros(B.shape, dtype=torch.complex128, device="cuda")
        _, its, rrs, sts = mgmod.mg_solve(gs, dev(B), Xs, 7, 1e-8)
        _, itp, rrp, stp = mgmod.mg_solve(gp, dev(B), Xp, 7, 1e-8)
        assert its == itp
        assert sts["dr_solves"] == stp["dr_solves"] == 1
        assert sts["mvps"] == stp["mvps"]
        assert np.array_equal(host(Xs), host(Xp))
        Xh = host(Xp)
        for i in range(7):
            assert rrp[i] <= 1e-8
            assert _true_relres(U, m0, Xh[i], B[i]) <= 1.0001e-8
        # a second call reuses the contexts (host buffers this time); right-hand side
        # 0 now runs GMRES-Proj instead of building the space, the others repeat exactly
        Xh2 = np.zeros_like(B)
        _, it2, rr2, st2 = mgmod.mg_solve(gp, B, Xh2, 7, 1e-8)
        assert st2["dr_solves"] == 0
        assert np.array_equal(Xh2[1:], Xh[1:])
        assert _true_relres(U, m0, Xh2[0], B[0]) <= 1.0001e-8
    finally:
        gs.close()
        gp.close()


def _requests():
    """(key, L, config, nrhs) of a small mixed stream over two lattice sizes."""
    return [(1032, 32, 0, 3), (1064, 64, 0, 2), (2032, 32, 1, 1), (1032, 32, 0, 2), (1064, 64, 0, 4),
            (2064, 64, 1, 1), (2032, 32, 1, 3)]


def _submit(srv, req, tag):
    key, L, c, nrhs = req
    U = synth.gauge_field(L, c)
    b = synth.rhs(L, c, 50 + tag, nrhs=nrhs)
    x = np.zeros_like(b)
    t = srv.submit(key, U, L, L, synth.m0_for(L, c), b, x, nrhs, 1e-8,
                   starts0=synth.nullvec_starts(L, c, 0, 12, L * L * 2),
                   starts1=synth.nullvec_starts(L, c, 1, 12, (L // 4) ** 2 * 24))
    return t, U, b, x


def test_server_results_same_alone_and_in_mix(mgmod):
    reqs = _requests()
    p = mgmod.default_params(precision=mgmod.MG_MIXED)
    alone = []
    with mgmod.Server(p, workers=4) as srv:
        for i, r in enumerate(reqs):
            t, U, b, x = _submit(srv, r, i)
            st, it, rr, lat = srv.wait(t, r[3])
            alone.append((x, rr))
    with mgmod.Server(p, workers=4) as srv:
        subs = [_submit(srv, r, i) for i, r in enumerate(reqs)]
        for (t, U, b, x), r, (xa, rra) in zip(subs, reqs, alone):
            st, it, rr, lat = srv.wait(t, r[3])
            assert lat > 0
            for j in range(r[3]):
                assert rr[j] <= 1e-8
                assert _true_relres(U, synth.m0_for(r[1], r[2]), x[j], b[j]) <= 1.0001e-8
            # the same arithmetic alone and in the mix
            assert np.array_equal(x, xa)
        info = srv.stats()
        assert info["completed"] == len(reqs) and info["resident_keys"] == 4 and info["evictions"] == 0


def test_server_budget_evicts_and_stays_correct(mgmod):
    p = mgmod.default_params(precision=mgmod.MG_MIXED)
    reqs = [(1032, 32, 0, 2), (2032, 32, 1, 2), (1032, 32, 0, 1), (2032, 32, 1, 1)]
    with mgmod.Server(p, hbm_budget_bytes=1, workers=2) as srv:  # room for one hierarchy at a time
        outs = []
        for i, r in enumerate(reqs):
            t, U, b, x = _submit(srv, r, i)
            st, it, rr, lat = srv.wait(t, r[3])
            outs.append((U, b, x, r))
        for U, b, x, r in outs:
            for j in range(r[3]):
                assert _true_relres(U, synth.m0_for(r[1], r[2]), x[j], b[j]) <= 1.0001e-8
        info = srv.stats()
        assert info["evictions"] >= 2 and info["resident_keys"] == 1


def _kappa(U, m0):
    """||D|| ||D^-1|| by power iterations (sparse LU for the inverse)."""
    import scipy.sparse.linalg as spla
    M = dirac.stencil_sparse(dirac.wilson_stencil(U, m0)).tocsc()
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


def test_block_server_batches_across_requests(mgmod):
    """Block precision: queued items of one key from several requests are solved
    together.  Every result meets the tolerance on the true residual, and a result
    differs from the same request served alone by at most what two solutions that
    both meet the tolerance can differ by (kappa (rr_alone + rr_mix))."""
    reqs = _requests()
    p = mgmod.default_params(precision=mgmod.MG_MIXED_BF16)
    alone = []
    with mgmod.Server(p, workers=3) as srv:
        for i, r in enumerate(reqs):
            t, U, b, x = _submit(srv, r, i)
            st, it, rr, lat = srv.wait(t, r[3])
            alone.append((x, rr))
        assert srv.stats()["max_batch"] == max(r[3] for r in reqs)
    kap = {}
    with mgmod.Server(p, workers=3) as srv:
        subs = [_submit(srv, r, i) for i, r in enumerate(reqs)]
        for (t, U, b, x), r, (xa, rra) in zip(subs, reqs, alone):
            st, it, rr, lat = srv.wait(t, r[3])
            m0 = synth.m0_for(r[1], r[2])
            if r[0] not in kap:
                kap[r[0]] = _kappa(U, m0)
            for j in range(r[3]):
                assert rr[j] <= 1e-8
                assert _true_relres(U, m0, x[j], b[j]) <= 1.0001e-8
                assert rel2(x[j], xa[j]) <= kap[r[0]] * (rr[j] + rra[j]), (r, j)
        info = srv.stats()
        assert info["completed"] == len(reqs) and info["resident_keys"] == 4
        # the items of a key queued during its cold start ran as one gathered block
        assert info["max_batch"] > max(r[3] for r in reqs)
        assert info["batches"] < sum(r[3] for r in reqs)


def test_block_server_budget_evicts_and_stays_correct(mgmod):
    p = mgmod.default_params(precision=mgmod.MG_MIXED_FP16, rhs_block=16)
    reqs = [(1032, 32, 0, 2), (2032, 32, 1, 3), (1032, 32, 0, 1), (2032, 32, 1, 1)]
    with mgmod.Server(p, hbm_budget_bytes=1, workers=2) as srv:  # room for one hierarchy at a time
        outs = []
        for i, r in enumerate(reqs):
            t, U, b, x = _submit(srv, r, i)
            st, it, rr, lat = srv.wait(t, r[3])
            outs.append((U, b, x, r))
        for U, b, x, r in outs:
            for j in range(r[3]):
                assert _true_relres(U, synth.m0_for(r[1], r[2]), x[j], b[j]) <= 1.0001e-8
        info = srv.stats()
        assert info["evictions"] >= 2 and info["resident_keys"] == 1
