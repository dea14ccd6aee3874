"""The mixed V-cycle as a CUDA graph (mg_params.vcycle_graph): once the
deflation space exists, every V-cycle is one graph launch of the same kernels
with the same arguments, so the solve is unchanged to the bit.

* three right-hand sides solved one after the other with vcycle_graph = 1 and
  = 0: the solutions are bitwise equal, and so are the outer iteration counts,
  the residuals and every counter of mg_solve_stats;
* the graph path still counts its kernels: mg_kernel_launches advances by the
  same amount per solve in both modes;
* with apply timing on, the graph is not used, and the timers see one
  coarse-grid solve per V-cycle.
"""
import numpy as np
import pytest

import synth
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mgmod(cuda_lib):
    import paper_1912_02868_gb300 as mg
    return mg


def _solve_all(mg, L, c, nrhs, graph, timing=False):
    import torch
    U = synth.gauge_field(L, c)
    m0 = synth.m0_for(L, c)
    g = mg.mg_setup(dev(U), L, L, m0, params=mg.default_params(precision=mg.MG_MIXED, vcycle_graph=graph),
                    starts0=dev(synth.nullvec_starts(L, c, 0, 12, L * L * 2)),
                    starts1=dev(synth.nullvec_starts(L, c, 1, 12, (L // 4) ** 2 * 24)))
    out = []
    try:
        B = synth.rhs(L, c, 0, nrhs=nrhs)
        for i in range(nrhs):
            if timing and i == nrhs - 1:
                mg.mg_timing_enable(g, 2, True)
            x = torch.zeros(B[i].shape, dtype=torch.complex128, device="cuda")
            l0 = mg.mg_kernel_launches()
            st, iters, relres, stats = mg.mg_solve(g, dev(B[i]), x, 1, 1e-8)
            torch.cuda.synchronize()
            out.append((host(x), iters[0], relres[0], dict(stats), mg.mg_kernel_launches() - l0))
        if timing:
            out.append(mg.mg_timing_read(g, 2))
    finally:
        g.close()
    return out


@pytest.mark.parametrize("L,c", [(64, 0), (256, 1)])
def test_graph_equals_launches(mgmod, L, c):
    a = _solve_all(mgmod, L, c, 3, 1)
    b = _solve_all(mgmod, L, c, 3, 0)
    for (xa, ia, ra, sa, la), (xb, ib, rb, sb, lb) in zip(a, b):
        assert np.array_equal(xa, xb)
        assert ia == ib and ra == rb
        assert sa == sb
        assert la == lb
        assert ra <= 1e-8


def test_timing_turns_graph_off(mgmod):
    out = _solve_all(mgmod, 64, 0, 3, 1, timing=True)
    ms, count = out[-1]
    stats = out[-2][3]
    assert count == stats["coarse_solves"] - stats["dr_solves"] > 0
    assert ms > 0
