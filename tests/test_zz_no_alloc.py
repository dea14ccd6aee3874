"""The allocation-free true residual, mg_wilson_residual_noalloc, against the
library's allocating paths (collected last; also passes alone in a fresh process).

* after an FP64 solve, ||b - D x|| / ||b|| equals the relative residual mg_solve
  reports for the same x (the solver computes it with the same residual kernel
  and its own handle's reduction workspace);
* for an arbitrary x, r equals b - mg_wilson_apply(x) and the two norms equal
  those of torch on the same vectors;
* two calls in a row give the same results, and the second allocates nothing
  (free device memory is unchanged across it);
* a lattice beyond the fixed scratch is rejected with MG_EINVAL.
"""
import numpy as np
import pytest

import synth
from gpu_util import dev, host, rel2

pytestmark = pytest.mark.gpu

TOL = 1e-12  # FP64 operator parity bound of the other GPU tests


@pytest.fixture(scope="module")
def mgmod(cuda_lib):
    import paper_1912_02868_gb300 as mg
    return mg


def test_relres_matches_solver_twice(mgmod):
    import torch
    L = 32
    U = synth.gauge_field(L, 0)
    m0 = synth.m0_for(L, 0)
    b = synth.rhs(L, 0, 0)[0]
    Ud, bd = dev(U), dev(b)
    g = mgmod.mg_setup(Ud, L, L, m0, params=mgmod.default_params(precision=mgmod.MG_FP64),
                       starts0=dev(synth.nullvec_starts(L, 0, 0, 12, L * L * 2)),
                       starts1=dev(synth.nullvec_starts(L, 0, 1, 12, (L // 4) ** 2 * 24)))
    try:
        x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
        _, _, relres, _ = mgmod.mg_solve(g, bd, x, 1, 1e-10)
    finally:
        g.close()
    r = torch.empty_like(x)
    results = []
    for call in range(2):
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        rn, bn = mgmod.mg_wilson_residual_noalloc(Ud, L, L, m0, bd, x, r)
        free1 = torch.cuda.mem_get_info()[0]
        if call == 1:  # the first call on the device may load the module and look up the scratch
            assert free1 == free0
        assert abs(rn / bn - relres[0]) <= TOL * relres[0]
        assert abs(bn - np.linalg.norm(b)) <= TOL * np.linalg.norm(b)
        assert abs(rn - np.linalg.norm(host(r))) <= TOL * rn
        results.append((rn, bn))
    assert results[0] == results[1]


def test_residual_matches_wilson_apply_twice(mgmod):
    import torch
    L = 64
    U = synth.gauge_field(L, 1)
    m0 = synth.m0_for(L, 1)
    b = synth.rhs(L, 1, 0)[0]
    xh = synth.complex_gaussian(b.shape, 4242)
    Ud, bd, xd = dev(U), dev(b), dev(xh)
    y = torch.empty_like(xd)
    mgmod.mg_wilson_apply(Ud, L, L, m0, xd, y)
    ref = host(bd - y)
    r = torch.empty_like(xd)
    for _ in range(2):
        r.fill_(0)
        rn, bn = mgmod.mg_wilson_residual_noalloc(Ud, L, L, m0, bd, xd, r)
        rh = host(r)
        assert rel2(rh, ref) <= TOL
        assert abs(rn - np.linalg.norm(ref)) <= TOL * np.linalg.norm(ref)
        assert abs(bn - np.linalg.norm(b)) <= TOL * np.linalg.norm(b)


def test_oversize_lattice_rejected(mgmod):
    import torch
    a = torch.zeros(8, dtype=torch.complex128, device="cuda")
    b = torch.zeros(8, dtype=torch.complex128, device="cuda")
    c = torch.zeros(8, dtype=torch.complex128, device="cuda")
    d = torch.zeros(8, dtype=torch.complex128, device="cuda")
    with pytest.raises(mgmod.MGError) as e:
        mgmod.mg_wilson_residual_noalloc(a, 2048, 1024, 0.1, b, c, d)
    assert e.value.status == mgmod._lib.MG_EINVAL
    assert "exceeds the fixed residual scratch" in str(e.value)
