"""Launch-shape autotuner (mg_params.autotune) and pinned shapes
(mg_set_launch_shape).

A launch shape only groups sites into blocks (threads per block of the
one-thread-per-site Wilson apply, sites per block of the FP32 stencils), so
every shape must give the same result bit for bit:

* every candidate shape of every level apply, pinned on one handle, gives the
  built-in shape's output bit for bit, in FP32 and (level 0) FP64, for D and
  D^+, on hierarchies whose grids span one block to many (64^2: 16 coarsest
  sites, fewer than the largest blocks hold; 256^2: 4096 intermediate sites),
  with ragged last blocks (4096 and 256 sites by 12 or 24 a block);
* the tuner reports a candidate shape (or 0) and a chosen time no slower than
  the built-in one where it tunes, nothing for the FP64 stencils, and nothing
  with autotune off;
* a whole mixed solve gives the same solution bits and outer count with the
  tuner on and off;
* on a 48^2 lattice, whose second tile (warp) of each row is ragged, the fine
  apply pinned to each shared-memory tile and register-column shape gives the
  built-in bits (D and D^+,
  FP32 and FP64), and so does a whole mixed solve with it pinned in both
  precisions (the fused residual b - D x then runs in the tile kernel too);
* shapes that are not candidates are refused.
"""
import numpy as np
import pytest

import synth
import oracle_cache as oc
from oracle import dirac
from gpu_util import dev, host

pytestmark = pytest.mark.gpu

WILSON = (64, 128, 256, 1004, 1008, 2002, 2004)  # threads a block; 1000 + r: 32 x r shared-memory tiles;
#                                                  2000 + r: r-site columns a lane, shuffles
LR = (4, 8, 12, 16)
DENSE = (4, 8, 16, 24, 32)


@pytest.fixture(scope="module")
def mgmod(cuda_lib):
    import paper_1912_02868_gb300 as mg
    return mg


def _handle(mgmod, L, **params):
    U, m0, h = oc.hier(L)
    p = mgmod.default_params(**params)
    return mgmod.mg_setup_from_vectors(dev(U), L, L, m0, dev(h.nullvecs[0]), dev(h.nullvecs[1]), params=p), h


def _cands(mgmod, g, level, prec):
    if level == 0:
        return WILSON
    if prec == mgmod.MG_F64:
        return ()
    return LR if mgmod.mg_stencil_info(g, level)[0] else DENSE


@pytest.mark.parametrize("L", [64, 256])
def test_every_shape_same_bits(mgmod, L):
    import torch
    g, h = _handle(mgmod, L, precision=mgmod.MG_MIXED)
    try:
        for level in range(3):
            shape = h.shapes[level]
            xv = synth.complex_gaussian(shape, 7700 + L + level)
            for prec, dt in ((mgmod.MG_F32, torch.complex64), (mgmod.MG_F64, torch.complex128)):
                cands = _cands(mgmod, g, level, prec)
                for dagger in (False, True):
                    ref = torch.zeros(shape, dtype=dt, device="cuda")
                    mgmod.mg_set_launch_shape(g, level, prec, 0)
                    mgmod.mg_apply(g, level, dev(xv, dt), ref, dagger=dagger, precision=prec)
                    for c in cands:
                        y = torch.full(shape, float("nan"), dtype=dt, device="cuda")
                        mgmod.mg_set_launch_shape(g, level, prec, c)
                        mgmod.mg_apply(g, level, dev(xv, dt), y, dagger=dagger, precision=prec)
                        assert torch.equal(y, ref), (level, prec, c, dagger)
                mgmod.mg_set_launch_shape(g, level, prec, 0)
    finally:
        g.close()


@pytest.mark.parametrize("autotune", [1, 0])
def test_reported_shapes(mgmod, autotune):
    g, _ = _handle(mgmod, 256, precision=mgmod.MG_MIXED, autotune=autotune)
    try:
        for level in range(3):
            for prec in (mgmod.MG_F32, mgmod.MG_F64):
                shape, t_chosen, t_builtin = mgmod.mg_launch_shape(g, level, prec)
                cands = _cands(mgmod, g, level, prec)
                if not autotune or not cands:
                    assert (shape, t_chosen, t_builtin) == (0, 0.0, 0.0), (level, prec)
                    continue
                assert shape == 0 or shape in cands
                assert 0 < t_chosen <= t_builtin
                if shape:
                    assert t_chosen <= 0.97 * t_builtin
        with pytest.raises(Exception):
            mgmod.mg_set_launch_shape(g, 0, mgmod.MG_F32, 96)
        with pytest.raises(Exception):
            mgmod.mg_set_launch_shape(g, 1, mgmod.MG_F64, 8)
    finally:
        g.close()


def test_solve_same_bits_tuned_or_not(mgmod):
    import torch
    L = 128
    out = []
    b = synth.rhs(L, 0, 3)[0]
    for autotune in (1, 0):
        g, _ = _handle(mgmod, L, precision=mgmod.MG_MIXED, autotune=autotune)
        try:
            x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
            _, it, rr, _ = mgmod.mg_solve(g, dev(b), x, 1, 1e-8)
            out.append((host(x), it[0], rr[0]))
        finally:
            g.close()
    assert out[0][1] == out[1][1] and out[0][2] == out[1][2]
    assert np.array_equal(out[0][0], out[1][0])



@pytest.mark.parametrize("tile", [1004, 1008, 2002, 2004])
def test_tiled_fine_apply_ragged_and_in_solve(mgmod, tile):
    """48^2 lattice: a tile row (a warp's columns) holds 32 sites, so the second of
    every row is ragged (16 sites) and its neighbours wrap inside it.  Level-0 applies (D and
    D^+, FP32 and FP64) equal the built-in shape's bit for bit, and so does a whole
    mixed solve with the fine apply pinned to the tile in both precisions, which
    also runs the fused residual b - D x of the V-cycle and of the FP64 outer
    solve in the tile kernel."""
    import torch
    L, m0 = 48, 0.2
    U = synth.gauge_field(L, 0)
    b = synth.rhs(L, 0, 4)[0]
    xv = synth.complex_gaussian((L * L * 2,), 7790)
    out = []
    for shape in (0, tile):
        g = mgmod.mg_setup(dev(U), L, L, m0, params=mgmod.default_params(precision=mgmod.MG_MIXED, autotune=0),
                           starts0=dev(synth.nullvec_starts(L, 0, 0, 12, L * L * 2)),
                           starts1=dev(synth.nullvec_starts(L, 0, 1, 12, (L // 4) ** 2 * 24)))
        try:
            applies = []
            for prec, dt in ((mgmod.MG_F32, torch.complex64), (mgmod.MG_F64, torch.complex128)):
                mgmod.mg_set_launch_shape(g, 0, prec, shape)
                assert mgmod.mg_launch_shape(g, 0, prec)[0] == shape
                for dagger in (False, True):
                    y = torch.full((L * L * 2,), float("nan"), dtype=dt, device="cuda")
                    mgmod.mg_apply(g, 0, dev(xv, dt), y, dagger=dagger, precision=prec)
                    applies.append(host(y))
            x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
            _, it, rr, _ = mgmod.mg_solve(g, dev(b), x, 1, 1e-8)
            out.append((applies, host(x), it[0], rr[0]))
        finally:
            g.close()
    for a, c in zip(out[0][0], out[1][0]):
        assert np.array_equal(a, c)
    r = np.linalg.norm(dirac.wilson(U, out[0][1], m0) - b) / np.linalg.norm(b)
    assert out[0][3] <= 1e-8 and r <= 1.0001e-8
    assert out[0][2] == out[1][2] and out[0][3] == out[1][3]
    assert np.array_equal(out[0][1], out[1][1])
