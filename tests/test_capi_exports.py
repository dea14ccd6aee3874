"""The C ABI library builds for sm_103a, loads, and exports every symbol that
include/mg.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "mg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    syms = header_symbols()
    for s in ("mg_setup", "mg_solve", "mg_destroy", "mg_last_error", "mg_apply", "mg_restrict", "mg_prolong"):
        assert s in syms


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="no CUDA toolkit")
def test_library_exports_every_declared_symbol():
    import paper_1912_02868_gb300 as pkg
    from paper_1912_02868_gb300 import _lib
    path = pkg.build()
    raw = ctypes.CDLL(path)
    for s in header_symbols():
        assert hasattr(raw, s), s
    lib = _lib.load()
    assert set(header_symbols()) == set(_lib.SYMBOLS)
    # host-only entry points work without a device
    p = pkg.default_params()
    assert (p.nvec, p.block, p.fgmres_m, p.dr_m, p.dr_k, p.smooth_steps) == (12, 4, 8, 30, 10, 2)
    assert (p.pair_rhs, p.vcycle_graph, p.coarse_half, p.coarse_dcgs2, p.partial_tol) == (0, 1, 1, 0, 0.0)
    assert (p.lowrank_hops, p.coarse_mma, p.autotune) == (1, 1, 1)
    out = ctypes.c_void_p()
    st = lib.mg_setup(None, 64, 64, 0.0, 12, 4, None, None, None, None, ctypes.byref(out))
    assert st == _lib.MG_EINVAL and b"gauge" in lib.mg_last_error()
    # the switches are validated before any device work (the gauge buffer is never read)
    dummy = ctypes.create_string_buffer(16)
    for field, bad in (("pair_rhs", 2), ("vcycle_graph", -1), ("coarse_half", 3), ("coarse_dcgs2", 2),
                       ("lowrank_hops", 2), ("coarse_mma", -1), ("autotune", 2)):
        q = pkg.default_params(**{field: bad})
        st = lib.mg_setup(ctypes.cast(dummy, ctypes.c_void_p), 64, 64, 0.1, 12, 4, ctypes.byref(q), None, None, None,
                          ctypes.byref(out))
        assert st == _lib.MG_EINVAL and field.encode() in lib.mg_last_error()


def test_product_path_has_no_fallback(tmp_path):
    from paper_1912_02868_gb300 import _lib
    with pytest.raises(ImportError):
        _lib.load(str(tmp_path / "libmg.so"))
