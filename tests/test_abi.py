"""The C-ABI library builds and exports every entry point include/rbx.h declares (CPU only,
no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "rbx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rbx_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_paper_boundary():
    names = declared()
    for n in ("rbx_set_geometry", "rbx_trace_rays", "rbx_forward", "rbx_adjoint", "rbx_update_frequency",
              "rbx_reconstruct"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2211_00316_gb300 import build as B
    lib = B.build()
    L = ctypes.CDLL(lib)
    missing = [n for n in declared() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2211_00316_gb300 import rbx
    assert set(declared()) <= set(rbx.exported_symbols())


def test_binding_fails_loudly_without_library(tmp_path):
    import pytest
    from paper_2211_00316_gb300 import rbx
    saved = rbx._lib
    rbx._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            rbx.load(str(tmp_path / "missing.so"))
    finally:
        rbx._lib = saved
