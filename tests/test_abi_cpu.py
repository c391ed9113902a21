"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every function that include/dg.h declares (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dg_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dg_init", "dg_rhs", "dg_step", "dg_limit", "dg_cfl_dt"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1602_09079_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_without_gpu():
    import paper_1602_09079_gb300 as dg
    assert dg.dg_strerror(dg.DG_ERR_POSITIVITY).startswith("cell mean")
    assert dg.dg_strerror(0) == "ok"


def test_graft_build_entry():
    import __graft_entry__
    __graft_entry__.build()
