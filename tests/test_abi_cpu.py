"""CPU-side checks of the boundary: the shared library builds/loads and
exports every entry point include/rtn.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "rtn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rtn_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("rtn_create", "rtn_linearize", "rtn_rti_step", "rtn_closed_loop", "rtn_destroy",
              "rtn_last_error", "rtn_mlp_eval", "rtn_qp_solve", "rtn_plant_step"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    import paper_2203_07747_b300 as rtn
    path = rtn._build.build()
    lib = ctypes.CDLL(path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    assert sorted(rtn.EXPORTS) == sorted(declared_symbols())


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2203_07747_b300 as rtn
    monkeypatch.setattr(rtn, "_lib", None)
    monkeypatch.setattr(rtn._build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(rtn.RtnError):
        rtn.load()
