"""The C-ABI library builds, loads, and exports every entry point declared in include/greem.h
(no GPU needed: nothing is called that touches a device)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "greem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(greem_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_boundary_calls():
    names = _declared()
    for n in ("greem_create", "greem_destroy", "greem_build_tree", "greem_short_force", "greem_short_force_ex",
              "greem_short_force_batched", "greem_pm_force", "greem_graph_capture", "greem_graph_launch",
              "greem_get_stats", "greem_debug_dump", "greem_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_0910_0121_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    lib.greem_strerror.restype = ctypes.c_char_p
    assert b"invalid" in lib.greem_strerror(-1)


def test_binding_fails_loudly_without_library(monkeypatch):
    from paper_0910_0121_gb300 import greem
    monkeypatch.setattr(greem, "LIB_PATH", "/nonexistent/libgreem.so")
    monkeypatch.setattr(greem, "_L", None)
    with pytest.raises(ImportError):
        greem.lib()
