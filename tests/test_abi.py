"""The C-ABI library builds for sm_103a and exports every entry point that
include/tpc.h declares (no GPU needed: no compute call is made)."""
from __future__ import annotations

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(tpc_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    from paper_2601_20569_gb300 import build

    lib = ctypes.CDLL(build.build())
    names = declared_functions()
    assert "tpc_init" in names and "tpc_track_timeframe" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2601_20569_gb300 import tpc

    monkeypatch.setattr(tpc, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(tpc, "_lib", None)
    import pytest

    with pytest.raises(ImportError):
        tpc.load()
