"""The C ABI library loads and exports every function include/grng.h declares (CPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:grng_status|void|const char\*)\s+(\w+)\s*\(", src, flags=re.M))
    return names


def test_library_exports_declared_symbols():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2208_10022_gb300 as g
    L = g.lib()
    declared = _declared()
    assert declared, "no declarations found"
    for name in sorted(declared):
        assert hasattr(L, name), f"{name} not exported"
    assert set(g.EXPORTS) <= declared


def test_binding_raises_without_library(monkeypatch, tmp_path):
    import paper_2208_10022_gb300 as g
    monkeypatch.setattr(g, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(g, "_lib", None)
    with pytest.raises(ImportError):
        g.lib()
