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
            names |= set(re.findall(r"^\s*(?:grng_status|void|const char\*|int64_t)\s+(\w+)\s*\(", src, flags=re.M))
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


def test_learned_entry_points_host_checks():
    """Parameter count agrees with the oracle; invalid arguments are refused on the host
    (no device work is started, so this runs without a GPU)."""
    import ctypes

    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_2208_10022_gb300 as g
    L = g.lib()
    assert "grng_mlp_nparams" in _declared()
    assert g.mlp_nparams() == oracle.mlp_nparams() == 20865
    assert L.grng_mlp_score(None, None, 0, None) == g.GRNG_EINVAL
    loss = ctypes.c_float(0.0)
    assert L.grng_mlp_loss_grad(None, None, None, None, 0, ctypes.byref(loss), None) == g.GRNG_EINVAL
    assert L.grng_mlp_train(None, None, None, 0, 1, 1, ctypes.c_float(1e-3), None, None) == g.GRNG_EINVAL
    assert L.grng_mlp_dataset(None, None, None, 0, None) == g.GRNG_EINVAL
    assert b"must" in L.grng_last_error() or b"NULL" in L.grng_last_error()


def test_search_and_skeleton_entry_points_host_checks():
    """The search and skeleton entry points refuse a NULL index on the host, before any device
    work (so this runs without a GPU)."""
    import ctypes

    import __graft_entry__
    __graft_entry__.build()
    import paper_2208_10022_gb300 as g
    L = g.lib()
    tot = ctypes.c_int64(-1)
    assert L.rng_search_batch(None, None, 1, ctypes.byref(tot)) == g.GRNG_EINVAL
    assert tot.value == -1
    assert L.rng_search_result(None, None, None, 0) == g.GRNG_EINVAL
    assert L.rng_build_skeleton(None, ctypes.c_double(1.0)) == g.GRNG_EINVAL
    assert b"NULL" in L.grng_last_error()
