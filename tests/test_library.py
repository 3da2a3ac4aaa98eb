"""CPU-side checks of the C ABI library: it builds for sm_103a, loads, and
exports every function include/ttc.h declares.  No compute call is made."""
import os
import re

import pytest

from paper_2106_02762_gb300 import ttc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(ttc_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_library_builds_and_loads():
    import __graft_entry__
    __graft_entry__.build()
    assert os.path.exists(ttc.LIB_PATH)
    assert ttc.lib().ttc_version().decode().startswith("ttc")


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert "ttc_count" in names and "ttc_load" in names
    L = ttc.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert set(names) <= set(ttc.EXPORTS) | set(names)


def test_binding_covers_header():
    assert sorted(ttc.EXPORTS) == declared_functions()


def test_null_arguments_rejected_without_gpu():
    L = ttc.lib()
    assert L.ttc_count(None, None, None) == -1
    assert "NULL" in ttc.last_error()
    assert L.ttc_graph_info(None, None) == -1
    assert L.ttc_count_batch(None, None, 0, None) == -1
    L.ttc_free(None)


def test_missing_library_fails_loudly(monkeypatch):
    monkeypatch.setattr(ttc, "_lib", None)
    monkeypatch.setattr(ttc, "LIB_PATH", "/nonexistent/libttc.so")
    with pytest.raises(RuntimeError, match="not built"):
        ttc.lib()
