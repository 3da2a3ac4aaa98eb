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


def test_count_hash_tracks_the_light_kernel_sources_only():
    # the hash that ties the light kernel's DRAM capture to its source moves
    # with the light bin and the device headers, not with the heavy bins or
    # the host-side handle
    from paper_2106_02762_gb300 import build
    files = {f: open(os.path.join(build.CSRC, f), "rb").read() for f, _ in build._LIGHT_SOURCES}

    def hashed(edit=None):
        return build.count_source_hash(lambda f: edit(f, files[f]) if edit else files[f])

    def after(name, marker, text):
        def edit(f, data):
            if f != name:
                return data
            i = data.index(marker.encode()) + len(marker)
            return data[:i] + text + data[i:]
        return edit

    base = hashed()
    assert base == build.count_source_hash()
    heavy = "// ---------------------------------------------------------------- heavy: per-edge math"
    assert hashed(after("count.cu", heavy, b"\n// a heavy-bin change\n")) == base
    assert hashed(after("graph.cuh", "struct ttc_graph {", b"\n    int host_side_field;\n")) == base
    light = "// ---------------------------------------------------------------- light bin"
    assert hashed(after("count.cu", light, b"\n// a light-bin change\n")) != base
    assert hashed(after("graph.cuh", "struct GraphView {", b"\n    int device_field;\n")) != base
    assert hashed(lambda f, d: d + b"\n" if f == "count_dev.cuh" else d) != base
