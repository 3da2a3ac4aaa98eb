"""ttc_count_noalloc: the count for callers that cannot allocate device memory
(beside a framework allocator that owns the device's memory, or in
latency-critical loops).  Its scratch is a fixed static device array, so this
checks, through the C ABI, that it gives exactly what ttc_count gives, on two
calls in a row (the array keeps the previous call's contents), including
graphs whose largest triangles take the flat path that keeps its prefix
arrays in that array, and that a graph too large for the array is refused.

Kept in a file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

from paper_2106_02762_gb300 import synth, ttc

pytestmark = pytest.mark.gpu

BIG = 1 << 40


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _noalloc(g, delta):
    d = np.ascontiguousarray(np.asarray(delta, dtype=np.int64))
    out = np.zeros(8, dtype=np.uint64)
    rc = ttc.lib().ttc_count_noalloc(g.handle, d.ctypes.data, out.ctypes.data, None)
    return rc, out


@pytest.mark.parametrize("light_max", [0, 1])
def test_noalloc_matches_count_twice(light_max):
    s, d, t = synth.large_plain(scale=0.002)
    g = ttc.Graph(s, d, t, light_max_pairs=light_max)
    assert g.info()["tau_heavy"] > 0
    for delta in (synth.LARGE_PLAIN_DELTA, (BIG, BIG, BIG)):
        want = g.count(delta)
        for _ in range(2):
            rc, got = _noalloc(g, delta)
            assert rc == 0, ttc.last_error()
            assert (got == want).all()
    g.free()


def _huge_graph(big):
    """Three pairs of a triangle {0, 1, 2} with `big`, 1500 and 1500 edges
    (so A + B exceeds one CTA's capacity and the triangle takes the flat
    path), plus the power-law fringe of a small seeded graph on other ids."""
    rng = np.random.default_rng(7)
    sizes = (big, 1500, 1500)
    ends = ((0, 1), (0, 2), (1, 2))
    src, dst = [], []
    for (a, b), k in zip(ends, sizes):
        flip = rng.integers(0, 2, size=k).astype(bool)
        src.append(np.where(flip, b, a))
        dst.append(np.where(flip, a, b))
    s, d, t = synth.large_plain(scale=0.001)
    src = np.concatenate(src + [s.astype(np.int64) + 3]).astype(np.uint32)
    dst = np.concatenate(dst + [d.astype(np.int64) + 3]).astype(np.uint32)
    tt = np.concatenate([rng.integers(0, 1 << 20, size=sum(sizes)), t]).astype(np.int64)
    return src, dst, tt


@pytest.mark.parametrize("big", [1500, 70000])
def test_noalloc_flat_path_twice(big):
    # 70000 edges on one pair need 64-bit prefix sums (lists of 2^16 or more)
    g = ttc.Graph(*_huge_graph(big))
    assert g.info()["tau_huge"] >= 1
    for delta in ((BIG, BIG, BIG), (200000, 150000, 120000), (3000, 1000, 2500)):
        want = g.count(delta)
        assert want.sum() > 0
        for _ in range(2):
            rc, got = _noalloc(g, delta)
            assert rc == 0, ttc.last_error()
            assert (got == want).all()
    g.free()


def test_noalloc_refuses_graph_beyond_its_scratch():
    # one triangle with 2^21 edges on each pair: its prefix arrays need about
    # 2 * 2^21 entries of 64 bytes, more than the static array holds
    k = 1 << 21
    s = np.concatenate([np.zeros(k), np.ones(k), np.zeros(k)]).astype(np.uint32)
    d = np.concatenate([np.ones(k), np.full(k, 2), np.full(k, 2)]).astype(np.uint32)
    t = np.arange(3 * k, dtype=np.int64)
    g = ttc.Graph(s, d, t)
    rc, _ = _noalloc(g, (10, 5, 5))
    assert rc == -2
    assert "ttc_count_noalloc holds" in ttc.last_error()
    g.free()
