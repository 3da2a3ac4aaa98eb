"""Participation counts (ttc_count_participation): the number of
delta-temporal triangles each vertex and each static pair belongs to.  The
expected values are built here from the oracle's per-static-triangle counts
(every static triangle listed by plain adjacency sets, its count added to
its three vertices and three pairs), on graphs that reach every bin."""
import numpy as np
import pytest

import oracle
from paper_2106_02762_gb300 import synth, ttc

pytestmark = pytest.mark.gpu

BIG = 1 << 40


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _expected(s, d, t, delta):
    keep = s != d
    lo = np.minimum(s[keep], d[keep]).astype(np.int64)
    hi = np.maximum(s[keep], d[keep]).astype(np.int64)
    pairs = set(zip(lo.tolist(), hi.tolist()))
    adj = {}
    for x, y in pairs:
        adj.setdefault(x, set()).add(y)
        adj.setdefault(y, set()).add(x)
    tris = [(x, y, z) for x, y in pairs for z in adj[x] & adj[y] if z > y]
    n = int(max(s.max(), d.max())) + 1
    vert = np.zeros(n, dtype=np.uint64)
    pair = {p: 0 for p in pairs}
    if tris:
        per = oracle.count_triangles(s, d, t, tris, [delta])[:, 0, :].sum(axis=1)
        for (x, y, z), c in zip(tris, per.tolist()):
            for v in (x, y, z):
                vert[v] += np.uint64(c)
            for p in ((x, y), (x, z), (y, z)):
                pair[p] += c
    return vert, pair


def _heavy_graph():
    # three pairs of 1500 edges (a triangle for the flat path) plus a fringe
    rng = np.random.default_rng(5)
    k = 1500
    s = np.concatenate([np.zeros(k), np.ones(k), np.zeros(k), rng.integers(0, 3, 400)]).astype(np.uint32)
    d = np.concatenate([np.ones(k), np.full(k, 2), np.full(k, 2), rng.integers(3, 30, 400)]).astype(np.uint32)
    flip = rng.integers(0, 2, s.size).astype(bool)
    s, d = np.where(flip, d, s), np.where(flip, s, d)
    return s, d, rng.integers(0, 20000, s.size).astype(np.int64)


@pytest.mark.parametrize("light_max", [0, 1])
def test_participation_matches_oracle(light_max):
    cases = [(synth.random_tiny(seed, 12, 160, 40), (10, 6, 7)) for seed in range(4)]
    cases.append((synth.large_plain(scale=0.002), synth.LARGE_PLAIN_DELTA))
    cases.append((_heavy_graph(), (3000, 2000, 2500)))
    for (s, d, t), delta in cases:
        g = ttc.Graph(s, d, t, light_max_pairs=light_max)
        info = g.info()
        vert, pair = g.participation(delta)
        pv = g.pairs()
        want_v, want_p = _expected(s, d, t, delta)
        assert vert.shape == (info["n"],) and pair.shape == (info["m_s"],)
        assert (vert == want_v).all()
        assert len(pv) == len(want_p)
        assert all(int(c) == want_p[(int(a), int(b))] for (a, b), c in zip(pv, pair))
        total = int(g.count(delta).sum())
        assert int(vert.sum()) == int(pair.sum()) == 3 * total
        g.free()


def test_participation_unbounded_and_bins():
    s, d, t = _heavy_graph()
    g = ttc.Graph(s, d, t, light_max_pairs=1)
    assert g.info()["tau_huge"] >= 1
    vert, pair = g.participation((BIG, BIG, BIG))
    want_v, _ = _expected(s, d, t, (BIG, BIG, BIG))
    assert (vert == want_v).all()
    # the flat-path triangle (0, 1, 2) alone holds 1500^3 triples
    assert int(vert[0]) >= 1500 ** 3
    g.free()
