"""TTC_LOAD_STRICT_TIME (Def. 1's t1 < t2 < t3 read literally: a triple
whose edges share a timestamp is not counted) against the oracle's strict
reading, on graphs where ties are common, through every counting path."""
import numpy as np
import pytest

import oracle
from paper_2106_02762_gb300 import synth, ttc

pytestmark = pytest.mark.gpu

UNB = tuple(int(x) for x in synth.LARGE_PLAIN_DELTA_UNBOUNDED)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _heavy_tied(k=400, t_hi=300):
    # three pairs of k edges (a heavy triangle) plus a light fringe, times in
    # [0, t_hi) so that most timestamps repeat
    rng = np.random.default_rng(11)
    s = np.concatenate([np.zeros(k), np.ones(k), np.zeros(k), rng.integers(0, 6, 500)]).astype(np.uint32)
    d = np.concatenate([np.ones(k), np.full(k, 2), np.full(k, 2), rng.integers(3, 30, 500)]).astype(np.uint32)
    flip = rng.integers(0, 2, s.size).astype(bool)
    s, d = np.where(flip, d, s), np.where(flip, s, d)
    t = rng.integers(0, t_hi, s.size).astype(np.int64)
    return s, d, t


def _tiny_tied():
    s, d, t = synth.tiny_plain()
    return s, d, t // 20000  # timestamps in [0, 50): ties everywhere


DELTAS = [(30, 15, 15), (10, 3, 8), (0, 0, 0), (100, 60, 70), UNB]


@pytest.mark.parametrize("light_max", [0, 1 << 20, 1])
def test_strict_matches_oracle_on_tied_graphs(light_max):
    # light_max 1: everything on the prefix-sum paths; 2^20: everything light
    for s, d, t in (_heavy_tied(), _tiny_tied(), synth.random_tiny(4, 8, 80, 5)):
        want = oracle.count(s, d, t, DELTAS, strict=True)
        g = ttc.Graph(s, d, t, light_max_pairs=light_max, strict_time=True)
        assert (g.count_batch(DELTAS) == want).all()
        assert (np.stack([g.count(q) for q in DELTAS]) == want).all()
        g.free()


def test_strict_huge_path():
    # pairs of 3000 edges: too large for one CTA, so the flat path counts it
    s, d, t = _heavy_tied(3000, 2000)
    want = oracle.count(s, d, t, DELTAS, strict=True)
    g = ttc.Graph(s, d, t, strict_time=True)
    assert g.info()["tau_huge"] >= 1
    assert (g.count_batch(DELTAS) == want).all()
    g.free()


def test_strict_streamed_and_many_graphs():
    graphs = [_heavy_tied(), _tiny_tied(), synth.random_tiny(9, 8, 80, 5)]
    q = (30, 15, 15)
    want = np.stack([oracle.count(s, d, t, [q], strict=True)[0] for s, d, t in graphs])
    hs = [ttc.Graph(s, d, t, strict_time=True) for s, d, t in graphs]
    assert (ttc.count_multi(hs, [q] * len(hs)) == want).all()
    st = [ttc.Graph(s, d, t, strict_time=True, streamed=True) for s, d, t in graphs]
    assert (np.stack([g.count(q) for g in st]) == want).all()
    # a table may not mix the two readings of ties
    plain = ttc.Graph(*graphs[0])
    with pytest.raises(ttc.TTCError):
        ttc.count_multi([hs[0], plain], [q, q])
    for g in hs + st + [plain]:
        g.free()


def test_strict_equals_key_order_on_distinct_timestamps():
    s, d, t = synth.large_plain(scale=0.002)
    t = np.random.default_rng(1).permutation(s.size).astype(np.int64)  # all distinct
    qs = [(50000, 20000, 30000), UNB]
    a = ttc.Graph(s, d, t, strict_time=True)
    b = ttc.Graph(s, d, t)
    assert (a.count_batch(qs) == b.count_batch(qs)).all()
    a.free()
    b.free()
