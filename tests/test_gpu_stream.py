"""TTC_LOAD_STREAM handles (no light-triangle list: every count enumerates
the triangles again and counts the light ones as it finds them) against the
oracle and against a handle that keeps the list."""
import numpy as np
import pytest

import oracle
from paper_2106_02762_gb300 import synth, ttc

pytestmark = pytest.mark.gpu

UNB = synth.LARGE_PLAIN_DELTA_UNBOUNDED
STATS = ("tau", "tau_light", "tau_heavy", "tau_hwarp", "tau_hcta", "tau_huge", "work_bytes", "work_bytes_heavy",
         "enum_elems", "light_pairs", "kappa", "peel_rounds", "m", "m_s")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _heavy_graph():
    # three pairs of 300 edges (one heavy triangle) plus a light fringe
    rng = np.random.default_rng(5)
    k = 300
    s = np.concatenate([np.zeros(k), np.ones(k), np.zeros(k), rng.integers(0, 6, 400)]).astype(np.uint32)
    d = np.concatenate([np.ones(k), np.full(k, 2), np.full(k, 2), rng.integers(3, 30, 400)]).astype(np.uint32)
    flip = rng.integers(0, 2, s.size).astype(bool)
    s, d = np.where(flip, d, s), np.where(flip, s, d)
    t = rng.integers(0, 5000, s.size).astype(np.int64)
    return s, d, t


GRAPHS = {
    "tiny_plain": synth.tiny_plain,
    "random_tiny": lambda: synth.random_tiny(3, 8, 60, 20),
    "heavy": _heavy_graph,
    "power_law_small": lambda: synth.large_plain(scale=0.002),
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_streamed_counts_match_oracle(name):
    s, d, t = GRAPHS[name]()
    # five queries: two full groups of two and a single one, plus the
    # unbounded query in the middle
    deltas = [tuple(int(x) for x in q) for q in synth.delta_sweep(4, 1, 4000)]
    deltas.insert(2, tuple(int(x) for x in UNB))
    want = oracle.count(s, d, t, deltas)
    g = ttc.Graph(s, d, t, streamed=True)
    ref = ttc.Graph(s, d, t)
    assert (g.count_batch(deltas) == want).all()
    assert (np.stack([g.count(q) for q in deltas]) == want).all()
    gi, ri = g.info(), ref.info()
    for key in STATS:
        assert gi[key] == ri[key], key
    g.free()
    ref.free()


def test_streamed_count_in_many_chunks(monkeypatch):
    # a collecting buffer of 64 records: the light triangles are collected
    # and counted in many chunks of work items (each at least one item)
    s, d, t = synth.large_plain(scale=0.002)
    deltas = [tuple(int(x) for x in synth.LARGE_PLAIN_DELTA), tuple(int(x) for x in UNB), (600, 300, 300)]
    want = oracle.count(s, d, t, deltas)
    monkeypatch.setenv("TTC_STREAM_CHUNK", "64")
    g = ttc.Graph(s, d, t, streamed=True)
    assert (g.count_batch(deltas) == want).all()
    assert (g.count(deltas[0]) == want[0]).all()
    g.free()


def test_streamed_light_path_only_and_heavy_path_only():
    # every triangle light (threshold 2^20), then every triangle heavy
    # (threshold 1): the streamed count covers both bins alone
    s, d, t = _heavy_graph()
    deltas = [(3000, 1500, 1500), tuple(int(x) for x in UNB)]
    want = oracle.count(s, d, t, deltas)
    for light_max in (1 << 20, 1):
        g = ttc.Graph(s, d, t, light_max_pairs=light_max, streamed=True)
        assert (g.count_batch(deltas) == want).all(), light_max
        g.free()


def test_streamed_matches_listed_handle_on_power_law():
    s, d, t = synth.large_plain(scale=0.05)
    deltas = [tuple(int(x) for x in synth.LARGE_PLAIN_DELTA), tuple(int(x) for x in UNB)]
    g = ttc.Graph(s, d, t, streamed=True)
    ref = ttc.Graph(s, d, t)
    assert (g.count_batch(deltas) == ref.count_batch(deltas)).all()
    assert int(g.count(UNB).sum()) == oracle.stats(s, d, t)["prod"]
    assert g.info()["device_bytes"] < ref.info()["device_bytes"]
    g.free()
    ref.free()


def test_streamed_handles_in_many_graph_counts():
    # a many-graph call mixing streamed and listed handles: the listed ones
    # share one launch, the streamed ones are counted alone; all equal the
    # oracle
    graphs = [synth.tiny_plain(), synth.random_tiny(3, 20, 300, 50), synth.large_plain(scale=0.002)]
    deltas = [(3600, 1800, 1800), (12, 7, 9), synth.LARGE_PLAIN_DELTA]
    want = np.stack([oracle.count(s, d, t, [q])[0] for (s, d, t), q in zip(graphs, deltas)])
    for mask in ((True, False, True), (True, True, True), (False, True, False)):
        hs = [ttc.Graph(*e, streamed=st) for e, st in zip(graphs, mask)]
        assert (ttc.count_multi(hs, deltas) == want).all(), mask
        for h in hs:
            h.free()


def test_streamed_handle_refuses_list_entry_points():
    s, d, t = synth.tiny_plain()
    g = ttc.Graph(s, d, t, streamed=True)
    with pytest.raises(ttc.TTCError):
        g.sample((3600, 1800, 1800), 0, 1, 4)
    with pytest.raises(ttc.TTCError):
        g.participation((3600, 1800, 1800))
    q = np.asarray((3600, 1800, 1800), dtype=np.int64)
    out = np.zeros(8, dtype=np.uint64)
    assert ttc.lib().ttc_count_noalloc(g.handle, q.ctypes.data, out.ctypes.data, None) == -1  # TTC_ERR_INVALID
    g.free()
