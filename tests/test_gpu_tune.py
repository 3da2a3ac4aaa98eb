"""The light-threshold tuner (ttc_tune_light): it times every candidate on
the graph, caches the fastest for graphs of that shape, later loads with no
threshold given use it, and the counts are the same at the tuned and the
default thresholds (and the oracle's)."""
import numpy as np
import pytest

import oracle
from paper_2106_02762_gb300 import synth, ttc

pytestmark = pytest.mark.gpu

BIG = 1 << 40


@pytest.fixture(scope="module", autouse=True)
def _built(tmp_path_factory):
    import os
    import __graft_entry__
    __graft_entry__.build()
    os.environ["TTC_TUNE_CACHE"] = str(tmp_path_factory.mktemp("tune") / "tune.json")


def test_tuned_threshold_is_used_and_counts_agree():
    s, d, t = synth.large_plain(scale=0.003)
    probe = [synth.LARGE_PLAIN_DELTA, (BIG, BIG, BIG)]
    chosen, ms = ttc.tune_light(s, d, t, probe)
    assert chosen in ttc.TUNE_CANDIDATES
    assert set(ms) == set(ttc.TUNE_CANDIDATES) and all(v > 0 for v in ms.values())
    assert ms[chosen] == min(ms.values())
    tuned = ttc.Graph(s, d, t)  # light_max_pairs = 0: the tuned value
    assert tuned.info()["light_max_pairs"] == chosen
    deltas = probe + [(200000, 150000, 120000), (3600, 600, 3000)]
    want = oracle.count(s, d, t, deltas)
    assert (tuned.count_batch(deltas) == want).all()
    for c in ttc.TUNE_CANDIDATES:
        g = ttc.Graph(s, d, t, light_max_pairs=c)
        assert g.info()["light_max_pairs"] == c
        assert (g.count_batch(deltas) == want).all()
        g.free()
    tuned.free()
