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


def test_tuned_heavy_caps_are_used_and_counts_agree():
    # light threshold 17: most triangles take the prefix-sum path, so the
    # caps move triangles between its one-warp, one-CTA and flat classes
    s, d, t = synth.large_plain(scale=0.003)
    probe = [synth.LARGE_PLAIN_DELTA, (BIG, BIG, BIG)]
    (w, c, mg), ms = ttc.tune_heavy(s, d, t, probe, light_max_pairs=17)
    assert set(ms) == set(ttc.TUNE_HEAVY_CANDIDATES) and all(v > 0 for v in ms.values())
    # the first candidate (the capacities, binary searches) stays unless
    # another is more than 1% faster
    first = ttc.TUNE_HEAVY_CANDIDATES[0]
    best = min(ms, key=ms.get)
    if ms[best] >= 0.99 * ms[first]:
        best = first
    assert (w, c, mg) == (min(best[0], 128), min(max(best[1], best[0]), 2048), best[2])
    tuned = ttc.Graph(s, d, t, light_max_pairs=17)  # caps and search form 0: the tuned ones
    info = tuned.info()
    assert (info["heavy_warp_cap"], info["heavy_cta_cap"], info["heavy_merge"]) == (w, c, mg)
    assert info["tau_heavy"] > 0
    deltas = probe + [(200000, 150000, 120000), (3600, 600, 3000)]
    want = oracle.count(s, d, t, deltas)
    assert (tuned.count_batch(deltas) == want).all()
    tuned.free()
    classes = {}
    for cw, cc, cm in ttc.TUNE_HEAVY_CANDIDATES + ((1, 1, ttc.HEAVY_BINARY), (1, 64, ttc.HEAVY_MERGE)):
        g = ttc.Graph(s, d, t, light_max_pairs=17, heavy_warp_cap=cw, heavy_cta_cap=cc, heavy_merge=cm)
        i = g.info()
        assert (i["heavy_warp_cap"], i["heavy_cta_cap"], i["heavy_merge"]) == (min(cw, 128), min(max(cc, cw), 2048), cm)
        assert i["tau_hwarp"] + i["tau_hcta"] + i["tau_huge"] == i["tau_heavy"] == info["tau_heavy"]
        classes[(cw, cc)] = (i["tau_hwarp"], i["tau_hcta"], i["tau_huge"])
        assert (g.count_batch(deltas) == want).all(), (cw, cc, cm)
        g.free()
    # smaller caps move triangles to the larger classes, never back
    assert classes[(1, 1)][2] == info["tau_heavy"]
    assert classes[(64, 1024)][0] <= classes[(128, 1024)][0]
    assert classes[(128, 512)][2] >= classes[(128, 2048)][2]
