"""The build with device index checks (TTC_DEBUG_BOUNDS; a memory checker's
stand-in): every pair id a count kernel reads from a triangle record, every
list range and every bulk copy's range is checked before use, and a failed
check makes the count return TTC_ERR_INTERNAL instead of reading outside an
array.  Run in a process of its own on small graphs that reach every bin,
both readings of the order and both labellings, each count compared with
the oracle: a clean run means no check fired."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent("""
    import sys
    sys.path.insert(0, %r)
    import numpy as np
    import oracle
    from paper_2106_02762_gb300 import synth, ttc
    assert ttc.LIB_PATH.endswith("_build_debug/libttc.so"), ttc.LIB_PATH
    BIG = 1 << 40
    deltas = [(3600, 1800, 1800), (BIG, BIG, BIG), (200000, 150000, 120000), (0, 0, 0)]
    rng = np.random.default_rng(5)
    k = 1500
    hs = np.concatenate([np.zeros(k), np.zeros(k), np.ones(k)]).astype(np.uint32)
    hd = np.concatenate([np.ones(k), np.full(k, 2), np.full(k, 2)]).astype(np.uint32)
    ht = rng.integers(0, 1 << 20, size=3 * k).astype(np.int64)
    graphs = [synth.large_plain(scale=0.002), (hs, hd, ht), synth.er_temporal(9, 300, 3000, 50000, 3.0)]
    graphs += [synth.random_tiny(70 + i, n=8, m=40, t_range=8) for i in range(5)]
    for s, d, t in graphs:
        for strict in (False, True):
            want = oracle.count(s, d, t, deltas, strict=strict)
            for labeling in (ttc.LABEL_HEAVIEST_VW, ttc.LABEL_SOURCE):
                g = ttc.Graph(s, d, t, labeling=labeling, strict_time=strict)
                assert (g.count_batch(deltas) == want).all()
                for q, dq in enumerate(deltas):
                    assert (g.count(dq) == want[q]).all()
                g.free()
    print("index checks clean")
""") % ROOT


def test_index_checked_build_counts_cleanly():
    from paper_2106_02762_gb300 import build
    lib = build.build(debug_bounds=True)
    env = dict(os.environ, TTC_LIB=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "index checks clean" in r.stdout
