"""Writes power_law_1m_counts.txt: the oracle's counts on the full power-law
workload (synth.large_plain(), n = 1M, 10M pairs, about 60M edges), for the
full-size parity test.

Only the oracle runs here: O1 with the static triangles found by the forward
rule (oracle.count_fwd; the same counts as oracle.count, which the tests
check on smaller graphs), and the static statistics of the same enumeration
(oracle.stats_fwd; ``prod`` is Def. 1's count with every window unbounded,
the sum over static triangles of s_uv s_uw s_vw).  The input's SHA-256 is
stored with the counts, so a test can tell that it regenerated the same
graph.

    python tests/golden/make_power_law_counts.py
"""
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "power_law_1m_counts.txt")

# the step's configured and unbounded windows, and a wide finite triple whose
# windows end inside many pairs' edge lists
DELTAS = [(86400, 43200, 43200), (1 << 31, 1 << 31, 1 << 31), (1 << 26, 1 << 25, 1 << 25)]


def graph_sha256(src, dst, t):
    h = hashlib.sha256()
    for a in (src, dst, t):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def main():
    import oracle
    from paper_2106_02762_gb300 import synth
    oracle.build()
    src, dst, t = synth.large_plain()
    w = time.perf_counter()
    counts = oracle.count_fwd(src, dst, t, DELTAS)
    count_s = time.perf_counter() - w
    st = oracle.stats_fwd(src, dst, t)
    with open(OUT, "w") as fh:
        fh.write("# oracle counts on synth.large_plain() (written by make_power_law_counts.py)\n")
        fh.write("sha256: %s\n" % graph_sha256(src, dst, t))
        for k in ("n", "m", "m_s", "tau", "sigma_max", "work_bytes", "prod"):
            fh.write("%s: %d\n" % (k, st[k]))
        for d, c in zip(DELTAS, counts):
            fh.write("delta %d %d %d: %s\n" % (d + (" ".join(str(int(x)) for x in c),)))
        fh.write("# oracle O1f wall time: %.1f s on %d host threads\n" % (count_s, os.cpu_count() or 1))
    print(open(OUT).read())


if __name__ == "__main__":
    main()
