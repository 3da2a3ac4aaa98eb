"""Full-size checks: the power-law workload at its benchmark size (n = 1M,
10M pairs, ~60M edges) in the launch configuration bench.py times.

- Totals: the oracle's counts for the step's two queries and a wide finite
  one, computed once by tests/golden/make_power_law_counts.py (O1 with the
  forward enumeration) and stored with the input's SHA-256, are compared
  bit-exactly; the unbounded total also equals Def. 1's closed form
  (sum over static triangles of s_uv s_uw s_vw).
- Per triangle: strided samples of the light and the prefix-sum bins are
  compared with the oracle one triangle at a time.
- Properties that hold at any size: monotonicity and normalisation.
"""
import hashlib

import numpy as np
import pytest

import oracle
from paper_2106_02762_gb300 import synth, ttc
from tests.golden import readers

pytestmark = pytest.mark.gpu

BIG = 1 << 40


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _sampled_parity(src, dst, t, g, deltas, n_light=600, n_heavy=300):
    info = g.info()
    for delta in deltas:
        for first, count, n in ((0, info["tau_light"], n_light),
                                (info["tau_light"], info["tau_heavy"], n_heavy)):
            if count == 0:
                continue
            stride = max(1, count // n)
            tri, got = g.sample(delta, first, stride, n)
            assert len(tri) > 0
            want = oracle.count_triangles(src, dst, t, tri, [delta])[:, 0, :]
            assert (got == want).all(), (delta, first)


def test_sample_matches_oracle_small():
    s, d, t = synth.large_plain(scale=0.003)
    g = ttc.Graph(s, d, t)
    _sampled_parity(s, d, t, g, [synth.LARGE_PLAIN_DELTA, (BIG, BIG, BIG), (7200, 600, 7000)])
    # the sampled triangles' counts also add up: sample everything
    info = g.info()
    tri, per = g.sample(synth.LARGE_PLAIN_DELTA, 0, 1, info["tau"])
    assert len(tri) == info["tau"]
    assert (per.sum(axis=0) == g.count(synth.LARGE_PLAIN_DELTA)).all()
    g.free()


def _sha256(src, dst, t):
    h = hashlib.sha256()
    for a in (src, dst, t):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


@pytest.mark.slow
def test_full_size_power_law_totals_match_oracle():
    fields, rows = readers.power_law_counts()
    s, d, t = synth.large_plain()
    assert _sha256(s, d, t) == fields["sha256"], "the generator made another graph than the stored counts'"
    g = ttc.Graph(s, d, t)
    info = g.info()
    for k in ("n", "m", "m_s", "tau", "sigma_max", "work_bytes"):
        assert info[k] == fields[k], k
    deltas = [r[0] for r in rows]
    want = np.array([r[1] for r in rows], dtype=np.uint64)
    # the bench step's launch configuration: one batched call of its queries
    got = g.count_batch(deltas[:2])
    assert (got == want[:2]).all()
    for q, dq in enumerate(deltas):
        assert (g.count(dq) == want[q]).all(), dq
    unb = deltas.index(synth.LARGE_PLAIN_DELTA_UNBOUNDED)
    assert int(want[unb].sum()) == fields["prod"]
    g.free()


@pytest.mark.slow
def test_full_size_power_law_sampled():
    s, d, t = synth.large_plain()
    g = ttc.Graph(s, d, t)
    info = g.info()
    assert info["m"] == s.size and info["tau"] > 10 ** 8
    _sampled_parity(s, d, t, g, [synth.LARGE_PLAIN_DELTA, synth.LARGE_PLAIN_DELTA_UNBOUNDED],
                    n_light=2000, n_heavy=500)
    # properties that hold at any size: monotone in each delta component,
    # and normalisation leaves the counts unchanged
    base = g.count(synth.LARGE_PLAIN_DELTA)
    for up in ((172800, 43200, 43200), (86400, 86400, 43200), (86400, 43200, 86400)):
        assert (g.count(up) >= base).all()
    assert (g.count((86400, 1 << 40, 43200)) == g.count((86400, 86400, 43200))).all()
    # orientation and labelling do not change the counts
    g2 = ttc.Graph(s, d, t, labeling=ttc.LABEL_SOURCE, orientation=ttc.ORIENT_DEGREE)
    assert (g2.count(synth.LARGE_PLAIN_DELTA) == base).all()
    g2.free()
    g.free()
