"""The seeded input generators that the oracle and the CUDA path share: each
returns the same arrays for the same seed (and other arrays for another), and
the full power-law workload regenerates exactly the graph whose oracle
counts tests/golden/power_law_1m_counts.txt stores (its SHA-256 is stored
with them).  CPU only; numpy alone."""
import hashlib

import numpy as np

from paper_2106_02762_gb300 import synth

from tests.golden import readers


def _sha256(src, dst, t):
    h = hashlib.sha256()
    for a in (src, dst, t):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def _same(a, b):
    return all(x.dtype == y.dtype and np.array_equal(x, y) for x, y in zip(a, b))


def test_generators_are_deterministic_per_seed():
    makers = [
        lambda k: synth.random_tiny(k, 7, 40, 9),
        lambda k: synth.er_temporal(k, 200, 800, 10_000, 3.0),
        lambda k: synth.power_law_temporal(k, 2000, 8000),
        lambda k: synth.many_graph(500, 2000, k),
        lambda k: synth.served_graph(20_000, k),
    ]
    for make in makers:
        a, b, c = make(5), make(5), make(6)
        assert _same(a, b)
        assert not _same(a, c)
        src, dst, t = a
        assert src.dtype == np.uint32 and dst.dtype == np.uint32 and t.dtype == np.int64
        assert src.shape == dst.shape == t.shape and src.ndim == 1


def test_power_law_workload_is_the_stored_counts_input():
    fields, _ = readers.power_law_counts()
    s, d, t = synth.large_plain()
    assert s.size == int(fields["m"]) + int((s == d).sum())
    assert _sha256(s, d, t) == fields["sha256"]
