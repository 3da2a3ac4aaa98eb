"""Pins for the CPU oracle: it is checked against what the paper and the
mathematics fix, never against itself.

- Table 1 (psi) cells, with Fig. 3 / Fig. 4 read as data: 48 one-triangle
  graphs must land in exactly the tabulated type.
- Hand-worked Def. 1 / Fig. 2 cases (tests/golden/hand_cases.txt).
- O1 (Lemma 1 summed directly) against O0 (every edge triple) on random tiny
  multigraphs with many timestamp ties.
- Unbounded windows: the total is the sum over static triangles of the product
  of the three multiplicities; per type, an independent route through Table 1
  counts the 3-patterns of each triangle's merged, key-sorted edge sequence.
- delta = 0, monotonicity in each delta component, invariance under vertex
  relabelling and time shift, and the type permutations that edge reversal and
  time reversal induce (derived from Fig. 2).
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2106_02762_gb300 import synth
from tests.golden import readers

BIG = 1 << 40


def _arr(edges):
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 3)
    return e[:, 0].astype(np.uint32), e[:, 1].astype(np.uint32), e[:, 2].astype(np.int64)


# ---------------------------------------------------------------- Table 1
def _psi_graph(order, orient, ids):
    """One edge per pair of triangle {u, v, w}: directed as in the
    orientation, at t = 1, 2, 3 in the order's sequence."""
    name = dict(zip("uvw", ids))
    t_of = {frozenset(p): i + 1 for i, p in enumerate(order)}
    edges = []
    for e in orient:
        edges.append((name[e[0]], name[e[1]], t_of[frozenset(e)]))
    return edges


@pytest.mark.parametrize("ids", [(0, 1, 2), (9, 4, 6), (100, 3, 50)])
def test_psi_table_cells(ids):
    orders, orients, psi = readers.psi_table()
    assert len(orders) == 6 and len(orients) == 8
    for k in range(1, 7):
        for r in range(1, 9):
            s, d, t = _arr(_psi_graph(orders[k], orients[r], ids))
            exp = np.zeros(8, dtype=np.uint64)
            exp[psi[k][r] - 1] = 1
            got0 = oracle.bruteforce(s, d, t, [(BIG, BIG, BIG)])[0]
            got1 = oracle.count(s, d, t, [(BIG, BIG, BIG)])[0]
            assert (got0 == exp).all(), (k, r, got0)
            assert (got1 == exp).all(), (k, r, got1)


def test_psi_table_is_consistent():
    """Each of the six orders maps the eight orientations onto the eight types
    one-to-one (a property of Table 1 itself, checked so a mistyped fixture
    cannot slip through)."""
    _, _, psi = readers.psi_table()
    for k in range(1, 7):
        assert sorted(psi[k].values()) == list(range(1, 9))


# ---------------------------------------------------------------- hand cases
@pytest.mark.parametrize("case", readers.hand_cases(), ids=lambda c: c[0])
def test_hand_cases(case):
    name, edges, checks = case
    s, d, t = _arr(edges)
    deltas = [c[0] for c in checks]
    exp = np.asarray([c[1] for c in checks], dtype=np.uint64)
    assert (oracle.bruteforce(s, d, t, deltas) == exp).all()
    assert (oracle.count(s, d, t, deltas) == exp).all()


# ---------------------------------------------------------------- O1 vs O0
def _delta_menu(rng, t_range):
    base = [(0, 0, 0), (BIG, BIG, BIG), (1, 1, 1), (t_range, 0, t_range), (0, t_range, t_range)]
    for _ in range(6):
        base.append(tuple(int(x) for x in rng.integers(0, t_range + 2, size=3)))
    return base


def test_o1_matches_bruteforce_random_tiny():
    rng = np.random.default_rng(7)
    for seed in range(400):
        n = int(rng.integers(3, 9))
        m = int(rng.integers(3, 41))
        tr = int(rng.integers(1, 25))
        s, d, t = synth.random_tiny(seed, n, m, tr)
        deltas = _delta_menu(rng, tr)
        a = oracle.bruteforce(s, d, t, deltas)
        b = oracle.count(s, d, t, deltas, threads=1)
        assert (a == b).all(), (seed, deltas)


def test_o1_threads_agree():
    s, d, t = synth.er_temporal(3, 60, 400, 2000, 3.0)
    deltas = [(300, 200, 200), (BIG, BIG, BIG)]
    assert (oracle.count(s, d, t, deltas, threads=1) == oracle.count(s, d, t, deltas, threads=4)).all()


# ---------------------------------------------------------------- unbounded windows
def _static_triangles(s, d):
    """Static triangles by plain set lookups (tiny graphs)."""
    adj = {}
    for a, b in zip(s.tolist(), d.tolist()):
        if a == b:
            continue
        adj.setdefault(a, set()).add(b)
        adj.setdefault(b, set()).add(a)
    tris = []
    for a in sorted(adj):
        for b in sorted(x for x in adj[a] if x > a):
            for c in sorted(x for x in adj[a] & adj[b] if x > b):
                tris.append((a, b, c))
    return tris


def test_unbounded_total_is_product_of_multiplicities():
    for seed in range(40):
        s, d, t = synth.random_tiny(1000 + seed, 7, 40, 6)
        total = int(oracle.count(s, d, t, [(BIG, BIG, BIG)]).sum())
        key = {}
        for a, b in zip(s.tolist(), d.tolist()):
            if a != b:
                key[frozenset((a, b))] = key.get(frozenset((a, b)), 0) + 1
        prod = sum(key[frozenset((a, b))] * key[frozenset((a, c))] * key[frozenset((b, c))]
                   for a, b, c in _static_triangles(s, d))
        assert total == prod
        assert oracle.stats(s, d, t)["prod"] == prod


def test_unbounded_per_type_via_table1():
    """Per type at unbounded windows, by an independent route: for each static
    triangle {u, v, w} (u < v < w), walk its merged key-sorted edge sequence;
    every middle edge y combines each earlier edge x and later edge z on the
    two other pairs.  The order of the three pairs names pi, the three
    directions name rho, and Table 1 gives the type."""
    orders, orients, psi = readers.psi_table()
    order_of = {tuple(v): k for k, v in orders.items()}
    orient_of = {frozenset(v): k for k, v in orients.items()}
    for seed in range(40):
        s, d, t = synth.random_tiny(2000 + seed, 6, 36, 5)
        want = np.zeros(8, dtype=np.int64)
        for tri in _static_triangles(s, d):
            name = dict(zip(tri, "uvw"))
            seq = []
            for i, (a, b, tt) in enumerate(zip(s.tolist(), d.tolist(), t.tolist())):
                if a in name and b in name and a != b:
                    seq.append((tt, i, name[a] + name[b]))
            seq.sort()
            pair = lambda e: "".join(sorted(e))
            for j, (_, _, ey) in enumerate(seq):
                for ex in (x[2] for x in seq[:j]):
                    for ez in (z[2] for z in seq[j + 1:]):
                        pairs = (pair(ex), pair(ey), pair(ez))
                        if len(set(pairs)) < 3:
                            continue
                        k = order_of[pairs]
                        r = orient_of[frozenset((ex, ey, ez))]
                        want[psi[k][r] - 1] += 1
        got = oracle.count(s, d, t, [(BIG, BIG, BIG)])[0].astype(np.int64)
        assert (got == want).all(), seed


# ---------------------------------------------------------------- delta edge cases
def test_delta_zero():
    s, d, t = synth.er_temporal(11, 30, 150, 10 ** 6, 3.0)
    # distinct timestamps: nothing fits a zero window
    t = np.arange(s.size, dtype=np.int64) * 7 + 3
    assert oracle.count(s, d, t, [(0, 0, 0)]).sum() == 0
    # all timestamps equal: every triangle triple counts once
    t0 = np.full(s.size, 42, dtype=np.int64)
    assert int(oracle.count(s, d, t0, [(0, 0, 0)]).sum()) == oracle.stats(s, d, t0)["prod"]


def test_monotone_in_each_delta():
    s, d, t = synth.er_temporal(12, 40, 250, 5000, 3.0)
    rng = np.random.default_rng(3)
    for _ in range(10):
        base = tuple(int(x) for x in rng.integers(0, 3000, size=3))
        lo = oracle.count(s, d, t, [base])[0]
        for c in range(3):
            up = list(base)
            up[c] += int(rng.integers(1, 800))
            hi = oracle.count(s, d, t, [tuple(up)])[0]
            assert (hi >= lo).all()


def test_relabel_and_time_shift_invariance():
    s, d, t = synth.er_temporal(13, 50, 300, 4000, 3.0)
    deltas = [(1500, 700, 900), (4000, 4000, 10), (BIG, BIG, BIG)]
    base = oracle.count(s, d, t, deltas)
    perm = np.random.default_rng(5).permutation(10 ** 6)[:50].astype(np.uint32)
    assert (oracle.count(perm[s], perm[d], t, deltas) == base).all()
    assert (oracle.count(s, d, t - (1 << 61), deltas) == base).all()
    assert (oracle.count(s, d, t + (1 << 61), deltas) == base).all()


def test_edge_reversal_permutes_types():
    """Reversing every edge maps T1<->T5, T2<->T7, T3<->T6, T4<->T8 (Fig. 2)."""
    s, d, t = synth.er_temporal(14, 40, 250, 3000, 3.0)
    deltas = [(1500, 700, 900), (BIG, BIG, BIG), (900, 900, 100)]
    a = oracle.count(s, d, t, deltas)
    b = oracle.count(d, s, t, deltas)
    perm = [4, 6, 5, 7, 0, 2, 1, 3]
    assert (b == a[:, perm]).all()


def test_time_reversal_permutes_types():
    """t -> -t with the edge order reversed (so ties flip too) and d12 <-> d23
    maps T1<->T3, T2<->T7, T5<->T6, T4<->T8 (Fig. 2)."""
    s, d, t = synth.er_temporal(15, 40, 250, 200, 3.0)  # many ties
    deltas = [(150, 70, 90), (BIG, BIG, BIG), (90, 10, 90), (0, 0, 0)]
    a = oracle.count(s, d, t, deltas)
    rev = [(d13, d23, d12) for d13, d12, d23 in deltas]
    b = oracle.count(s[::-1], d[::-1], -t[::-1], rev)
    perm = [2, 6, 0, 7, 5, 4, 1, 3]
    assert (b == a[:, perm]).all()


def test_extreme_timestamps():
    # a T1 spanning 2^62 exactly: the largest window the interface allows
    s, d, t = _arr([(0, 1, -(1 << 61)), (2, 1, 0), (0, 2, 1 << 61)])
    lim = 1 << 62
    assert list(oracle.count(s, d, t, [(lim, lim, lim)])[0]) == [1] + [0] * 7
    assert list(oracle.count(s, d, t, [(lim - 1, lim, lim)])[0]) == [0] * 8
    assert list(oracle.count(s, d, t, [(lim, (1 << 61) - 1, lim)])[0]) == [0] * 8


def test_empty_and_degenerate_inputs():
    e = np.zeros(0, dtype=np.uint32)
    assert oracle.count(e, e, np.zeros(0, dtype=np.int64), [(1, 1, 1)]).sum() == 0
    s, d, t = _arr([(3, 3, 1), (4, 4, 2), (3, 3, 3)])  # self-loops only
    assert oracle.count(s, d, t, [(BIG, BIG, BIG)]).sum() == 0
    assert oracle.stats(s, d, t)["m"] == 0


def test_per_triangle_counts_sum_to_total():
    s, d, t = synth.er_temporal(16, 40, 300, 3000, 3.0)
    deltas = [(1500, 700, 900), (BIG, BIG, BIG)]
    tris = _static_triangles(s, d)
    per = oracle.count_triangles(s, d, t, tris, deltas)
    assert (per.sum(axis=0) == oracle.count(s, d, t, deltas)).all()
    # a non-triangle triple gives zeros
    assert oracle.count_triangles(s, d, t, [(0, 0, 1)], deltas).sum() == 0


def test_stats_against_networkx():
    nx = pytest.importorskip("networkx")
    s, d, t = synth.er_temporal(17, 80, 600, 3000, 3.0)
    g = nx.Graph()
    g.add_edges_from(zip(s.tolist(), d.tolist()))
    st = oracle.stats(s, d, t)
    assert st["tau"] == sum(nx.triangles(g).values()) // 3
    assert st["m_s"] == g.number_of_edges()
    assert st["m"] == s.size


def test_stats_hand_case():
    # pairs {0,1} x2, {0,2} x3, {1,2} x1, {2,3} x1, {1,3} x4 (directions mixed):
    # static triangles {0,1,2} (multiplicities 2, 3, 1) and {1,2,3} (1, 1, 4), so
    # work_bytes = (8 (2+3+1) + 12) + (8 (1+1+4) + 12) = 120 and the unbounded
    # total (Def. 1 with every window open) = 2*3*1 + 1*1*4 = 10
    edges = [(0, 1, 5), (1, 0, 9), (0, 2, 1), (2, 0, 2), (0, 2, 3), (1, 2, 7),
             (3, 2, 4), (1, 3, 6), (3, 1, 8), (1, 3, 10), (3, 1, 11)]
    s, d, t = _arr(edges)
    for st in (oracle.stats(s, d, t), oracle.stats_fwd(s, d, t)):
        assert st == {"n": 4, "m": 11, "m_s": 5, "tau": 2, "sigma_max": 4, "work_bytes": 120, "prod": 10}
    assert int(oracle.count(s, d, t, [(BIG, BIG, BIG)]).sum()) == 10


def test_forward_rule_matches_plain_rule():
    # the forward enumeration must visit the same triangles: identical
    # statistics and identical counts, on uniform and on hub-heavy graphs
    deltas = [(1500, 700, 900), (BIG, BIG, BIG), (0, 0, 0), (3000, 3000, 100)]
    graphs = [synth.er_temporal(31, 60, 500, 3000, 3.0), synth.large_plain(scale=0.002)]
    graphs += [synth.random_tiny(40 + i, n=7, m=30, t_range=6) for i in range(20)]
    for s, d, t in graphs:
        assert oracle.stats_fwd(s, d, t) == oracle.stats(s, d, t)
        assert (oracle.count_fwd(s, d, t, deltas) == oracle.count(s, d, t, deltas)).all()
        assert (oracle.count_fwd(s, d, t, deltas, strict=True) == oracle.count(s, d, t, deltas, strict=True)).all()


def test_full_size_golden_counts_are_consistent():
    # the stored full-size counts: unbounded total = sum of s_uv s_uw s_vw,
    # and monotone in the windows (the wide finite triple lies between)
    fields, rows = readers.power_law_counts()
    by = {d: np.asarray(c, dtype=np.uint64) for d, c in rows}
    unb = by[synth.LARGE_PLAIN_DELTA_UNBOUNDED]
    assert int(unb.sum()) == fields["prod"]
    for d, c in by.items():
        assert (c <= unb).all()
    assert (by[synth.LARGE_PLAIN_DELTA] <= by[(1 << 26, 1 << 25, 1 << 25)]).all()


def test_parts_partition_the_count():
    s, d, t = synth.er_temporal(18, 60, 400, 3000, 3.0)
    deltas = [(1500, 700, 900), (BIG, BIG, BIG)]
    total = oracle.count(s, d, t, deltas)
    parts = sum(oracle.count_part(s, d, t, deltas, p, 5) for p in range(5))
    assert (parts == total).all()


# --------------------------------------------------------------------------
# strict variant: Def. 1's t1 < t2 < t3 read literally
# --------------------------------------------------------------------------
def test_strict_o1_matches_strict_bruteforce():
    # O0 drops a key-ordered triple unless its timestamps strictly increase;
    # O1 starts each later role after the earlier edge's time instead of its
    # key.  Tiny graphs with timestamps in [0, 6) tie often.
    ds = [(5, 3, 3), (0, 0, 0), (2, 1, 2), (BIG, BIG, BIG), (4, 0, 4)]
    for seed in range(40):
        s, d, t = synth.random_tiny(100 + seed, 6, 30, 6)
        assert (oracle.count(s, d, t, ds, strict=True) == oracle.bruteforce(s, d, t, ds, strict=True)).all(), seed


def test_strict_equals_key_order_without_ties():
    ds = [(5, 3, 3), (BIG, BIG, BIG)]
    for seed in range(10):
        s, d, _ = synth.random_tiny(200 + seed, 7, 40, 6)
        t = np.random.default_rng(seed).permutation(s.size).astype(np.int64)  # all distinct
        assert (oracle.count(s, d, t, ds, strict=True) == oracle.count(s, d, t, ds)).all()


def test_strict_counts_nothing_when_all_times_are_equal():
    s, d, _ = synth.random_tiny(7, 6, 40, 6)
    t = np.zeros(s.size, dtype=np.int64)
    assert oracle.count(s, d, t, [(BIG, BIG, BIG)], strict=True).sum() == 0
    # key order counts every triple on a triangle exactly once instead
    assert oracle.count(s, d, t, [(BIG, BIG, BIG)]).sum() == oracle.stats(s, d, t)["prod"]


def test_strict_hand_case():
    # the first hand case of Def. 1 (T1 at delta = (20, 10, 10)) with its
    # last edge moved onto the second edge's time: key order still counts it
    # (the input index breaks the tie), the strict reading does not; one
    # second later both count it
    s, d, t = _arr([(0, 1, 0), (2, 1, 10), (0, 2, 10)])
    q = [(20, 10, 10)]
    assert oracle.count(s, d, t, q).sum() == 1
    assert oracle.count(s, d, t, q, strict=True).sum() == 0
    s, d, t = _arr([(0, 1, 0), (2, 1, 10), (0, 2, 11)])
    q = [(20, 10, 10)]
    assert (oracle.count(s, d, t, q, strict=True) == oracle.count(s, d, t, q)).all()
    assert oracle.count(s, d, t, q, strict=True).sum() == 1
