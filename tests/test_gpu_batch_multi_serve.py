"""Batched, many-graph and served entry points against the oracle and
against the plain single-query path (bit for bit)."""
import time

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


def _small_graphs(count=6, seed=7):
    n, pairs, deltas, seeds = synth.many_graph_specs(seed=seed, count=count, n_lo=200, n_hi=3000)
    out = []
    for i in range(count):
        s, d, t = synth.many_graph(n[i], pairs[i], seeds[i])
        out.append((s, d, t, tuple(int(x) for x in deltas[i])))
    return out


def _heavy_triangle_graph():
    # three pairs of 1500 edges each (a huge prefix-sum triangle) plus a light fringe
    rng = np.random.default_rng(3)
    k = 1500
    s = np.concatenate([np.zeros(k), np.ones(k), np.zeros(k), rng.integers(0, 3, 300)]).astype(np.uint32)
    d = np.concatenate([np.ones(k), np.full(k, 2), np.full(k, 2), rng.integers(3, 40, 300)]).astype(np.uint32)
    flip = rng.integers(0, 2, s.size).astype(bool)
    s, d = np.where(flip, d, s), np.where(flip, s, d)
    t = rng.integers(0, 20000, s.size).astype(np.int64)
    return s, d, t


def test_count_multi_matches_oracle_and_replays():
    gs = _small_graphs()
    gs.append(_heavy_triangle_graph() + ((2000, 900, 1500),))
    handles = [ttc.Graph(s, d, t) for s, d, t, _ in gs]
    handles.append(ttc.Graph(*gs[0][:3], light_max_pairs=1))  # every triangle on the prefix-sum path
    gs.append(gs[0])
    deltas = [q for *_, q in gs]
    want = np.stack([oracle.count(s, d, t, [q])[0] for s, d, t, q in gs])
    assert handles[-2].info()["tau_huge"] >= 1
    got1 = ttc.count_multi(handles, deltas)
    got2 = ttc.count_multi(handles, deltas)  # replay of the captured graph
    assert (got1 == want).all()
    assert (got2 == want).all()
    # new deltas on the same plan
    deltas2 = [(BIG, BIG, BIG)] * len(handles)
    want2 = np.stack([oracle.count(s, d, t, [q])[0] for (s, d, t, _), q in zip(gs, deltas2)])
    assert (ttc.count_multi(handles, deltas2) == want2).all()
    # another order is another plan; a freed graph drops its plans
    order = list(reversed(range(len(handles))))
    assert (ttc.count_multi([handles[i] for i in order], [deltas[i] for i in order]) == want[order]).all()
    handles[0].free()
    rest = handles[1:]
    assert (ttc.count_multi(rest, deltas[1:]) == want[1:]).all()
    for h in rest:
        h.free()


def test_batched_flat_path_in_passes(monkeypatch):
    # a batch on a graph whose heavy triangles take the flat path, with the
    # pass cap of that path set so that a pass takes one query, two queries,
    # or all of them: every split equals the oracle
    s, d, t = _heavy_triangle_graph()
    g = ttc.Graph(s, d, t, light_max_pairs=1)  # every triangle on the prefix-sum path
    assert g.info()["tau_huge"] >= 1
    deltas = [(BIG, BIG, BIG), (2000, 900, 1500), (500, 300, 400), (3000, 3000, 0), (0, 0, 0), (9000, 100, 8900),
              (1200, 1200, 1200)]
    want = oracle.count(s, d, t, deltas)
    for cap in ("1", "200000", None):  # about 96 KB of prefix entries a query here
        if cap is None:
            monkeypatch.delenv("TTC_HUGE_PASS_BYTES", raising=False)
        else:
            monkeypatch.setenv("TTC_HUGE_PASS_BYTES", cap)
        assert (g.count_batch(deltas) == want).all(), cap
    g.free()


def test_count_stream_batches_within_budget():
    # the streaming many-graph count: graphs loaded from host arrays in
    # order, counted batch by batch under a device-memory budget; results
    # equal the oracle's whatever the batching
    gs = _small_graphs() + [_heavy_triangle_graph() + ((2000, 900, 1500),)]
    edges = [(s, d, t) for s, d, t, _ in gs]
    deltas = [q for *_, q in gs]
    want = np.stack([oracle.count(s, d, t, [q])[0] for s, d, t, q in gs])
    one = [ttc.Graph(*e) for e in edges]
    sizes = [g.info()["device_bytes"] for g in one]
    for g in one:
        g.free()
    got, nb = ttc.count_stream(edges, deltas)  # half the free memory: one batch
    assert (got == want).all() and nb == 1
    budget = max(sizes)  # the largest alone, the others a few a batch
    got, nb = ttc.count_stream(edges, deltas, budget_bytes=budget)
    assert (got == want).all()
    # the batches follow the rule: a graph joins while the batch stays within
    # the budget
    expect, run = 1, 0
    for b in sizes:
        if run and run + b > budget:
            expect, run = expect + 1, 0
        run += b
    assert nb == expect > 1
    got, nb = ttc.count_stream(edges, deltas, budget_bytes=1)  # one graph a batch
    assert (got == want).all() and nb == len(edges)
    got, nb = ttc.count_stream(edges, deltas, budget_bytes=1, light_max_pairs=1)  # every triangle heavy
    assert (got == want).all()
    with pytest.raises(ValueError):
        ttc.count_stream(edges, deltas[:-1])


def test_count_stream_retries_a_load_after_freeing_the_batch():
    # A load that runs out of device memory while a batch is resident is
    # tried again once that batch is counted and freed.  The injected failure
    # (the n-th device allocation of the call) lands in turn in the first
    # graph's load (an error: no batch to free), a later graph's load (the
    # retry: one batch more, same counts) and the count (an error); every
    # outcome leaves no device memory behind.
    import torch
    gs = _small_graphs(count=3)
    edges = [(s, d, t) for s, d, t, _ in gs]
    deltas = [q for *_, q in gs]
    want = np.stack([oracle.count(s, d, t, [q])[0] for s, d, t, q in gs])
    got, nb = ttc.count_stream(edges, deltas)
    assert (got == want).all() and nb == 1
    torch.cuda.synchronize()
    used0 = ttc.memory_info()["pool_used"]
    outcomes = set()
    for n in range(1, 5000):
        ttc.debug_fail_alloc_after(n)
        try:
            got, nb = ttc.count_stream(edges, deltas)
            outcomes.add(nb)
            assert (got == want).all()
        except ttc.TTCError as e:
            assert e.status == -3
            outcomes.add("error")
        finally:
            ttc.debug_fail_alloc_after(0)
        torch.cuda.synchronize()
        assert ttc.memory_info()["pool_used"] == used0, n
        if 1 in outcomes:  # n is past the call's last allocation
            break
    assert outcomes == {"error", 1, 2}


@pytest.mark.slow
def test_many_graph_workload_sample_matches_oracle():
    # a seeded sample of 64 of the 4096 graphs of the many-graphs workload
    # (every 64th spec: n log-uniform in [1e3, 1e5], average degree U[4, 32],
    # Chung-Lu 2.3, Geometric(0.3) multiplicities, own delta per graph), in
    # one many-graph launch, against the oracle graph by graph
    n, pairs, deltas, seeds = synth.many_graph_specs()
    pick = np.arange(0, n.size, 64)
    gs = [synth.many_graph(n[i], pairs[i], seeds[i]) for i in pick]
    dl = [tuple(int(x) for x in deltas[i]) for i in pick]
    handles = [ttc.Graph(*e) for e in gs]
    got = ttc.count_multi(handles, dl)
    want = np.stack([oracle.count_fwd(*e, [q])[0] for e, q in zip(gs, dl)])
    assert (got == want).all()
    assert (want.sum(axis=1) > 0).sum() >= 32
    for h in handles:
        h.free()


def test_count_multi_equals_plain_calls():
    gs = _small_graphs(count=12, seed=11)
    handles = [ttc.Graph(s, d, t) for s, d, t, _ in gs]
    deltas = [q for *_, q in gs]
    multi = ttc.count_multi(handles, deltas)
    plain = np.stack([h.count(q) for h, q in zip(handles, deltas)])
    assert (multi == plain).all()
    for h in handles:
        h.free()


def test_batch_equals_sequential_on_heavy_graph():
    s, d, t = _heavy_triangle_graph()
    g = ttc.Graph(s, d, t)
    deltas = synth.delta_sweep(16, 10, 30000)
    want = oracle.count(s, d, t, deltas)
    assert (g.count_batch(deltas) == want).all()
    assert (np.stack([g.count(q) for q in deltas]) == want).all()
    g.free()


def test_server_results_equal_alone_runs():
    graphs = [synth.served_graph(m, 100 + j) for j, m in enumerate((20_000, 60_000, 150_000))]
    alone = [ttc.Graph(*gr) for gr in graphs]
    srv = ttc.Server(streams=3, max_batch=64)
    ids = [srv.load(*gr) for gr in graphs]
    rng = np.random.default_rng(9)
    menu = [tuple(int(x) for x in synth.log_uniform_int(rng, 60, 2.6e6, size=3)) for _ in range(40)]
    tickets = []
    for i in range(600):
        j = int(rng.integers(0, len(ids)))
        q = menu[int(rng.integers(0, len(menu)))]
        tickets.append((srv.submit(ids[j], q), j, q))
        if i % 50 == 0:
            time.sleep(0.001)  # arrivals while earlier batches are on the device
    srv.drain(60.0)
    expected = {}
    for tk, j, q in tickets:
        if (j, q) not in expected:
            expected[(j, q)] = alone[j].count(q)
        res = srv.poll(tk)
        assert res is not None
        counts, lat = res
        assert (counts == expected[(j, q)]).all()
        assert lat >= 0
    info = srv.info()
    assert info["completed"] == info["submitted"] == 600
    assert info["launches"] < 600  # queries were batched
    # a handful against the oracle directly
    for (j, q), want in list(expected.items())[:3]:
        assert (oracle.count(*graphs[j], [q])[0] == want).all()
    with pytest.raises(ttc.TTCError, match="NOT_FOUND"):
        srv.submit(12345, (1, 1, 1))
    with pytest.raises(ttc.TTCError, match="NOT_FOUND"):
        srv.poll(tickets[0][0])  # already collected
    srv.close()
    for g in alone:
        g.free()


def test_server_queue_limit_and_eviction():
    import torch
    gr1 = synth.served_graph(20_000, 1)
    gr2 = synth.served_graph(20_000, 2)
    srv = ttc.Server(streams=1, max_queue=4)
    gid = srv.load(*gr1)
    srv.pause(True)
    tks = [srv.submit(gid, (100, 50, 50)) for _ in range(4)]
    with pytest.raises(ttc.TTCError, match="BUSY"):
        srv.submit(gid, (100, 50, 50))
    assert srv.poll(tks[0]) is None  # still queued
    with pytest.raises(ttc.TTCError, match="TIMEOUT"):
        srv.drain(0.05)
    srv.pause(False)
    srv.drain(30.0)
    want = oracle.count(*gr1, [(100, 50, 50)])[0]
    for tk in tks:
        assert (srv.poll(tk)[0] == want).all()
    srv.close()
    # admission: once g1 is resident, keep all but slightly less than g2's
    # load estimate free, so loading g2 must evict the idle g1 first
    srv = ttc.Server()
    g1 = srv.load(*gr1)
    torch.cuda.synchronize()
    ttc.release_cached()
    free = ttc.memory_info()["admission_free"]  # device free + the pool's cached blocks
    estimate = 96 * gr2[0].size + (64 << 20)
    srv.set_reserve(max(0, free - estimate + 4096))
    g2 = srv.load(*gr2)
    info = srv.info()
    assert info["evictions"] == 1 and info["graphs_resident"] == 1 and info["admissions"] == 2
    with pytest.raises(ttc.TTCError, match="NOT_FOUND"):
        srv.submit(g1, (1, 1, 1))
    tk = srv.submit(g2, (100_000, 50_000, 50_000))
    srv.drain(30.0)
    counts, _ = srv.poll(tk)
    assert (counts == oracle.count(*gr2, [(100_000, 50_000, 50_000)])[0]).all()
    # a load that evicting every idle graph could not make room for is
    # refused, and nothing is evicted for it
    srv.set_reserve(1 << 62)
    with pytest.raises(ttc.TTCError, match="NOMEM"):
        srv.load(*gr1)
    info = srv.info()
    assert info["evictions"] == 1 and info["graphs_resident"] == 1
    srv.close()


def test_delta_grid_matches_oracle():
    s, d, t = synth.tiny_plain()
    g = ttc.Graph(s, d, t)
    d13 = 7200
    d12 = [0, 600, 1800, 3600, 7200]
    d23 = [300, 1800, 5400, 9000]
    counts, cyc = g.count_grid(d13, d12, d23)
    want = oracle.count(s, d, t, [(d13, a, b) for a in d12 for b in d23]).reshape(len(d12), len(d23), 8)
    assert (counts == want).all()
    tot = want.sum(axis=2).astype(np.float64)
    share = np.where(tot > 0, (want[:, :, 3] + want[:, :, 7]) / np.maximum(tot, 1), 0.0)
    assert np.allclose(cyc, share, rtol=0, atol=1e-12)
    assert (counts == np.stack([g.count_batch([(d13, a, b) for b in d23]) for a in d12])).all()
    g.free()


def _one_triangle(n_a, n_b, n_c, a_before_b=None, seed=11):
    # u = 0, v = 1, w = 2: A = {0, 1}, B = {0, 2} and the heaviest pair
    # C = {1, 2}, every edge directed the same way; A's and B's edges take
    # the times 0 .. n_a + n_b - 1 (A's all first, B's all first, or mixed),
    # C's edges come after all of them
    rng = np.random.default_rng(seed)
    if a_before_b is None:
        ab = rng.permutation(n_a + n_b)
    else:
        ab = np.arange(n_a + n_b) if a_before_b else np.concatenate([np.arange(n_b, n_a + n_b), np.arange(n_b)])
    s = np.concatenate([np.zeros(n_a), np.zeros(n_b), np.ones(n_c)]).astype(np.uint32)
    d = np.concatenate([np.ones(n_a), np.full(n_b, 2), np.full(n_c, 2)]).astype(np.uint32)
    t = np.concatenate([ab, 10**6 + np.arange(n_c)]).astype(np.int64)
    return s, d, t


def test_batched_light_counts_past_32_bits():
    # one light triangle with 1023 x 1024 enumerated pairs and 150000 edges
    # on C: each lane of the batched light path takes 32736 pairs, and with
    # every window unbounded each pair puts all of C's edges in one type, so
    # a lane's 32-bit accumulator carries past 2^32 several times
    unb = synth.LARGE_PLAIN_DELTA_UNBOUNDED
    # the type of "A's edge, then B's edge, then C's" and of "B, A, C" on
    # this layout, from the oracle on small copies of it
    t_ab = int(np.flatnonzero(oracle.count(*_one_triangle(2, 2, 3, True), [unb])[0])[0])
    t_ba = int(np.flatnonzero(oracle.count(*_one_triangle(2, 2, 3, False), [unb])[0])[0])
    assert t_ab != t_ba
    n_a, n_b, n_c = 1023, 1024, 150000
    s, d, t = _one_triangle(n_a, n_b, n_c)
    g = ttc.Graph(s, d, t, light_max_pairs=1 << 20)
    assert g.info()["tau_light"] == 1
    # pairs (a, b) with a earlier: for each b, the A edges before it
    ta, tb = np.sort(t[:n_a]), t[n_a:n_a + n_b]
    n_ab = int(np.searchsorted(ta, tb).sum())
    want = np.zeros(8, np.uint64)
    want[t_ab] = n_ab * n_c
    want[t_ba] = (n_a * n_b - n_ab) * n_c
    assert int(want.sum()) == n_a * n_b * n_c
    assert (g.count(unb) == want).all()
    assert (g.count_batch([unb, unb]) == np.stack([want, want])).all()
    g.free()
