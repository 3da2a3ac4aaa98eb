#!/usr/bin/env python
"""Benchmark: exact temporal triangle counting on the power-law workload.

One step = the whole hot path on one synthetic graph whose edge arrays are
already resident in device memory: ttc_load (ingest, pair lists, k-core peel,
orientation, triangle list) followed by one ttc_count_batch of the
configured delta and the same delta with every window unbounded (so no
window lets a kernel skip work).  The metric is temporal edges per second
per step; on N GPUs every rank loads the graph and counts its shard of the
triangles, and the counts are summed.

Workload (default): Chung-Lu power-law skeleton, n = 1M vertices, 10M vertex
pairs, degree exponent 2.1, multiplicity pmf k^-2 on [1, 1e4] (about 60M
edges), lognormal(6, 2) inter-arrival times over a 2^31 s span; delta =
(86400, 43200, 43200).  The edge arrays (~1 GB) and the resident graph exceed
the 129 MB L2, so no flush is needed between steps.

Beside the step the line carries per-kernel times of the configured, the
unbounded and the batched queries, the roofline of the unbounded light
kernel, the tuned light threshold, the 64-delta sweep, and (unless
--no-extras) the many-graphs and served measurements.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle
instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "temporal edges/s per delta-query"
UNIT = "edges/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--scale", type=float, default=1.0, help="workload scale (1.0 = the full workload)")
    ap.add_argument("--query-iters", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", choices=["plain", "multi", "serve", "grid", "zipf15"], default="plain",
                    help="plain: the power-law workload (default line); multi: many graphs in one launch; "
                         "serve: Poisson queries against a resident pool; grid: a delta grid; zipf15: the "
                         "power-law workload with multiplicity exponent 1.5 (about 766M edges)")
    ap.add_argument("--graphs", type=int, default=4096, help="multi: number of graphs")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve: query arrivals per second")
    ap.add_argument("--duration", type=float, default=20.0, help="serve: seconds of arrivals")
    ap.add_argument("--load-rate", type=float, default=1.0, help="serve: new-graph loads per second")
    ap.add_argument("--multi-graphs", type=int, default=512,
                    help="default line: graphs of the many-graphs workload measured beside the step")
    ap.add_argument("--serve-seconds", type=float, default=4.0,
                    help="default line: seconds of arrivals per rate in the served measurement")
    ap.add_argument("--no-extras", action="store_true",
                    help="default line: skip the many-graphs and served measurements")
    return ap.parse_args()


def workload_name(scale):
    return "power-law n=%d pairs=%d gamma=2.1 zipf2-cap1e4 lognormal(6,2) span 2^31" % (
        int(round(1_000_000 * scale)), int(round(10_000_000 * scale)))


def workload(scale):
    from paper_2106_02762_gb300 import synth
    src, dst, t = synth.large_plain(scale=scale)
    return src, dst, t, synth.LARGE_PLAIN_DELTA, workload_name(scale)


# ------------------------------------------------------------------ clocks
class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], 0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ distributed
def dist_setup(backend):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, ws, device=None):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ CPU oracle timing
SAMPLE_SCALE = 0.1


def step_queries(delta):
    """The queries one timed step answers: the configured one and the same
    with every window unbounded."""
    from paper_2106_02762_gb300 import synth
    return [tuple(delta), synth.LARGE_PLAIN_DELTA_UNBOUNDED]


def oracle_sample(delta, reps=3):
    """Times the oracle (O1, every host core) on a bounded sample of the
    workload: the same recipe at 10% scale (100K vertices, 1M pairs, about
    6M edges), whole graph, `reps` runs of the step's two queries (about
    10 to 30 s of host work).  Returns
    (edges/s, description, cores, seconds per run)."""
    import oracle
    from paper_2106_02762_gb300 import synth
    oracle.build()
    src, dst, t = synth.large_plain(scale=SAMPLE_SCALE)
    m = int((src != dst).sum())
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.count(src, dst, t, step_queries(delta))
        times.append(time.perf_counter() - t0)
    sec = statistics.median(times)
    desc = ("O1 answering the step's two queries on the whole power-law recipe at %g scale (%d vertices, "
            "%d pairs, %d edges), median of %d runs; the per-edge cost grows with scale (hub degrees), so the "
            "full-size oracle is slower per edge"
            % (SAMPLE_SCALE, int(1e6 * SAMPLE_SCALE), int(1e7 * SAMPLE_SCALE), m, reps))
    return m / sec, desc, os.cpu_count() or 1, sec


def run_reference(args):
    ws, rank, _ = dist_setup("gloo")
    if rank != 0:
        barrier(ws)
        return
    import oracle
    from paper_2106_02762_gb300 import synth
    oracle.build()
    delta = synth.LARGE_PLAIN_DELTA
    name = workload_name(args.scale)
    src, dst, t = synth.large_plain(scale=SAMPLE_SCALE)
    m = int((src != dst).sum())
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.count(src, dst, t, step_queries(delta))
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    step_s = statistics.median(times)
    value = m / step_s
    desc = ("O1 (plain adjacency + Lemma 1, every host core) answering the step's two queries on the whole "
            "power-law recipe at %g scale (%d edges) per step" % (SAMPLE_SCALE, m))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": name, "delta": list(delta), "step_deltas": [list(q) for q in step_queries(delta)],
                   "sample_m": m},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    barrier(ws)


# ------------------------------------------------------------------ batched sweep
def batched_sweep(ttc, torch, reps=20):
    """64 delta-triples on the tiny-plain graph: one ttc_count_batch call
    against 64 sequential ttc_count calls (queries per second each)."""
    from paper_2106_02762_gb300 import synth
    s, d, t = synth.tiny_plain()
    deltas = synth.delta_sweep()
    g = ttc.Graph(s, d, t)
    ref = g.count_batch(deltas)
    seq_t, bat_t = [], []
    for _ in range(reps):
        w = time.perf_counter()
        seq = [g.count(q) for q in deltas]
        seq_t.append(time.perf_counter() - w)
        w = time.perf_counter()
        b = g.count_batch(deltas)
        bat_t.append(time.perf_counter() - w)
    assert (np.stack(seq) == ref).all() and (b == ref).all()
    g.free()
    seq_s, bat_s = statistics.median(seq_t), statistics.median(bat_t)
    return {"workload": "tiny plain graph (n=1000, 5000 pairs), 64 delta-triples log-spaced 60 s..30 d",
            "batch_queries_per_s": len(deltas) / bat_s, "sequential_queries_per_s": len(deltas) / seq_s,
            "speedup": seq_s / bat_s, "batch_ms": bat_s * 1e3, "sequential_ms": seq_s * 1e3}


# ------------------------------------------------------------------ many graphs
def _gen_many(item):
    from paper_2106_02762_gb300 import synth
    n, pairs, seed = item
    return synth.many_graph(n, pairs, seed)


STREAM_GRAPHS = 128  # graphs the streamed many-graph count takes


def multi_measure(ttc, torch, graphs, steps=5, warmup=2):
    """The many-graphs workload (its first `graphs` of 4096 specs): one
    persistent, graph-captured ttc_count_multi launch over all of them,
    timed, against one ttc_count call per graph; every graph's count is
    checked equal to its alone-run.  Returns a dict."""
    import concurrent.futures as cf
    import multiprocessing as mp
    from paper_2106_02762_gb300 import synth
    n, pairs, deltas, seeds = synth.many_graph_specs(count=4096)
    items = [(int(n[i]), int(pairs[i]), int(seeds[i])) for i in range(graphs)]
    # generated on the host cores (spawned workers) while loading in order
    pool = cf.ProcessPoolExecutor(max_workers=max(1, (os.cpu_count() or 2) - 1), mp_context=mp.get_context("spawn"))
    hs, m_tot = [], 0
    kept = []  # host arrays of the first graphs, for the streamed count below
    t0 = time.perf_counter()
    for s, d, t in pool.map(_gen_many, items, chunksize=4):
        hs.append(ttc.Graph(s, d, t))
        m_tot += s.size
        if len(kept) < STREAM_GRAPHS:
            kept.append((s, d, t))
    pool.shutdown()
    load_s = time.perf_counter() - t0
    dl = [tuple(int(x) for x in q) for q in deltas[:graphs]]
    first = ttc.count_multi(hs, dl)  # plan, autotune, capture
    for _ in range(warmup):
        assert (ttc.count_multi(hs, dl) == first).all()
    times = []
    for _ in range(steps):
        torch.cuda.synchronize()
        w = time.perf_counter()
        out = ttc.count_multi(hs, dl)
        times.append(time.perf_counter() - w)
        assert (out == first).all()
    step = statistics.median(times)
    seq = []
    for _ in range(2):
        torch.cuda.synchronize()
        w = time.perf_counter()
        alone = np.stack([g.count(q) for g, q in zip(hs, dl)])
        seq.append(time.perf_counter() - w)
        assert (alone == first).all()  # every graph's count equals its alone-run
    seq_s = min(seq)
    tau = sum(g.info()["tau"] for g in hs)
    # the streaming many-graph count of the first graphs from host arrays,
    # under a device budget of a quarter of their resident footprint
    ks = len(kept)
    budget = sum(g.info()["device_bytes"] for g in hs[:ks]) // 4
    for g in hs:
        g.free()
    m_str = sum(e[0].size for e in kept)
    st_times, nb = [], 0
    for _ in range(2):
        torch.cuda.synchronize()
        w = time.perf_counter()
        got, nb = ttc.count_stream(kept, dl[:ks], budget_bytes=budget)
        st_times.append(time.perf_counter() - w)
        assert (got == first[:ks]).all()
    st_s = min(st_times)
    return {"graphs": graphs, "m_total": m_tot, "tau_total": tau, "ms_per_launch": step * 1e3,
            "edges_per_s": m_tot / step, "sequential_ms": seq_s * 1e3, "speedup_vs_sequential": seq_s / step,
            "load_generate_s": load_s, "checked": "every graph's count equals its alone ttc_count call",
            "streamed": {"graphs": ks, "m_total": m_str, "budget_bytes": budget, "batches": nb, "s": st_s,
                         "edges_per_s": m_str / st_s,
                         "checked": "equal to the resident many-graph launch",
                         "note": "ttc_count_stream: loads from host arrays included, one many-graph launch a batch"},
            "workload": "many graphs: the first %d of 4096 specs (n log-uniform [1e3,1e5], degree U[4,32], "
                        "Chung-Lu 2.3, Geometric(0.3) multiplicity, t uniform [0,1e7), one delta per graph)"
                        % graphs}


def run_multi(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_02762_gb300 import ttc
    r = multi_measure(ttc, torch, args.graphs, steps=args.steps, warmup=args.warmup)
    print(json.dumps({"mode": "multi", "metric": METRIC, "value": r["edges_per_s"], "unit": UNIT,
                      "higher_is_better": True, **r}), flush=True)


# ------------------------------------------------------------------ served
def serve_measure(ttc, torch, rates, duration, ladder_scale=1.0, load_rate=1.0):
    """Served pool: 16 resident graphs (the ladder of 1e5 to 1e8 edges, times
    ladder_scale), Poisson query arrivals at each rate in `rates` for
    `duration` seconds, and new-graph loads at load_rate per second admitted
    under an HBM budget (the pool's resident bytes plus one arriving graph's
    load estimate), so arrivals evict least recently used idle graphs.  Every
    served result is checked equal to the same query counted alone on a
    separately loaded copy of its graph.  Returns a dict per rate."""
    import threading
    from paper_2106_02762_gb300 import synth
    ladder = synth.served_ladder()
    if ladder_scale != 1.0:
        ladder = [max(1000, int(x * ladder_scale)) for x in ladder]
    edges = {}  # graph id -> its edge arrays (for the alone-runs)
    srv = ttc.Server(streams=4, max_batch=256)
    pool_graphs = [synth.served_graph(m, synth.MASTER_SEED + 5 + j) for j, m in enumerate(ladder)]
    ids, m_tot = [], 0
    for gr in pool_graphs:
        gid = srv.load(*gr)
        ids.append(gid)
        edges[gid] = gr
        m_tot += gr[0].size
    arrive = [synth.served_graph(ladder[4 + 2 * j], synth.MASTER_SEED + 200 + j) for j in range(4)]
    torch.cuda.synchronize()
    ttc.release_cached()
    free, _ = torch.cuda.mem_get_info()
    est = max(96 * a[0].size + (64 << 20) for a in arrive)
    srv.set_reserve(max(0, free - est))
    for gid in ids:  # warm every graph once
        srv.submit(gid, (3600, 1800, 1800))
    srv.drain(60.0)
    results = []
    live = list(ids)  # graphs resident as far as the submitter knows (evictions found at submit)
    for ri, rate in enumerate(rates):
        rng = synth.rng_for(synth.MASTER_SEED + 50 + ri)
        arrivals = synth.poisson_arrivals(synth.MASTER_SEED + 51 + ri, rate, duration)
        picks = rng.random(size=arrivals.size)
        qs = synth.log_uniform_int(rng, 60, 2.6e6, size=(arrivals.size, 3))
        live_mu = threading.Lock()
        load_log = []
        stop = threading.Event()
        before = srv.info()

        def loader(t0):
            k = 0
            while not stop.is_set():
                due = (k + 1) / load_rate
                while time.perf_counter() - t0 < due and not stop.is_set():
                    time.sleep(0.001)
                if stop.is_set():
                    break
                w = time.perf_counter()
                a = arrive[k % len(arrive)]
                try:
                    gid = srv.load(*a)
                    ok = True
                except ttc.TTCError:
                    gid, ok = None, False
                load_log.append((time.perf_counter() - w, ok))
                if ok:
                    with live_mu:
                        edges[gid] = a
                        live.append(gid)
                k += 1

        tickets, missed = [], 0
        t0 = time.perf_counter()
        th = threading.Thread(target=loader, args=(t0,), daemon=True)
        th.start()
        for a, u, q in zip(arrivals, picks, qs):
            while time.perf_counter() - t0 < a:
                pass
            while True:
                with live_mu:
                    gid = live[int(u * len(live)) % len(live)]
                try:
                    tickets.append((srv.submit(gid, tuple(int(x) for x in q)), gid, tuple(int(x) for x in q)))
                    break
                except ttc.TTCError as e:
                    if "NOT_FOUND" not in str(e):
                        raise
                    missed += 1  # evicted since it was picked: pick again
                    with live_mu:
                        if gid in live:
                            live.remove(gid)
        stop.set()
        srv.drain(120.0)
        wall = time.perf_counter() - t0
        th.join(60.0)
        polled = [(srv.poll(tk), gid, q) for tk, gid, q in tickets]
        lat = np.asarray([p[0][1] for p in polled])
        after = srv.info()
        # every served result against the same query counted alone
        by_graph = {}
        for (cnt, _), gid, q in polled:
            by_graph.setdefault(gid, []).append((q, cnt))
        for gid, lst in by_graph.items():
            g = ttc.Graph(*edges[gid])
            alone = g.count_batch([q for q, _ in lst])
            g.free()
            assert all((alone[i] == cnt).all() for i, (_, cnt) in enumerate(lst)), gid
        loads_ok = [d for d, ok in load_log if ok]
        launches = after["launches"] - before["launches"]
        results.append({"arrival_rate": rate, "queries": len(tickets), "queries_per_s": len(tickets) / wall,
                        "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                        "mean_ms": float(lat.mean() * 1e3), "launches": launches,
                        "queries_per_launch": len(tickets) / max(1, launches),
                        "graph_loads": len(load_log), "graph_loads_admitted": len(loads_ok),
                        "evictions": after["evictions"] - before["evictions"], "resubmits_after_eviction": missed,
                        "checked": "every result equals its alone-run (tolerance 0)"})
    info = srv.info()
    srv.close()
    return {"graphs": len(ids), "m_total": m_tot, "hbm_headroom_bytes": int(est),
            "queue_depth_max": info["queue_depth_max"], "rates": results,
            "workload": "16 resident ER graphs, %.0e..%.0e edges (log-spaced), Poisson query arrivals, uniform "
                        "live graph, delta components log-uniform [60, 2.6e6] s, graph loads at %g/s admitted "
                        "with %.2f GB of headroom beyond the pool, LRU eviction"
                        % (ladder[0], ladder[-1], load_rate, est / 1e9)}


def run_serve(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_02762_gb300 import ttc
    r = serve_measure(ttc, torch, [args.rate, 10 * args.rate], args.duration, ladder_scale=args.scale,
                      load_rate=args.load_rate)
    print(json.dumps({"mode": "serve", "metric": "served latency", **r}), flush=True)


# ------------------------------------------------------------------ δ-grid
def run_grid(args):
    """δ-grid analytics on the power-law workload: a 16 x 16 (δ12, δ23) grid,
    log-spaced from 1 hour to δ13 = 2^31 s (the whole span: each pair's
    edges form one burst at a random time, so shorter windows close few
    temporal triangles on this recipe), in one batched call; reports the time
    per grid and the cyclic (T4 + T8) share."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_02762_gb300 import ttc
    src, dst, t, delta, name = workload(args.scale)
    g = ttc.Graph(src, dst, t)
    d13 = 1 << 31
    axis = np.unique(np.round(np.logspace(np.log10(3600), np.log10(d13), 16)).astype(np.int64))
    for _ in range(max(1, args.warmup)):
        counts, cyc = g.count_grid(d13, axis, axis)
    times = []
    for _ in range(max(1, args.steps)):
        torch.cuda.synchronize()
        w = time.perf_counter()
        counts, cyc = g.count_grid(d13, axis, axis)
        times.append(time.perf_counter() - w)
    sec = statistics.median(times)
    k = axis.size * axis.size
    info = g.info()
    g.free()
    print(json.dumps({"mode": "grid", "metric": "delta-grid queries/s", "grid": [int(axis.size), int(axis.size)],
                      "d13": d13, "axis": axis.tolist(), "ms_per_grid": sec * 1e3, "queries_per_s": k / sec,
                      "edges_per_s_per_query": info["m"] * k / sec,
                      "cyclic_share_min": float(cyc.min()), "cyclic_share_max": float(cyc.max()),
                      "cyclic_share_at_d12_eq_d23": [float(cyc[i, i]) for i in range(axis.size)],
                      "config": {"workload": name}}), flush=True)


# ------------------------------------------------------------------ DRAM traffic
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "light_kernel_dram_unbounded_power_law_1m.txt")


def light_traffic(ttc):
    """DRAM bytes (read + write) of one light-kernel launch on the full
    power-law workload, from the one-pass ncu capture summarised in
    profiles/; None when that capture was taken on other light-kernel source
    than the library built here (the version string carries its hash)."""
    try:
        fields = dict(line.split(":", 1) for line in open(TRAFFIC_FILE) if ":" in line)
    except OSError:
        return None
    built = ttc.lib().ttc_version().decode().rsplit("count:", 1)[-1].strip()
    if fields.get("count_source", "").strip() != built:
        return None
    try:
        return int(fields["dram_bytes_per_launch"].strip())
    except (KeyError, ValueError):
        return None


# ------------------------------------------------------------------ our arm
def timed_query(g, stream, torch, fn, iters):
    """Median CUDA-event time of fn() on the graph's stream (after one
    warm-up call) and the mean time of each kernel the library launched
    (seconds)."""
    g.set_profiling(True)
    fn()
    kern, times = {}, []
    for _ in range(iters):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        per = {}
        for kname, ms in g.profile():
            per[kname] = per.get(kname, 0.0) + ms / 1e3
        for kname, v in per.items():
            kern.setdefault(kname, []).append(v)
    g.set_profiling(False)
    return statistics.median(times), {k: sum(v) / len(v) for k, v in kern.items()}


def run_ours(args):
    import torch
    ws, rank, local = dist_setup("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    barrier(ws)
    from paper_2106_02762_gb300 import ttc
    ttc.lib()

    src, dst, t, delta, name = workload(args.scale)
    m_in = src.size
    stream = torch.cuda.Stream(device=dev)
    sptr = stream.cuda_stream
    d_src = torch.from_numpy(src.view(np.int32)).to(dev)
    d_dst = torch.from_numpy(dst.view(np.int32)).to(dev)
    d_t = torch.from_numpy(t).to(dev)
    h_src = torch.from_numpy(src.view(np.int32)).pin_memory()
    h_dst = torch.from_numpy(dst.view(np.int32)).pin_memory()
    h_t = torch.from_numpy(t).pin_memory()
    torch.cuda.synchronize()

    # a step answers the configured query and the same query with every
    # window unbounded, in one batched pass: with the second one present no
    # window lets the kernels skip work, so the step time does not rest on
    # the windows pruning it (the paper's cost does not depend on the windows)
    step_deltas = step_queries(delta)

    # the light threshold, tuned on this graph (rank 0; every rank then loads
    # with the same explicit value, so all hold the same bins)
    chosen, tune_ms = 0, None
    caps, caps_ms = (0, 0, 0), None
    if rank == 0:
        chosen, tune_ms = ttc.tune_light(d_src, d_dst, d_t, step_deltas, stream=sptr)
        # then the prefix-sum path's class caps and the one-CTA class's search
        # form at that threshold
        caps, caps_ms = ttc.tune_heavy(d_src, d_dst, d_t, step_deltas, light_max_pairs=chosen, stream=sptr)
    chosen = int(allreduce_max(float(chosen), ws, dev))
    caps = tuple(int(allreduce_max(float(x), ws, dev)) for x in caps)
    bins = dict(light_max_pairs=chosen, heavy_warp_cap=caps[0], heavy_cta_cap=caps[1], heavy_merge=caps[2])

    # on N GPUs every rank loads the same graph and counts its shard of the
    # triangle list; the ranks' counts are summed (the one exchange)
    def count(g):
        if ws == 1:
            return g.count_batch(step_deltas)
        from paper_2106_02762_gb300 import shard
        return shard.count_sharded(g, step_deltas, rank, ws, device=dev)

    def step_device():
        g = ttc.Graph(d_src, d_dst, d_t, stream=sptr, **bins)
        return g, count(g)

    def step_host():
        g = ttc.Graph(h_src.numpy().view(np.uint32), h_dst.numpy().view(np.uint32), h_t.numpy(), stream=sptr,
                      **bins)
        return g, count(g)

    # warm-up
    ref = None
    for _ in range(max(3, args.warmup)):
        g, out = step_device()
        if ref is None:
            ref = out
        assert (out == ref).all()
        info = g.info()
        g.free()
    m = info["m"]

    # timed: device-resident inputs, whole hot path
    clocks = Clocks(local)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    l0 = ttc.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    w0 = time.perf_counter()
    for _ in range(args.steps):
        g, out = step_device()
        assert (out == ref).all()
        g.free()
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    launches = ttc.launch_count() - l0
    clk = clocks.stop()
    dev_s = ev0.elapsed_time(ev1) / 1e3
    step_s = allreduce_max(max(dev_s, 1e-9) / args.steps, ws, dev)
    value = m / step_s  # one graph per step, whatever the number of GPUs

    # the load alone, device-timed on the graph's stream
    load_ms = []
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g = ttc.Graph(d_src, d_dst, d_t, stream=sptr, **bins)
        e1.record(stream)
        e1.synchronize()
        load_ms.append(e0.elapsed_time(e1))
        g.free()
    load_s = statistics.median(load_ms) / 1e3

    # queries on a resident graph, each with per-kernel CUDA-event times
    # recorded by the library on the graph's stream
    torch.cuda.synchronize()
    w = time.perf_counter()
    g = ttc.Graph(d_src, d_dst, d_t, stream=sptr, profile_load=True, **bins)
    load_wall = time.perf_counter() - w
    load_phases = {k: v for k, v in g.profile()}
    info = g.info()
    from paper_2106_02762_gb300 import synth
    unb = synth.LARGE_PLAIN_DELTA_UNBOUNDED
    q_s, kern_cfg = timed_query(g, stream, torch, lambda: g.count(delta), args.query_iters)
    # every window unbounded: no window lets a kernel skip a pair, so this is
    # the query the count kernels' roofline is taken on
    u_s, kern_unb = timed_query(g, stream, torch, lambda: g.count(unb), max(3, args.query_iters // 2))
    b_s, kern_step = timed_query(g, stream, torch, lambda: g.count_batch(step_deltas), max(3, args.query_iters // 2))
    # the 64-delta sweep on this graph: one batched call against 64 plain calls
    sweep = synth.delta_sweep()
    ref_sw = g.count_batch(sweep)
    sw_b, sw_q = [], []
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b = g.count_batch(sweep)
        e1.record(stream)
        e1.synchronize()
        sw_b.append(e0.elapsed_time(e1) / 1e3)
        assert (b == ref_sw).all()
        e0.record(stream)
        seq = [g.count(q) for q in sweep]
        e1.record(stream)
        e1.synchronize()
        sw_q.append(e0.elapsed_time(e1) / 1e3)
        assert (np.stack(seq) == ref_sw).all()
    sw_b_s, sw_q_s = statistics.median(sw_b), statistics.median(sw_q)
    batched_large = {"workload": name + ", 64 delta-triples log-spaced 60 s..30 d (d13), resident graph",
                     "batch_queries_per_s": len(sweep) / sw_b_s, "sequential_queries_per_s": len(sweep) / sw_q_s,
                     "speedup": sw_q_s / sw_b_s, "batch_ms": sw_b_s * 1e3, "sequential_ms": sw_q_s * 1e3}
    listed_bytes = g.info()["device_bytes"]
    g.free()
    # the same step with a streamed handle (no light-triangle list: each
    # count enumerates again), device-timed
    st_step, st_load = [], []
    for i in range(4):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gs = ttc.Graph(d_src, d_dst, d_t, stream=sptr, streamed=True, **bins)
        e1.record(stream)
        out_s = gs.count_batch(step_deltas)
        e2.record(stream)
        e2.synchronize()
        assert (out_s == ref).all()
        if i:
            st_step.append(e0.elapsed_time(e2))
            st_load.append(e0.elapsed_time(e1))
        st_bytes = gs.info()["device_bytes"]
        gs.free()
    streamed = {"step_ms": statistics.median(st_step), "load_ms": statistics.median(st_load),
                "device_bytes": st_bytes, "listed_device_bytes": listed_bytes,
                "note": "TTC_LOAD_STREAM: the handle keeps the oriented graph instead of the light-triangle list"}
    wb_heavy = info["work_bytes_heavy"]
    wb_light = info["work_bytes"] - wb_heavy
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        try:
            peaks = json.load(open(pk_path))
        except ValueError:
            peaks = {}
    hbm_peak = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm_peak else "fallback"
    hbm_peak = float(hbm_peak or 6800.0)
    roof = None
    if kern_unb.get("light"):
        # dominant kernel: the single-query light bin on the unbounded query;
        # algorithmic bytes = sum over its triangles of 8 (s_uv + s_uw + s_vw) + 12
        k_s = kern_unb["light"]
        ach = wb_light / k_s / 1e9
        roof = {"kernel": "light", "delta": list(unb), "bound": "hbm", "achieved": ach, "peak": hbm_peak,
                "unit": "GB/s", "frac": ach / hbm_peak, "traffic": light_traffic(ttc), "peak_source": peak_src,
                "algorithmic_bytes": wb_light, "kernel_ms": k_s * 1e3,
                "query": {"ms": u_s * 1e3, "algorithmic_bytes": info["work_bytes"],
                          "achieved": info["work_bytes"] / u_s / 1e9,
                          "frac": info["work_bytes"] / u_s / 1e9 / hbm_peak},
                "pruned": {"delta": list(delta), "kernel_ms": kern_cfg.get("light", 0.0) * 1e3,
                           "note": "configured windows: the light bin skips every pair whose time gap exceeds "
                                   "d13 before searching C, so its bytes/time is not a roofline figure"}}

    # e2e: host (pinned) buffers through the C ABI, copies inside the timed region
    barrier(ws)
    torch.cuda.synchronize()
    e_times = []
    for _ in range(max(1, args.steps // 2)):
        w = time.perf_counter()
        g, out = step_host()
        e_times.append(time.perf_counter() - w)
        assert (out == ref).all()
        g.free()
    e_s = allreduce_max(statistics.median(e_times), ws, dev)
    e2e = {"value": m / e_s, "unit": UNIT, "h2d_bytes_per_step": int(m_in * 16),
           "d2h_bytes_per_step": 64 * len(step_deltas)}

    batched = batched_sweep(ttc, torch) if rank == 0 else None
    # the many-graphs and served workloads, reduced to a few seconds each
    multi = served = None
    if rank == 0 and not args.no_extras:
        multi = multi_measure(ttc, torch, args.multi_graphs)
        served = serve_measure(ttc, torch, [2000.0, 50000.0], args.serve_seconds, ladder_scale=0.1)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, desc, cores, sec = oracle_sample(delta)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
               "sample_seconds": sec}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": name, "m": m, "tau": info["tau"], "delta": list(delta),
                       "step": "ttc_load (device-resident edges) + one ttc_count_batch of the configured delta "
                               "and the unbounded delta (2^31, 2^31, 2^31), so no window pruning applies",
                       "step_deltas": [list(q) for q in step_deltas],
                       "l2": "inputs larger than L2 (no flush)",
                       "parallelism": ("every rank loads the graph and counts 1/%d of its triangles; counts summed"
                                       % ws) if ws > 1 else "1 gpu"},
            "query": {"edges_per_s": m / q_s, "static_triangles_per_s": info["tau"] / q_s, "ms": q_s * 1e3,
                      "kernels_ms": {k: v * 1e3 for k, v in kern_cfg.items()}},
            "query_unbounded": {"delta": list(unb), "edges_per_s": m / u_s,
                                "static_triangles_per_s": info["tau"] / u_s, "ms": u_s * 1e3,
                                "kernels_ms": {k: v * 1e3 for k, v in kern_unb.items()}},
            "step_count": {"deltas": [list(q) for q in step_deltas], "ms": b_s * 1e3,
                           "kernels_ms": {k: v * 1e3 for k, v in kern_step.items()}},
            "kernels_ms_note": "CUDA events around each kernel on the stream it runs on; a count runs its heavy "
                               "bins on a side stream beside the light kernel, so their times include waiting for "
                               "the SM slots the light kernel holds, and the query's ms is less than the sum",
            "light_threshold": {"chosen": chosen, "candidates_ms": tune_ms,
                                "note": "ttc_tune_light: load + the step's batch at each threshold"},
            "heavy_caps": {"chosen": list(caps),
                           "candidates_ms": {"%d/%d/%s" % (w, c, "merge" if mg == ttc.HEAVY_MERGE else "binary"): v
                                             for (w, c, mg), v in caps_ms.items()} if caps_ms else None,
                           "note": "ttc_tune_heavy at the chosen light threshold: the prefix-sum path's "
                                   "one-warp and one-CTA caps (edges of A plus B) and the one-CTA class's "
                                   "search form (1 binary, 2 two-pointer)"},
            "load_ms": load_s * 1e3,
            "load_edges_per_s": m / load_s,
            "load_phases_ms": {"wall": load_wall * 1e3, **load_phases},
            "roofline": roof,
            "batched": batched,
            "batched_large": batched_large,
            "multi": multi,
            "served": served,
            "streamed": streamed,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "wall_s_timed": wall,
            "clocks": clk,
            "cpu_baseline": cpu,
            "graph": {k: info[k] for k in ("n", "m", "m_s", "tau", "kappa", "sigma_max", "peel_rounds",
                                            "work_bytes", "work_bytes_heavy", "tau_light", "tau_heavy",
                                            "enum_elems", "light_pairs", "device_bytes")},
        }
        print(json.dumps(line), flush=True)
    barrier(ws)


def run_zipf15(args):
    """The power-law recipe with the multiplicity exponent 1.5 taken
    literally (about 766M edges, mean multiplicity 77): the same timed step
    (load from device edges + one batched count of the configured and the
    unbounded delta) with a listed and with a streamed handle, device-timed."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_02762_gb300 import ttc, synth
    w = time.perf_counter()
    src, dst, t = synth.large_plain_zipf15(scale=args.scale)
    gen_s = time.perf_counter() - w
    dev = torch.device("cuda", 0)
    d_src = torch.from_numpy(src.view(np.int32)).to(dev)
    d_dst = torch.from_numpy(dst.view(np.int32)).to(dev)
    d_t = torch.from_numpy(t).to(dev)
    del src, dst, t
    stream = torch.cuda.Stream(device=dev)
    qs = step_queries(synth.LARGE_PLAIN_DELTA)
    res, ref = {}, None
    for streamed in (False, True):
        st, ld = [], []
        for i in range(max(1, args.warmup) + max(1, args.steps)):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e2 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g = ttc.Graph(d_src, d_dst, d_t, stream=stream.cuda_stream, streamed=streamed)
            e1.record(stream)
            out = g.count_batch(qs)
            e2.record(stream)
            e2.synchronize()
            if ref is None:
                ref = out
            assert (out == ref).all()
            if i >= max(1, args.warmup):
                st.append(e0.elapsed_time(e2))
                ld.append(e0.elapsed_time(e1))
            info = g.info()
            g.free()
        res["streamed" if streamed else "listed"] = {"step_ms": statistics.median(st), "load_ms": statistics.median(ld),
                                                     "device_bytes": info["device_bytes"]}
    m = info["m"]
    print(json.dumps({"mode": "zipf15", "metric": "temporal edges/s per delta-query",
                      "value": m / (res["listed"]["step_ms"] / 1e3), "unit": UNIT, **res,
                      "graph": {k: info[k] for k in ("n", "m", "m_s", "tau", "tau_light", "tau_heavy", "tau_huge",
                                                     "kappa", "sigma_max", "work_bytes", "light_pairs")},
                      "unbounded_total": int(ref[1].sum()), "generate_s": gen_s,
                      "config": {"workload": "power-law n=%d pairs=%d gamma=2.1 zipf1.5-cap1e4 lognormal(6,2) span 2^31"
                                 % (int(round(1_000_000 * args.scale)), int(round(10_000_000 * args.scale))),
                                 "step_deltas": [list(q) for q in qs]}}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "multi":
        run_multi(args)
    elif args.mode == "serve":
        run_serve(args)
    elif args.mode == "grid":
        run_grid(args)
    elif args.mode == "zipf15":
        run_zipf15(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
