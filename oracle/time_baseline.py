"""Times the CPU oracle on the workloads the CUDA path is measured on, for
the reported CPU baseline (test infrastructure, like the oracle itself):

- tiny plain (n = 1000, 5000 pairs, ~20K edges), one query, O1 on one host
  thread and on every host thread;
- the full power-law workload (n = 1M, 10M pairs, ~60M edges), the bench
  step's two queries, O1 with the forward enumeration (O1f) on every host
  thread (the plain enumeration visits about deg^2 vertex pairs at each hub
  and does not finish in useful time at this size), with the time of its
  graph build (one sort of the edges and the adjacency) stated apart.

Prints one JSON line.

    python oracle/time_baseline.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    import oracle
    from paper_2106_02762_gb300 import synth
    oracle.build()
    cores = os.cpu_count() or 1
    out = {"host_threads": cores}
    s, d, t = synth.tiny_plain()
    q = [(3600, 1800, 1800)]
    for threads, key in ((1, "tiny_plain_1_thread_s"), (0, "tiny_plain_all_threads_s")):
        best = None
        for _ in range(3):
            w = time.perf_counter()
            oracle.count(s, d, t, q, threads=threads)
            dt = time.perf_counter() - w
            best = dt if best is None else min(best, dt)
        out[key] = best
    out["tiny_plain_m"] = int(s.size)
    s, d, t = synth.large_plain()
    step = [synth.LARGE_PLAIN_DELTA, synth.LARGE_PLAIN_DELTA_UNBOUNDED]
    w = time.perf_counter()
    st = oracle.stats_fwd(s, d, t)
    out["power_law_build_and_enumerate_s"] = time.perf_counter() - w
    w = time.perf_counter()
    oracle.count_fwd(s, d, t, step)
    out["power_law_o1f_step_s"] = time.perf_counter() - w
    out["power_law_m"] = st["m"]
    out["power_law_tau"] = st["tau"]
    out["power_law_o1f_edges_per_s"] = st["m"] / out["power_law_o1f_step_s"]
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
