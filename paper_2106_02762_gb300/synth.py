"""Seeded synthetic temporal multigraphs shaped like the paper's workloads.

This module only draws inputs.  It holds none of the counting arithmetic, so
both the CUDA path and the CPU oracle may take their inputs from it.

A temporal multigraph is returned as three numpy arrays ``(src, dst, t)``:
``uint32`` vertex ids and ``int64`` timestamps (Sec. 3: a directed temporal
edge is a tuple (u, v, t); many edges may share a vertex pair).  The edge
index used to break timestamp ties is the array position.  Unless a recipe
says otherwise, each edge's direction is uniform and the edge order is a
seeded shuffle, so inputs are not time-sorted.

The paper's datasets (Sec. 6, Table 2) are not available; these recipes stand
in for them.  Every generator is deterministic in its seed and draws from a
counter-based bit generator (Philox), so a given seed gives the same graph on
any machine.
"""
from __future__ import annotations

import math

import numpy as np

MASTER_SEED = 20210614
T_SPAN_2_31 = 1 << 31


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


# --------------------------------------------------------------------------
# static skeletons
# --------------------------------------------------------------------------
def er_pairs(rng: np.random.Generator, n: int, n_pairs: int) -> np.ndarray:
    """``n_pairs`` distinct unordered pairs {a, b}, a != b, uniform over all
    C(n, 2) pairs (rejection of self-loops and repeats).  Returns an
    (n_pairs, 2) uint32 array with a < b."""
    if n_pairs > n * (n - 1) // 2:
        raise ValueError("more pairs than the complete graph has")
    keys = np.empty(0, dtype=np.int64)
    while keys.size < n_pairs:
        k = int((n_pairs - keys.size) * 1.2) + 16
        a = rng.integers(0, n, size=k, dtype=np.int64)
        b = rng.integers(0, n, size=k, dtype=np.int64)
        keep = a != b
        a, b = a[keep], b[keep]
        cat = np.concatenate([keys, np.minimum(a, b) * n + np.maximum(a, b)])
        _, first = np.unique(cat, return_index=True)
        keys = cat[np.sort(first)]
    keys = keys[:n_pairs]
    return np.stack([keys // n, keys % n], axis=1).astype(np.uint32)


def chung_lu_pairs(rng: np.random.Generator, n: int, n_pairs: int, gamma: float) -> np.ndarray:
    """Chung-Lu power-law skeleton: vertex i gets weight (i+1)^(-1/(gamma-1));
    endpoints are drawn i.i.d. in proportion to weight, self-loops and repeats
    are rejected until ``n_pairs`` distinct pairs exist, and the ids then get a
    seeded random permutation.  Returns (n_pairs, 2) uint32 with a < b."""
    w = np.power(np.arange(1, n + 1, dtype=np.float64), -1.0 / (gamma - 1.0))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    keys = np.empty(0, dtype=np.int64)
    while keys.size < n_pairs:
        need = n_pairs - keys.size
        k = int(need * 1.5) + 1024
        a = np.searchsorted(cdf, rng.random(k), side="right").astype(np.int64)
        b = np.searchsorted(cdf, rng.random(k), side="right").astype(np.int64)
        np.minimum(a, n - 1, out=a)
        np.minimum(b, n - 1, out=b)
        keep = a != b
        a, b = a[keep], b[keep]
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        cat = np.concatenate([keys, lo * n + hi])
        _, first = np.unique(cat, return_index=True)
        keys = cat[np.sort(first)]
    keys = keys[:n_pairs]
    perm = rng.permutation(n).astype(np.int64)
    a, b = perm[keys // n], perm[keys % n]
    return np.stack([np.minimum(a, b), np.maximum(a, b)], axis=1).astype(np.uint32)


# --------------------------------------------------------------------------
# multiplicities and timestamps
# --------------------------------------------------------------------------
def truncated_zipf(rng: np.random.Generator, size: int, exponent: float, cap: int) -> np.ndarray:
    """pmf proportional to k^-exponent on {1, ..., cap}."""
    k = np.arange(1, cap + 1, dtype=np.float64)
    cdf = np.cumsum(np.power(k, -exponent))
    cdf /= cdf[-1]
    return (np.searchsorted(cdf, rng.random(size), side="right") + 1).astype(np.int64)


def _expand(rng: np.random.Generator, pairs: np.ndarray, mult: np.ndarray):
    """One edge per unit of multiplicity, each with a uniform direction."""
    rep = np.repeat(np.arange(pairs.shape[0], dtype=np.int64), mult)
    flip = rng.integers(0, 2, size=rep.size, dtype=np.int8).astype(bool)
    a = pairs[rep, 0]
    b = pairs[rep, 1]
    src = np.where(flip, b, a).astype(np.uint32)
    dst = np.where(flip, a, b).astype(np.uint32)
    return rep, src, dst


def _shuffle(rng: np.random.Generator, src, dst, t):
    perm = rng.permutation(src.size)
    return (np.ascontiguousarray(src[perm]), np.ascontiguousarray(dst[perm]),
            np.ascontiguousarray(t[perm]))


def renewal_times(rng: np.random.Generator, rep: np.ndarray, mult: np.ndarray,
                  mu: float, sigma: float, span: int) -> np.ndarray:
    """Per-pair renewal process: the first edge of a pair starts uniform in
    [0, span), each later edge follows after round(LogNormal(mu, sigma))
    seconds, and times wrap modulo ``span``.  ``rep`` must be grouped by pair
    (as ``_expand`` returns it)."""
    m = rep.size
    gaps = np.rint(rng.lognormal(mu, sigma, size=m)).astype(np.int64)
    starts = np.repeat(np.cumsum(mult) - mult, mult)  # first position of each pair
    first_pos = np.cumsum(mult) - mult
    gaps[first_pos] = 0
    cs = np.cumsum(gaps)
    within = cs - cs[starts]
    start_t = rng.integers(0, span, size=mult.size, dtype=np.int64)
    return (start_t[rep] + within) % span


# --------------------------------------------------------------------------
# workload recipes
# --------------------------------------------------------------------------
def random_tiny(seed: int, n: int = 6, m: int = 24, t_range: int = 12):
    """Tiny random multigraph for brute-force checks: ids in [0, n), any
    directed pair (self-loops included), timestamps in [0, t_range) so that
    equal timestamps are common."""
    rng = rng_for(seed)
    src = rng.integers(0, n, size=m, dtype=np.int64).astype(np.uint32)
    dst = rng.integers(0, n, size=m, dtype=np.int64).astype(np.uint32)
    t = rng.integers(0, max(1, t_range), size=m, dtype=np.int64)
    return src, dst, t


def er_temporal(seed: int, n: int = 1000, n_pairs: int = 5000, t_hi: int = 1_000_000,
                poisson_mean: float = 3.0):
    """Erdos-Renyi skeleton G(n, n_pairs distinct pairs); each pair carries
    1 + Poisson(poisson_mean) edges; timestamps uniform in [0, t_hi)."""
    rng = rng_for(seed)
    pairs = er_pairs(rng, n, n_pairs)
    mult = 1 + rng.poisson(poisson_mean, size=n_pairs).astype(np.int64)
    _, src, dst = _expand(rng, pairs, mult)
    t = rng.integers(0, t_hi, size=src.size, dtype=np.int64)
    return _shuffle(rng, src, dst, t)


def tiny_plain(seed: int = MASTER_SEED + 1):
    """Erdos-Renyi, n = 1,000 vertices, 5,000 pairs, 1 + Poisson(3) edges per
    pair, timestamps uniform in [0, 1e6)."""
    return er_temporal(seed, 1000, 5000, 1_000_000, 3.0)


TINY_PLAIN_DELTA = (3600, 1800, 1800)


def power_law_temporal(seed: int, n: int, n_pairs: int, gamma: float = 2.1,
                       zipf_exponent: float = 2.0, zipf_cap: int = 10_000,
                       mu: float = 6.0, sigma: float = 2.0, span: int = T_SPAN_2_31):
    """Chung-Lu skeleton with degree exponent ``gamma``; multiplicity per pair
    truncated Zipf(``zipf_exponent``) on [1, ``zipf_cap``]; bursty per-pair
    timestamps (lognormal inter-arrival, wrapped modulo ``span``)."""
    rng = rng_for(seed)
    pairs = chung_lu_pairs(rng, n, n_pairs, gamma)
    mult = truncated_zipf(rng, n_pairs, zipf_exponent, zipf_cap)
    rep, src, dst = _expand(rng, pairs, mult)
    t = renewal_times(rng, rep, mult, mu, sigma, span)
    return _shuffle(rng, src, dst, t)


def large_plain(seed: int = MASTER_SEED + 2, scale: float = 1.0):
    """Power-law workload: n = 1M vertices, 10M pairs (both times ``scale``),
    degree exponent 2.1, multiplicity pmf k^-2 on [1, 1e4] (about 60M edges at
    scale 1), lognormal(6, 2) inter-arrival times over a 2^31 s span."""
    n = max(16, int(round(1_000_000 * scale)))
    pairs = max(8, int(round(10_000_000 * scale)))
    return power_law_temporal(seed, n, pairs, 2.1, 2.0, 10_000, 6.0, 2.0, T_SPAN_2_31)


def large_plain_zipf15(seed: int = MASTER_SEED + 2, scale: float = 1.0):
    """The power-law workload with the multiplicity exponent taken literally:
    pmf k^-1.5 on [1, 1e4] (mean about 77, so about 766M edges at scale 1);
    the same skeleton and timestamps recipe as ``large_plain``."""
    n = max(16, int(round(1_000_000 * scale)))
    pairs = max(8, int(round(10_000_000 * scale)))
    return power_law_temporal(seed, n, pairs, 2.1, 1.5, 10_000, 6.0, 2.0, T_SPAN_2_31)


LARGE_PLAIN_DELTA = (86400, 43200, 43200)
LARGE_PLAIN_DELTA_UNBOUNDED = (1 << 31, 1 << 31, 1 << 31)


def delta_sweep(k: int = 64, lo: int = 60, hi: int = 2_592_000):
    """``k`` delta-triples (d13, d12, d23): d13 log-spaced from ``lo`` to
    ``hi`` seconds; even entries use d12 = d23 = d13 // 2, odd entries use
    d12 = d13 // 4 and d23 = 3 * d13 // 4."""
    out = []
    for i in range(k):
        d13 = int(round(lo * (hi / lo) ** (i / max(1, k - 1))))
        if i % 2 == 0:
            out.append((d13, d13 // 2, d13 // 2))
        else:
            out.append((d13, d13 // 4, (3 * d13) // 4))
    return np.asarray(out, dtype=np.int64)


def log_uniform_int(rng: np.random.Generator, lo: float, hi: float, size=None):
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=size))).astype(np.int64)


def many_graph_specs(seed: int = MASTER_SEED + 4, count: int = 4096,
                     n_lo: float = 1e3, n_hi: float = 1e5):
    """Per-graph parameters of the many-graphs workload: vertex count
    log-uniform in [n_lo, n_hi], average degree uniform in [4, 32], one
    delta-triple per graph with each component log-uniform in [60, 1e6]."""
    rng = rng_for(seed)
    n = log_uniform_int(rng, n_lo, n_hi, size=count)
    deg = rng.uniform(4.0, 32.0, size=count)
    pairs = np.maximum(1, np.rint(n * deg / 2.0)).astype(np.int64)
    pairs = np.minimum(pairs, n * (n - 1) // 2)
    deltas = log_uniform_int(rng, 60, 1e6, size=(count, 3))
    seeds = rng.integers(0, 1 << 62, size=count, dtype=np.int64)
    return n, pairs, deltas, seeds


def many_graph(n: int, n_pairs: int, seed: int, gamma: float = 2.3, p: float = 0.3,
               t_hi: int = 10_000_000):
    """One graph of the many-graphs workload: Chung-Lu skeleton (exponent
    ``gamma``), Geometric(``p``) multiplicity on {1, 2, ...}, timestamps
    uniform in [0, t_hi)."""
    rng = rng_for(int(seed))
    pairs = chung_lu_pairs(rng, int(n), int(n_pairs), gamma)
    mult = rng.geometric(p, size=pairs.shape[0]).astype(np.int64)
    _, src, dst = _expand(rng, pairs, mult)
    t = rng.integers(0, t_hi, size=src.size, dtype=np.int64)
    return _shuffle(rng, src, dst, t)


def served_ladder(count: int = 16, m_lo: float = 1e5, ratio: float = 1000.0):
    """Edge counts of the served pool: m_j = round(m_lo * ratio^(j/(count-1)))."""
    return [int(round(m_lo * ratio ** (j / max(1, count - 1)))) for j in range(count)]


def served_graph(m_target: int, seed: int):
    """An Erdos-Renyi graph with about ``m_target`` edges: m/4 pairs,
    n = pairs/5 vertices, 1 + Poisson(3) edges per pair, t in [0, 1e6)."""
    n_pairs = max(4, m_target // 4)
    n = max(8, n_pairs // 5)
    return er_temporal(seed, n, n_pairs, 1_000_000, 3.0)


def poisson_arrivals(seed: int, rate: float, duration_s: float):
    rng = rng_for(seed)
    k = rng.poisson(rate * duration_s)
    return np.sort(rng.uniform(0.0, duration_s, size=k))
