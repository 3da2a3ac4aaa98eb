"""Thin Python binding of the ttc C ABI (include/ttc.h).

Argument marshalling only: every step of loading and counting runs in the
CUDA library ``_build/libttc.so``.  If that library is missing this module
raises instead of falling back to anything else.

Edge arrays may be numpy arrays (host; copied by the library) or torch CUDA
tensors (device; passed as device pointers).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# TTC_LIB selects another build of the library (the one with device index
# checks, build.build(debug_bounds=True)); the default is the in-tree build
LIB_PATH = os.environ.get("TTC_LIB") or os.path.join(HERE, "_build", "libttc.so")
NUM_TYPES = 8

OK, PENDING = 0, 1
STATUS = {-1: "INVALID", -2: "RANGE", -3: "NOMEM", -4: "CUDA", -5: "TIMEOUT", -6: "OVERFLOW",
          -7: "BUSY", -8: "INTERNAL", -9: "NOT_FOUND"}

LOAD_DEVICE_INPUT = 1
LOAD_PROFILE = 2
LOAD_STREAM = 4
LOAD_STRICT_TIME = 8
ORIENT_DEGENERACY, ORIENT_ID, ORIENT_DEGREE, ORIENT_RANDOM = 0, 1, 2, 3
LABEL_HEAVIEST_VW, LABEL_SOURCE = 0, 1
HEAVY_BINARY, HEAVY_MERGE = 1, 2  # the one-CTA class's search form (TTC_HEAVY_*)

EXPORTS = ["ttc_load", "ttc_load_ex", "ttc_free", "ttc_graph_info", "ttc_count", "ttc_count_batch",
           "ttc_count_batch_async", "ttc_count_multi", "ttc_count_sample", "ttc_server_create",
           "ttc_server_destroy", "ttc_serve_load", "ttc_serve_submit", "ttc_serve_poll", "ttc_serve_drain",
           "ttc_serve_pause", "ttc_serve_set_reserve",
           "ttc_server_info", "ttc_last_error", "ttc_version", "ttc_debug_fail_alloc_after",
           "ttc_debug_launch_count", "ttc_set_profiling", "ttc_profile_read", "ttc_count_noalloc",
           "ttc_release_cached", "ttc_memory_info", "ttc_count_grid", "ttc_count_shard", "ttc_tune_light", "ttc_tune_heavy",
           "ttc_count_stream", "ttc_count_participation", "ttc_graph_pairs"]
TUNE_CANDIDATES = (17, 65, 257, 1025, 4097, 16385)  # ttc_tune_candidates in ttc.h
# ttc_tune_heavy_candidates in ttc.h: (warp cap, CTA cap, search form)
TUNE_HEAVY_CANDIDATES = ((128, 2048, HEAVY_BINARY), (64, 2048, HEAVY_BINARY), (32, 2048, HEAVY_BINARY),
                         (128, 1024, HEAVY_BINARY), (64, 1024, HEAVY_BINARY), (128, 512, HEAVY_BINARY),
                         (128, 2048, HEAVY_MERGE), (64, 2048, HEAVY_MERGE))


class TTCError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status


class Delta(ctypes.Structure):
    _fields_ = [("d13", ctypes.c_int64), ("d12", ctypes.c_int64), ("d23", ctypes.c_int64)]


class LoadOpts(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_uint32), ("orientation", ctypes.c_uint32), ("labeling", ctypes.c_uint32),
                ("light_max_pairs", ctypes.c_uint32), ("heavy_warp_cap", ctypes.c_uint32),
                ("heavy_cta_cap", ctypes.c_uint32), ("heavy_merge", ctypes.c_uint32), ("seed", ctypes.c_uint64),
                ("stream", ctypes.c_void_p)]


class GraphStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in
                ("n", "m", "m_self_loops", "m_s", "tau", "kappa", "sigma_max", "peel_rounds", "work_bytes",
                 "enum_elems", "tau_light", "tau_heavy", "device_bytes", "work_bytes_heavy", "tau_huge", "tau_hwarp", "tau_hcta", "light_pairs")] + \
               [("key_bits", ctypes.c_uint32), ("light_max_pairs", ctypes.c_uint32),
                ("heavy_warp_cap", ctypes.c_uint32), ("heavy_cta_cap", ctypes.c_uint32),
                ("heavy_merge", ctypes.c_uint32)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("ms", ctypes.c_float)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_reserve_bytes", ctypes.c_uint64), ("max_batch", ctypes.c_uint32),
                ("max_queue", ctypes.c_uint32), ("streams", ctypes.c_uint32), ("wait_limit_us", ctypes.c_uint32)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in
                ("submitted", "completed", "launches", "graphs_resident", "admissions", "evictions",
                 "queue_depth_max")]


_lib = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("ttc CUDA library not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        p, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
        sig = {
            "ttc_load": ([p, p, p, u64], p),
            "ttc_load_ex": ([p, p, p, u64, p, p], ctypes.c_int),
            "ttc_free": ([p], None),
            "ttc_graph_info": ([p, p], ctypes.c_int),
            "ttc_count": ([p, p, p], ctypes.c_int),
            "ttc_count_batch": ([p, p, u32, p], ctypes.c_int),
            "ttc_count_batch_async": ([p, p, u32, p, p], ctypes.c_int),
            "ttc_count_shard": ([p, p, u32, u32, u32, p], ctypes.c_int),
            "ttc_tune_light": ([p, p, p, u64, p, p, u32, p, p], ctypes.c_int),
            "ttc_tune_heavy": ([p, p, p, u64, p, p, u32, p, p, p, p], ctypes.c_int),
            "ttc_count_stream": ([p, p, p, p, p, u32, p, u64, p, p], ctypes.c_int),
            "ttc_count_participation": ([p, p, p, p], ctypes.c_int),
            "ttc_graph_pairs": ([p, p], ctypes.c_int),
            "ttc_count_multi": ([p, p, u32, p], ctypes.c_int),
            "ttc_count_sample": ([p, p, u64, u64, u64, p, p, p], ctypes.c_int),
            "ttc_server_create": ([p], p),
            "ttc_server_destroy": ([p], None),
            "ttc_serve_load": ([p, p, p, p, u64, p], ctypes.c_int),
            "ttc_serve_submit": ([p, u64, p, p], ctypes.c_int),
            "ttc_serve_poll": ([p, u64, p, p], ctypes.c_int),
            "ttc_serve_drain": ([p, ctypes.c_double], ctypes.c_int),
            "ttc_serve_pause": ([p, ctypes.c_int], ctypes.c_int),
            "ttc_serve_set_reserve": ([p, u64], ctypes.c_int),
            "ttc_server_info": ([p, p], ctypes.c_int),
            "ttc_last_error": ([], ctypes.c_char_p),
            "ttc_version": ([], ctypes.c_char_p),
            "ttc_debug_fail_alloc_after": ([u64], None),
            "ttc_release_cached": ([p], ctypes.c_int),
            "ttc_memory_info": ([p, p, p], ctypes.c_int),
            "ttc_count_grid": ([p, ctypes.c_int64, p, u32, p, u32, p, p], ctypes.c_int),
            "ttc_debug_launch_count": ([], u64),
            "ttc_set_profiling": ([p, ctypes.c_int], ctypes.c_int),
            "ttc_profile_read": ([p, p, u32], u32),
            "ttc_count_noalloc": ([p, p, p, p], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def last_error() -> str:
    return lib().ttc_last_error().decode()


def check(status):
    if status < 0:
        raise TTCError(status, last_error())
    return status


def _deltas(deltas):
    d = np.ascontiguousarray(np.asarray(deltas, dtype=np.int64).reshape(-1, 3))
    return d, d.ctypes.data_as(ctypes.c_void_p)


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _edge_ptrs(src, dst, t):
    """Returns (ptrs, m, flags, keepalive)."""
    if _is_torch(src):
        import torch
        if not (src.is_cuda and dst.is_cuda and t.is_cuda):
            raise ValueError("torch edge tensors must be CUDA tensors")
        if src.dtype != torch.int32 and src.dtype != torch.uint32:
            raise ValueError("src/dst must be int32/uint32 tensors")
        if t.dtype != torch.int64:
            raise ValueError("t must be an int64 tensor")
        src, dst, t = src.contiguous(), dst.contiguous(), t.contiguous()
        m = src.numel()
        if dst.numel() != m or t.numel() != m:
            raise ValueError("src, dst, t must have equal length")
        return (src.data_ptr(), dst.data_ptr(), t.data_ptr()), m, LOAD_DEVICE_INPUT, (src, dst, t)
    src = np.ascontiguousarray(src, dtype=np.uint32)
    dst = np.ascontiguousarray(dst, dtype=np.uint32)
    t = np.ascontiguousarray(t, dtype=np.int64)
    if not (src.shape == dst.shape == t.shape) or src.ndim != 1:
        raise ValueError("src, dst, t must be 1-D arrays of equal length")
    ptrs = tuple(a.ctypes.data if a.size else None for a in (src, dst, t))
    return ptrs, src.size, 0, (src, dst, t)


class Graph:
    """A device-resident temporal graph (``ttc_load_ex``)."""

    def __init__(self, src, dst, t, orientation=ORIENT_DEGENERACY, labeling=LABEL_HEAVIEST_VW,
                 light_max_pairs=0, seed=0, stream=None, profile_load=False, streamed=False, strict_time=False,
                 heavy_warp_cap=0, heavy_cta_cap=0, heavy_merge=0):
        """streamed: TTC_LOAD_STREAM (no light-triangle list; every count
        enumerates the triangles again and counts light ones as it finds them).
        strict_time: TTC_LOAD_STRICT_TIME (count a triple only if its three
        timestamps strictly increase).  heavy_merge: HEAVY_BINARY or
        HEAVY_MERGE for the one-CTA class (0: tuned, else binary)."""
        ptrs, m, flags, keep = _edge_ptrs(src, dst, t)
        if profile_load:
            flags |= LOAD_PROFILE
        if streamed:
            flags |= LOAD_STREAM
        if strict_time:
            flags |= LOAD_STRICT_TIME
        opts = LoadOpts(flags=flags, orientation=orientation, labeling=labeling, light_max_pairs=light_max_pairs,
                        heavy_warp_cap=heavy_warp_cap, heavy_cta_cap=heavy_cta_cap, heavy_merge=heavy_merge,
                        seed=seed, stream=stream)
        h = ctypes.c_void_p()
        check(lib().ttc_load_ex(ptrs[0], ptrs[1], ptrs[2], m, ctypes.byref(opts), ctypes.byref(h)))
        self._h = h
        del keep

    @property
    def handle(self):
        if not self._h:
            raise ValueError("graph was freed")
        return self._h

    def free(self):
        if getattr(self, "_h", None):
            lib().ttc_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def info(self) -> dict:
        s = GraphStats()
        check(lib().ttc_graph_info(self.handle, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in GraphStats._fields_}

    def count(self, delta) -> np.ndarray:
        d, dp = _deltas(delta)
        out = np.zeros(NUM_TYPES, dtype=np.uint64)
        check(lib().ttc_count(self.handle, dp, out.ctypes.data))
        return out

    def count_batch(self, deltas) -> np.ndarray:
        d, dp = _deltas(deltas)
        out = np.zeros((d.shape[0], NUM_TYPES), dtype=np.uint64)
        check(lib().ttc_count_batch(self.handle, dp, d.shape[0], out.ctypes.data))
        return out

    def count_shard(self, deltas, shard: int, nshards: int) -> np.ndarray:
        """Shard `shard` of `nshards` of count_batch (the shards' counts sum to it)."""
        d, dp = _deltas(deltas)
        out = np.zeros((d.shape[0], NUM_TYPES), dtype=np.uint64)
        check(lib().ttc_count_shard(self.handle, dp, d.shape[0], shard, nshards, out.ctypes.data))
        return out

    def count_batch_async(self, d_dev_ptr: int, k: int, out_dev_ptr: int, stream_ptr: int = 0):
        """Device pointers: k deltas (int64 x 3) in, k x 8 uint64 out."""
        check(lib().ttc_count_batch_async(self.handle, d_dev_ptr, k, out_dev_ptr, stream_ptr or None))

    def set_profiling(self, on: bool = True):
        check(lib().ttc_set_profiling(self.handle, 1 if on else 0))

    def profile(self):
        """[(kernel name, ms)] of the most recent count call."""
        buf = (KernelTime * 64)()
        n = lib().ttc_profile_read(self.handle, buf, 64)
        return [(buf[i].name.decode(), buf[i].ms) for i in range(n)]

    def count_grid(self, d13: int, d12, d23):
        """Counts at every (δ12, δ23) of the grid for one δ13:
        ([len(d12)][len(d23)][8] uint64, [len(d12)][len(d23)] cyclic share)."""
        a = np.ascontiguousarray(np.asarray(d12, dtype=np.int64).ravel())
        b = np.ascontiguousarray(np.asarray(d23, dtype=np.int64).ravel())
        out = np.zeros((a.size, b.size, 8), dtype=np.uint64)
        cyc = np.zeros((a.size, b.size), dtype=np.float64)
        check(lib().ttc_count_grid(self.handle, int(d13), a.ctypes.data, a.size, b.ctypes.data, b.size,
                                   out.ctypes.data, cyc.ctypes.data))
        return out, cyc

    def participation(self, delta):
        """ttc_count_participation: (per-vertex counts [n], per-pair counts
        [m_s]) of the delta-temporal triangles (all types) each vertex and
        each static pair (in pairs() order) belongs to."""
        d, dp = _deltas(delta)
        info = self.info()
        vert = np.zeros(info["n"], dtype=np.uint64)
        pair = np.zeros(info["m_s"], dtype=np.uint64)
        check(lib().ttc_count_participation(self.handle, dp, vert.ctypes.data if vert.size else None,
                                            pair.ctypes.data if pair.size else None))
        return vert, pair

    def pairs(self) -> np.ndarray:
        """ttc_graph_pairs: the static pairs (lo, hi) in the library's pair order, [m_s, 2]."""
        out = np.zeros((self.info()["m_s"], 2), dtype=np.uint32)
        check(lib().ttc_graph_pairs(self.handle, out.ctypes.data if out.size else None))
        return out

    def sample(self, delta, first: int, stride: int, cap: int):
        d, dp = _deltas(delta)
        tri = np.zeros((cap, 3), dtype=np.uint32)
        out = np.zeros((cap, NUM_TYPES), dtype=np.uint64)
        n = ctypes.c_uint64()
        check(lib().ttc_count_sample(self.handle, dp, first, stride, cap, tri.ctypes.data, out.ctypes.data,
                                     ctypes.byref(n)))
        return tri[:n.value], out[:n.value]


def tune_light(src, dst, t, probe_deltas, stream=None, orientation=ORIENT_DEGENERACY, labeling=LABEL_HEAVIEST_VW):
    """ttc_tune_light: times load + count of the probe queries at each light
    threshold in TUNE_CANDIDATES, caches the fastest for graphs of this
    shape and returns (chosen threshold, {candidate: ms})."""
    ptrs, m, flags, keep = _edge_ptrs(src, dst, t)
    opts = LoadOpts(flags=flags, orientation=orientation, labeling=labeling, stream=stream)
    d, dp = _deltas(probe_deltas)
    chosen = ctypes.c_uint32()
    ms = (ctypes.c_float * len(TUNE_CANDIDATES))()
    check(lib().ttc_tune_light(ptrs[0], ptrs[1], ptrs[2], m, ctypes.byref(opts), dp, d.shape[0],
                               ctypes.byref(chosen), ms))
    del keep
    return int(chosen.value), {c: float(v) for c, v in zip(TUNE_CANDIDATES, ms)}


def tune_heavy(src, dst, t, probe_deltas, light_max_pairs=0, stream=None, orientation=ORIENT_DEGENERACY,
               labeling=LABEL_HEAVIEST_VW):
    """ttc_tune_heavy: times load + count of the probe queries at each (warp
    cap, CTA cap, search form) of TUNE_HEAVY_CANDIDATES at the given light
    threshold, caches the fastest and returns ((warp cap, CTA cap, search
    form) the loads used, {candidate: ms})."""
    ptrs, m, flags, keep = _edge_ptrs(src, dst, t)
    opts = LoadOpts(flags=flags, orientation=orientation, labeling=labeling, light_max_pairs=light_max_pairs,
                    stream=stream)
    d, dp = _deltas(probe_deltas)
    w, c, mg = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    ms = (ctypes.c_float * len(TUNE_HEAVY_CANDIDATES))()
    check(lib().ttc_tune_heavy(ptrs[0], ptrs[1], ptrs[2], m, ctypes.byref(opts), dp, d.shape[0],
                               ctypes.byref(w), ctypes.byref(c), ctypes.byref(mg), ms))
    del keep
    return ((int(w.value), int(c.value), int(mg.value)),
            {cand: float(v) for cand, v in zip(TUNE_HEAVY_CANDIDATES, ms)})


def count_stream(edge_lists, deltas, budget_bytes=0, orientation=ORIENT_DEGENERACY, labeling=LABEL_HEAVIEST_VW,
                 light_max_pairs=0):
    """ttc_count_stream: counts many graphs given as host (src, dst, t)
    arrays, loaded in order into batches whose device footprint stays within
    budget_bytes (0: half of the free device memory), one ttc_count_multi
    launch per batch.  Returns (counts [G, 8], number of batches)."""
    G = len(edge_lists)
    d, dp = _deltas(deltas)
    if d.shape[0] != G:
        raise ValueError("one delta-triple per graph")
    keep, ms = [], []
    ps = [(ctypes.c_void_p * G)() for _ in range(3)]
    for i, (src, dst, t) in enumerate(edge_lists):
        if _is_torch(src):
            raise ValueError("count_stream takes host arrays")
        ptrs, m, _, k = _edge_ptrs(src, dst, t)
        for j in range(3):
            ps[j][i] = ptrs[j]
        ms.append(m)
        keep.append(k)
    m_arr = np.asarray(ms, dtype=np.uint64)
    opts = LoadOpts(orientation=orientation, labeling=labeling, light_max_pairs=light_max_pairs)
    out = np.zeros((G, NUM_TYPES), dtype=np.uint64)
    nb = ctypes.c_uint32(0)
    check(lib().ttc_count_stream(ps[0], ps[1], ps[2], m_arr.ctypes.data, dp, G, ctypes.byref(opts),
                                 int(budget_bytes), out.ctypes.data, ctypes.byref(nb)))
    del keep
    return out, int(nb.value)


def count_multi(graphs, deltas) -> np.ndarray:
    d, dp = _deltas(deltas)
    G = len(graphs)
    if d.shape[0] != G:
        raise ValueError("one delta-triple per graph")
    hs = (ctypes.c_void_p * G)(*[g.handle.value for g in graphs])
    out = np.zeros((G, NUM_TYPES), dtype=np.uint64)
    check(lib().ttc_count_multi(hs, dp, G, out.ctypes.data))
    return out


class Server:
    """Continuous-batching server (``ttc_server_*``)."""

    def __init__(self, hbm_reserve_bytes=0, max_batch=0, max_queue=0, streams=0, wait_limit_us=0):
        o = ServerOpts(hbm_reserve_bytes, max_batch, max_queue, streams, wait_limit_us)
        h = lib().ttc_server_create(ctypes.byref(o))
        if not h:
            raise TTCError(-8, last_error())
        self._h = ctypes.c_void_p(h)

    def close(self):
        if getattr(self, "_h", None):
            lib().ttc_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, src, dst, t) -> int:
        ptrs, m, flags, keep = _edge_ptrs(src, dst, t)
        if flags:
            raise ValueError("the server takes host arrays")
        gid = ctypes.c_uint64()
        check(lib().ttc_serve_load(self._h, ptrs[0], ptrs[1], ptrs[2], m, ctypes.byref(gid)))
        return gid.value

    def submit(self, graph_id: int, delta) -> int:
        d, dp = _deltas(delta)
        tk = ctypes.c_uint64()
        check(lib().ttc_serve_submit(self._h, graph_id, dp, ctypes.byref(tk)))
        return tk.value

    def poll(self, ticket: int):
        """Returns (counts, latency_s) or None while pending."""
        out = np.zeros(NUM_TYPES, dtype=np.uint64)
        lat = ctypes.c_double()
        st = check(lib().ttc_serve_poll(self._h, ticket, out.ctypes.data, ctypes.byref(lat)))
        if st == PENDING:
            return None
        return out, lat.value

    def pause(self, paused: bool = True):
        check(lib().ttc_serve_pause(self._h, 1 if paused else 0))

    def set_reserve(self, hbm_reserve_bytes: int):
        check(lib().ttc_serve_set_reserve(self._h, int(hbm_reserve_bytes)))

    def drain(self, timeout_s: float = 60.0):
        check(lib().ttc_serve_drain(self._h, timeout_s))

    def info(self) -> dict:
        s = ServerStats()
        check(lib().ttc_server_info(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in ServerStats._fields_}


def release_cached() -> int:
    """Return the library's cached device blocks to the device; bytes released."""
    out = ctypes.c_uint64(0)
    check(lib().ttc_release_cached(ctypes.byref(out)))
    return int(out.value)


def memory_info() -> dict:
    """Free device memory and the library pool's mapped / handed-out bytes."""
    f, r, u = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
    check(lib().ttc_memory_info(ctypes.byref(f), ctypes.byref(r), ctypes.byref(u)))
    return {"device_free": int(f.value), "pool_reserved": int(r.value), "pool_used": int(u.value),
            "admission_free": int(f.value) + max(0, int(r.value) - int(u.value))}


def debug_fail_alloc_after(n: int):
    lib().ttc_debug_fail_alloc_after(n)


def launch_count() -> int:
    return int(lib().ttc_debug_launch_count())
