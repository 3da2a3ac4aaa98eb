"""Python handle on the plain CPU oracle (``ttc_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product library never
imports this package, and this package imports nothing from the product.

``build()`` compiles ``ttc_oracle.c`` with gcc (``-O2 -fopenmp``) into
``oracle/_build/libttc_oracle.so``.  Every function takes numpy arrays
``src`` (uint32), ``dst`` (uint32), ``t`` (int64) and delta-triples given as
``(d13, d12, d23)``, and returns uint64 counts with slot k-1 = type T_k.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ttc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libttc_oracle.so")
_lib = None

OK, ERR_INVALID, ERR_NOMEM, ERR_OVERFLOW = 0, -1, -3, -6


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        p = ctypes.c_void_p
        u64, u32, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        lib.ttc_oracle_bruteforce.argtypes = [p, p, p, u64, p, u32, p]
        lib.ttc_oracle_bruteforce_ex.argtypes = [p, p, p, u64, p, u32, i32, p]
        lib.ttc_oracle_count.argtypes = [p, p, p, u64, p, u32, i32, p]
        lib.ttc_oracle_count_ex.argtypes = [p, p, p, u64, p, u32, i32, i32, p]
        lib.ttc_oracle_count_part.argtypes = [p, p, p, u64, p, u32, i32, u32, u32, p]
        lib.ttc_oracle_count_triangles.argtypes = [p, p, p, u64, p, u64, p, u32, i32, p]
        lib.ttc_oracle_stats.argtypes = [p, p, p, u64, i32, p]
        lib.ttc_oracle_count_fwd.argtypes = [p, p, p, u64, p, u32, i32, i32, p]
        lib.ttc_oracle_stats_fwd.argtypes = [p, p, p, u64, i32, p]
        for f in (lib.ttc_oracle_bruteforce, lib.ttc_oracle_bruteforce_ex, lib.ttc_oracle_count,
                  lib.ttc_oracle_count_ex, lib.ttc_oracle_count_part,
                  lib.ttc_oracle_count_triangles, lib.ttc_oracle_stats, lib.ttc_oracle_count_fwd,
                  lib.ttc_oracle_stats_fwd):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _edges(src, dst, t):
    src = np.ascontiguousarray(src, dtype=np.uint32)
    dst = np.ascontiguousarray(dst, dtype=np.uint32)
    t = np.ascontiguousarray(t, dtype=np.int64)
    if not (src.shape == dst.shape == t.shape) or src.ndim != 1:
        raise ValueError("src, dst, t must be 1-D arrays of equal length")
    return src, dst, t


def _deltas(deltas):
    d = np.ascontiguousarray(np.asarray(deltas, dtype=np.int64).reshape(-1, 3))
    return d


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a.size else None


def _check(rc, allow_overflow=False):
    if rc == OK or (allow_overflow and rc == ERR_OVERFLOW):
        return
    raise OracleError({ERR_INVALID: "invalid argument", ERR_NOMEM: "out of memory",
                       ERR_OVERFLOW: "count exceeds 2^64-1"}.get(rc, "error %d" % rc))


def bruteforce(src, dst, t, deltas, strict: bool = False):
    """O0: every edge triple checked against Def. 1.  Returns [k][8].
    strict: t1 < t2 < t3 literally (no two edges of a counted triple share a
    timestamp) instead of key order."""
    src, dst, t = _edges(src, dst, t)
    d = _deltas(deltas)
    out = np.zeros((d.shape[0], 8), dtype=np.uint64)
    _check(_load().ttc_oracle_bruteforce_ex(_ptr(src), _ptr(dst), _ptr(t), src.size,
                                            _ptr(d), d.shape[0], int(bool(strict)), _ptr(out)))
    return out


def count(src, dst, t, deltas, threads: int = 0, strict: bool = False):
    """O1: plain adjacency + Lemma 1 summed directly.  Returns [k][8].
    strict: as for bruteforce."""
    src, dst, t = _edges(src, dst, t)
    d = _deltas(deltas)
    out = np.zeros((d.shape[0], 8), dtype=np.uint64)
    _check(_load().ttc_oracle_count_ex(_ptr(src), _ptr(dst), _ptr(t), src.size,
                                       _ptr(d), d.shape[0], int(threads), int(bool(strict)), _ptr(out)))
    return out


def count_fwd(src, dst, t, deltas, threads: int = 0, strict: bool = False):
    """O1 with the static triangles found by the forward rule (pairs oriented
    by (degree, id)) instead of plain adjacency: the same counts, in time that
    suits graphs with hubs.  Returns [k][8]."""
    src, dst, t = _edges(src, dst, t)
    d = _deltas(deltas)
    out = np.zeros((d.shape[0], 8), dtype=np.uint64)
    _check(_load().ttc_oracle_count_fwd(_ptr(src), _ptr(dst), _ptr(t), src.size,
                                        _ptr(d), d.shape[0], int(threads), int(bool(strict)), _ptr(out)))
    return out


def count_part(src, dst, t, deltas, part: int, nparts: int, threads: int = 0):
    """O1 over the triangles whose smallest vertex id is part mod nparts
    (the parts partition the triangles).  Returns [k][8]."""
    src, dst, t = _edges(src, dst, t)
    d = _deltas(deltas)
    out = np.zeros((d.shape[0], 8), dtype=np.uint64)
    _check(_load().ttc_oracle_count_part(_ptr(src), _ptr(dst), _ptr(t), src.size, _ptr(d), d.shape[0],
                                         int(threads), int(part), int(nparts), _ptr(out)))
    return out


def count_triangles(src, dst, t, tris, deltas, threads: int = 0):
    """Per static triangle (given as vertex triples): returns [k][nd][8]."""
    src, dst, t = _edges(src, dst, t)
    tris = np.ascontiguousarray(np.asarray(tris, dtype=np.uint32).reshape(-1, 3))
    d = _deltas(deltas)
    out = np.zeros((tris.shape[0], d.shape[0], 8), dtype=np.uint64)
    _check(_load().ttc_oracle_count_triangles(_ptr(src), _ptr(dst), _ptr(t), src.size,
                                              _ptr(tris), tris.shape[0], _ptr(d), d.shape[0],
                                              int(threads), _ptr(out)))
    return out


def stats(src, dst, t, threads: int = 0):
    """Static statistics: dict with n, m, m_s, tau, sigma_max, work_bytes and
    prod (= total count when every window is unbounded)."""
    src, dst, t = _edges(src, dst, t)
    s = np.zeros(8, dtype=np.uint64)
    _check(_load().ttc_oracle_stats(_ptr(src), _ptr(dst), _ptr(t), src.size, int(threads), _ptr(s)))
    return {"n": int(s[0]), "m": int(s[1]), "m_s": int(s[2]), "tau": int(s[3]),
            "sigma_max": int(s[4]), "work_bytes": int(s[5]),
            "prod": int(s[6]) + (int(s[7]) << 64)}


def stats_fwd(src, dst, t, threads: int = 0):
    """stats() with the triangles found by the forward rule."""
    src, dst, t = _edges(src, dst, t)
    s = np.zeros(8, dtype=np.uint64)
    _check(_load().ttc_oracle_stats_fwd(_ptr(src), _ptr(dst), _ptr(t), src.size, int(threads), _ptr(s)))
    return {"n": int(s[0]), "m": int(s[1]), "m_s": int(s[2]), "tau": int(s[3]),
            "sigma_max": int(s[4]), "work_bytes": int(s[5]),
            "prod": int(s[6]) + (int(s[7]) << 64)}
