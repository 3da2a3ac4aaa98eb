"""Compiles the CUDA library in-tree: csrc/*.cu -> _build/libttc.so.

One ``-gencode arch=compute_103a,code=sm_103a`` target (GB300), translation
units compiled in parallel, then linked as a shared library with a C ABI
(``include/ttc.h``).  Rebuilds only what changed.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libttc.so")
# the build with device index checks (TTC_DEBUG_BOUNDS) goes beside it
DEBUG_OUT = os.path.join(HERE, "_build_debug")
DEBUG_LIB = os.path.join(DEBUG_OUT, "libttc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-Wno-deprecated-gpu-targets"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the ttc CUDA library cannot be built")


def _headers():
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(HERE, "..", "include", "*.h"))
    return max((os.path.getmtime(h) for h in hs), default=0.0)


# The light kernel's sources: count.cu up to its heavy-bin section (the file's
# head and the light bin), graph.cuh up to the host-side graph handle (the
# key format, TriRec and GraphView, which the kernels read), and the device
# helpers in full.
_LIGHT_SOURCES = [("count.cu", "// ---------------------------------------------------------------- heavy: per-edge math"),
                  ("count_dev.cuh", None), ("graph.cuh", "struct ttc_graph {"), ("common.cuh", None)]


def count_source_hash(read=None) -> str:
    """Short hash of the light count kernel's source (the parts listed in
    _LIGHT_SOURCES); the ncu profile of that kernel records it, so a stale
    profile can be told from a current one while changes elsewhere (the
    heavy bins, host code) leave it valid.  read(name) -> bytes overrides the
    source files (to hash another revision)."""
    import hashlib
    h = hashlib.sha1()
    for f, stop in _LIGHT_SOURCES:
        if read is not None:
            data = read(f)
        else:
            with open(os.path.join(CSRC, f), "rb") as fh:
                data = fh.read()
        if stop is not None:
            cut = data.find(stop.encode())
            if cut < 0:
                raise RuntimeError("%s: marker %r not found" % (f, stop))
            data = data[:cut]
        h.update(data)
    return h.hexdigest()[:12]


def build(force: bool = False, verbose: bool = False, debug_bounds: bool = False) -> str:
    """Builds _build/libttc.so, or with debug_bounds the library whose count
    kernels check their indices on the device (_build_debug/libttc.so)."""
    out_dir = DEBUG_OUT if debug_bounds else OUT
    lib_path = DEBUG_LIB if debug_bounds else LIB
    os.makedirs(out_dir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    hdr_t = _headers()
    cc = nvcc()
    defs = ["-DTTC_COUNT_HASH=\"%s\"" % count_source_hash()] + (["-DTTC_DEBUG_BOUNDS=1"] if debug_bounds else [])

    # the object that embeds the count hash is rebuilt whenever the hash changes
    stamp = os.path.join(out_dir, "count_hash.txt")
    old_hash = open(stamp).read().strip() if os.path.exists(stamp) else ""

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.basename(src) + ".o")
        stale_hash = os.path.basename(src) == "capi.cu" and old_hash != count_source_hash()
        if (not force and not stale_hash and os.path.exists(obj)
                and os.path.getmtime(obj) >= max(os.path.getmtime(src), hdr_t)):
            return obj, False
        cmd = [cc, *ARCH, *FLAGS, *defs, "-c", src, "-o", obj + ".tmp"]
        if src.endswith(".cpp"):
            cmd = [cc, *FLAGS, "-x", "c++", "-c", src, "-o", obj + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s%s" % (os.path.basename(src), r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        os.replace(obj + ".tmp", obj)
        return obj, True

    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        results = list(ex.map(compile_one, srcs))
    with open(stamp, "w") as fh:
        fh.write(count_source_hash())
    objs = [o for o, _ in results]
    changed = any(c for _, c in results)
    if force or changed or not os.path.exists(lib_path):
        tmp = lib_path + ".%d.tmp" % os.getpid()
        cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread", "-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
