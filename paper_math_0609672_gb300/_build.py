"""Build librwpc.so (the CUDA library) in-tree for sm_103a.

Each translation unit is compiled by its own nvcc process, in parallel, then
linked into one shared library.  Objects are rebuilt when their source, the
headers or the flags change.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "librwpc.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--expt-relaxed-constexpr", "-I" + INCLUDE, "-I" + CSRC]
SOURCES = ["rw_api.cu", "rw_tables.cu", "rw_walk.cu", "rw_emit.cu", "rw_levels.cu", "rw_sched.cu",
           "rw_solve.cu", "rw_learn.cu", "rw_batch.cu", "rw_tune.cu", "rw_io.cu",
           "rw_adapt.cu"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _headers_digest():
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for f in sorted(os.listdir(d)):
            if f.endswith((".h", ".cuh")):
                with open(os.path.join(d, f), "rb") as fh:
                    h.update(f.encode() + fh.read())
    return h.hexdigest()


def _compile(nvcc, src, hdr_digest, extra):
    srcp = os.path.join(CSRC, src)
    obj = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
    stamp = obj + ".stamp"
    with open(srcp, "rb") as fh:
        key = hashlib.sha256(fh.read() + hdr_digest.encode() + " ".join(ARCH + FLAGS + extra).encode()).hexdigest()
    if os.path.exists(obj) and os.path.exists(stamp) and open(stamp).read() == key:
        return obj, False
    cmd = [nvcc] + ARCH + FLAGS + extra + ["-c", srcp, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    with open(stamp, "w") as fh:
        fh.write(key)
    return obj, True


def build(verbose=False, extra=()):
    """Compile every translation unit for sm_103a and link librwpc.so."""
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    hd = _headers_digest()
    extra = list(extra)
    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        results = list(ex.map(lambda s: _compile(nvcc, s, hd, extra), SOURCES))
    objs = [o for o, _ in results]
    changed = any(c for _, c in results) or not os.path.exists(LIB)
    if changed:
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    if verbose:
        print(f"built {LIB} ({'relinked' if changed else 'up to date'})")
    return LIB


if __name__ == "__main__":
    build(verbose=True)
