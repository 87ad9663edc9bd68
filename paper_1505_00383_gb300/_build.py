"""Build the CUDA library libht.so in-tree for sm_103a.

Each translation unit (and each precision of the templated kernels) compiles
as its own nvcc process, in parallel; the objects link into one shared library
with the CUDA runtime linked statically.  No CMake.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libht.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC,
         "--expt-relaxed-constexpr"]

# (source, extra defines, object name)
UNITS = [
    ("ht_api.cu", [], "ht_api.o"),
    ("ht_bench.cu", [], "ht_bench.o"),
    ("ht_evaldiff.cu", ["-DHT_LIMBS=1"], "ht_evaldiff_1.o"),
    ("ht_evaldiff.cu", ["-DHT_LIMBS=2"], "ht_evaldiff_2.o"),
    ("ht_evaldiff.cu", ["-DHT_LIMBS=4"], "ht_evaldiff_4.o"),
    ("ht_track.cu", ["-DHT_LIMBS=1"], "ht_track_1.o"),
    ("ht_track.cu", ["-DHT_LIMBS=2"], "ht_track_2.o"),
    ("ht_track.cu", ["-DHT_LIMBS=4"], "ht_track_4.o"),
    ("ht_track_host.cu", [], "ht_track_host.o"),
    ("ht_noalloc.cu", [], "ht_noalloc.o"),
    ("ht_mlp.cu", [], "ht_mlp.o"),
    ("ht_refine.cu", [], "ht_refine.o"),
    ("ht_unfused.cu", ["-DHT_LIMBS=1"], "ht_unfused_1.o"),
    ("ht_unfused.cu", ["-DHT_LIMBS=2"], "ht_unfused_2.o"),
    ("ht_unfused.cu", ["-DHT_LIMBS=4"], "ht_unfused_4.o"),
]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libht.so")
    return p


def _sources_mtime() -> float:
    t = 0.0
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            t = max(t, os.path.getmtime(os.path.join(d, f)))
    return max(t, os.path.getmtime(__file__))


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _sources_mtime():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()

    def compile_one(unit):
        src, defs, obj = unit
        cmd = [cc] + ARCH + FLAGS + defs + ["-c", os.path.join(CSRC, src), "-o", os.path.join(OUT_DIR, obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr[-4000:]))
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    jobs = jobs or min(len(UNITS), max(1, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + [os.path.join(OUT_DIR, o) for o in objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s" % r.stderr[-4000:])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
