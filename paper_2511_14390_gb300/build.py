"""Build libdfilt.so in-tree: every CUDA translation unit compiled for sm_103a in
parallel, then linked into one shared library with the C ABI of include/dfilt.h.

    python -m paper_2511_14390_gb300.build [--force] [-v] [--debug]

--debug also builds libdfilt_debug.so: the same library with the device-side index
checks of the decoupled path compiled in (-DDFILT_DEBUG; the translation units that
hold them are recompiled, the others are shared with the release build).
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libdfilt.so")
DEBUG_LIB = os.path.join(PKG, "libdfilt_debug.so")
BUCKETS = [2, 4, 8, 16, 32, 64]
HI_BUCKETS = [8, 16, 32, 64]   # the decoupled high-order path
# (object name, source, extra defines): the chunked kernels compile once per state bucket
UNITS = ([("api", "api.cu", []), ("seq", "seq.cu", []), ("chunk_setup", "chunk_setup.cu", []),
          ("chunk_dispatch", "chunk_dispatch.cu", []), ("noalloc", "noalloc.cu", []),
          ("jvp", "jvp.cu", []), ("ss", "ss.cu", []), ("diag", "diag.cu", []), ("tv", "tv.cu", []),
          ("ic", "ic.cu", [])]
         + [(f"chunk_fwd_{m}", "chunk_fwd.cu", [f"-DDFILT_MB={m}"]) for m in BUCKETS]
         + [(f"chunk_bwd_{m}", "chunk_bwd.cu", [f"-DDFILT_MB={m}"]) for m in BUCKETS]
         + [(f"hi_tc_{m}", "hi_tc.cu", [f"-DDFILT_MB={m}"]) for m in HI_BUCKETS]
         + [(f"hi_scan_{m}", "hi_scan.cu", [f"-DDFILT_MB={m}"]) for m in HI_BUCKETS])
# the units whose code changes under -DDFILT_DEBUG (the checks and their entry points)
DEBUG_UNITS = {"api", *(f"hi_tc_{m}" for m in HI_BUCKETS), *(f"hi_scan_{m}" for m in HI_BUCKETS)}
HEADERS = ["common.cuh", "kernels.h", "chunk.cuh", "chunk_pipe.cuh", "dword.cuh", "hi.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-fmad=true",
              "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _newest_dep() -> float:
    deps = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "dfilt.h"),
                                                        os.path.abspath(__file__)]
    return max(os.path.getmtime(p) for p in deps)


def _compile(unit, extra: list[str], verbose: bool, prefix: str = "") -> str:
    name, src, defs = unit
    obj = os.path.join(OUT, prefix + name + ".o")
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *defs, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and (r.stdout or r.stderr):
        print(r.stdout + r.stderr, flush=True)
    return obj


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compile (when stale) and link libdfilt.so; returns its path."""
    extra = extra or []
    os.makedirs(OUT, exist_ok=True)
    dep_time = _newest_dep()
    todo = []
    for u in UNITS:
        obj = os.path.join(OUT, u[0] + ".o")
        if (force or extra or not os.path.exists(obj) or os.path.getmtime(obj) < max(
                dep_time, os.path.getmtime(os.path.join(CSRC, u[1])))):
            todo.append(u)
    workers = max(1, min(len(UNITS), os.cpu_count() or 4))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        list(ex.map(lambda u: _compile(u, extra, verbose), todo))
    objs = [os.path.join(OUT, u[0] + ".o") for u in UNITS]
    if force or todo or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(o) for o in objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


def build_debug(force: bool = False, verbose: bool = False) -> str:
    """Build (when stale) libdfilt_debug.so: the release objects, with the units in
    DEBUG_UNITS recompiled with -DDFILT_DEBUG; returns its path."""
    build(verbose=verbose)
    dep_time = _newest_dep()
    units = [u for u in UNITS if u[0] in DEBUG_UNITS]
    todo = [u for u in units
            if force or not os.path.exists(os.path.join(OUT, "dbg_" + u[0] + ".o"))
            or os.path.getmtime(os.path.join(OUT, "dbg_" + u[0] + ".o")) < max(
                dep_time, os.path.getmtime(os.path.join(CSRC, u[1])))]
    workers = max(1, min(len(todo) or 1, os.cpu_count() or 4))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        list(ex.map(lambda u: _compile(u, ["-DDFILT_DEBUG"], verbose, "dbg_"), todo))
    objs = [os.path.join(OUT, ("dbg_" if u[0] in DEBUG_UNITS else "") + u[0] + ".o") for u in UNITS]
    if force or todo or not os.path.exists(DEBUG_LIB) or os.path.getmtime(DEBUG_LIB) < max(
            os.path.getmtime(o) for o in objs):
        tmp = DEBUG_LIB + f".{os.getpid()}.tmp"
        subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"], check=True)
        os.replace(tmp, DEBUG_LIB)
    return DEBUG_LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("-v", "--verbose", action="store_true")
    ap.add_argument("--ptxas-v", action="store_true", help="print register/spill usage")
    ap.add_argument("--debug", action="store_true", help="also build libdfilt_debug.so")
    a = ap.parse_args()
    extra = ["-Xptxas", "-v"] if a.ptxas_v else []
    print(build(force=a.force, verbose=a.verbose or a.ptxas_v, extra=extra))
    if a.debug:
        print(build_debug(force=a.force, verbose=a.verbose))
    sys.exit(0)
