"""Build libdfilt.so in-tree: every CUDA translation unit compiled for sm_103a in
parallel, then linked into one shared library with the C ABI of include/dfilt.h.

    python -m paper_2511_14390_gb300.build [--force] [-v]
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


def _compile(unit, extra: list[str], verbose: bool) -> str:
    name, src, defs = unit
    obj = os.path.join(OUT, name + ".o")
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


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("-v", "--verbose", action="store_true")
    ap.add_argument("--ptxas-v", action="store_true", help="print register/spill usage")
    a = ap.parse_args()
    extra = ["-Xptxas", "-v"] if a.ptxas_v else []
    print(build(force=a.force, verbose=a.verbose or a.ptxas_v, extra=extra))
    sys.exit(0)
