"""FP64 CPU oracle for batched direct-form IIR filters (test infrastructure).

This package is TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline / ``--impl reference`` legs may import it.  The
product path (``paper_2511_14390_gb300``) never imports it and shares no code
with it.

What it computes (paper, "Accelerating Automatic Differentiation of Direct Form
Digital Filters"):

* forward  -- Eq. rtf as the TDF-II state recursion (Sec. 2), initial state ``zi``
  in the TDF-II (SciPy ``lfilter``) convention; a second formulation (initial
  state injected into the all-pole input) cross-checks it;
* backward -- the reverse-time adjoint of Sec. 3.1 (Eqs. dLdz, dLdx, dLdvBA, with
  the boundary condition of App. A) written as scalar difference equations;
* forward mode (JVP) -- the TDF-II recursion carried with its derivative along
  tangents of every input (the forward-mode derivative Sec. 5 mentions);
* direct-form initial conditions -- the difference equation extended into negative
  time with given past inputs and outputs, and its gradients.

The heavy loops live in ``dfilt_oracle.c`` (plain C, FP64, OpenMP over channels);
``pyref.py`` holds a pure-Python FP64 restatement for tiny cases, ``statespace.py``
the state-space operator of App. B, and ``chunked.py`` an FP64 model of the chunk
algebra.  Every function states the passage it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dfilt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libdfilt_oracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``dfilt_oracle.c`` into ``oracle/_build/libdfilt_oracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
           "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def compile_variant(src_text: str, out_path: str) -> str:
    """Compile an arbitrary C source text with the oracle's flags (used by tests
    that plant a mistake in a copy of the oracle to show the pins catch it)."""
    c_path = out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
                    "-fno-fast-math", "-ffp-contract=off", c_path, "-o", out_path, "-lm"],
                   check=True)
    return out_path


def _bind(lib):
    P = ctypes.c_void_p
    i64, i32 = ctypes.c_int64, ctypes.c_int
    lib.oracle_forward_ragged.argtypes = [P, P, P, P, P, P, P, P, i64, i32, i32, i32, i32]
    lib.oracle_forward_ragged.restype = i32
    lib.oracle_backward_ragged.argtypes = [P, P, P, P, P, P, P, P, P, P, P, P, i64, i32, i32, i32]
    lib.oracle_backward_ragged.restype = i32
    lib.oracle_jvp.argtypes = [P, P, P, P, P, P, P, P, P, P, i64, i64, i32, i32, i32]
    lib.oracle_jvp.restype = i32
    lib.oracle_forward_df1.argtypes = [P, P, P, P, P, P, i64, i64, i32, i32, i32]
    lib.oracle_forward_df1.restype = i32
    lib.oracle_backward_df1.argtypes = [P, P, P, P, P, P, P, P, P, P, P, P, i64, i64, i32, i32,
                                        i32]
    lib.oracle_backward_df1.restype = i32
    lib.oracle_forward_tv.argtypes = [P, P, P, P, P, i64, i64, i32, i32, i32]
    lib.oracle_forward_tv.restype = i32
    lib.oracle_backward_tv.argtypes = [P, P, P, P, P, P, P, P, P, P, i64, i64, i32, i32, i32]
    lib.oracle_backward_tv.restype = i32
    lib.oracle_max_threads.argtypes = []
    lib.oracle_max_threads.restype = i32
    return lib


def load(path: str | None = None):
    """Load the oracle library (building it if needed).  ``path`` loads another
    compiled variant instead (returned, not cached)."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def max_threads() -> int:
    return int(load().oracle_max_threads())


# ----------------------------------------------------------------------------
# array helpers
# ----------------------------------------------------------------------------

def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _uniform_meta(B: int, T: int, N: int, M: int):
    offs = np.arange(B + 1, dtype=np.int64) * T
    Ms = np.full(B, M, dtype=np.int32)
    Ns = np.full(B, N, dtype=np.int32)
    return offs, Ms, Ns


# ----------------------------------------------------------------------------
# fixed-shape batch  x[B,T], b[B,N+1], a[B,M], zi[B,M]
# ----------------------------------------------------------------------------

def forward(x, b, a, zi=None, *, form: str = "tdf2", nthreads: int = 0, lib=None):
    """y[B,T] in FP64 (Eq. rtf; TDF-II recursion or the injection form)."""
    x, b, a = _f64(x), _f64(b), _f64(a)
    B, T = x.shape
    N, M = b.shape[1] - 1, a.shape[1]
    zi = None if zi is None else _f64(zi)
    offs, Ms, Ns = _uniform_meta(B, T, N, M)
    return forward_ragged(x.reshape(-1), offs, Ms, Ns, b, a, zi, form=form,
                          nthreads=nthreads, lib=lib).reshape(B, T)


def backward(gy, x, y, b, a, *, nthreads: int = 0, lib=None):
    """(grad_x[B,T], grad_b[B,N+1], grad_a[B,M], grad_zi[B,M]) in FP64 (Sec. 3.1)."""
    gy, x, y, b, a = _f64(gy), _f64(x), _f64(y), _f64(b), _f64(a)
    B, T = x.shape
    N, M = b.shape[1] - 1, a.shape[1]
    offs, Ms, Ns = _uniform_meta(B, T, N, M)
    gx, gb, ga, gzi = backward_ragged(gy.reshape(-1), x.reshape(-1), y.reshape(-1),
                                      offs, Ms, Ns, b, a, nthreads=nthreads, lib=lib)
    return gx.reshape(B, T), gb, ga, gzi


def jvp(x, b, a, zi=None, dx=None, db=None, da=None, dzi=None, *, nthreads: int = 0,
        lib=None):
    """(y[B,T], dy[B,T]) in FP64: the forward and its directional derivative along the
    tangents (dx, db, da, dzi) -- forward mode, the TDF-II recursion differentiated
    step by step (Sec. 5 notes forward mode follows like the reverse mode).  A tangent
    left as None is zero."""
    lib = lib or load()
    x, b, a = _f64(x), _f64(b), _f64(a)
    B, T = x.shape
    N, M = b.shape[1] - 1, a.shape[1]
    zi, dx, db, da, dzi = (None if v is None else _f64(v) for v in (zi, dx, db, da, dzi))
    y = np.zeros_like(x)
    dy = np.zeros_like(x)
    rc = lib.oracle_jvp(_ptr(x), _ptr(b), _ptr(a), _ptr(zi), _ptr(dx), _ptr(db), _ptr(da),
                        _ptr(dzi), _ptr(y), _ptr(dy), B, T, N, M, int(nthreads))
    if rc != 0:
        raise MemoryError("oracle jvp: allocation failed")
    return y, dy


def forward_df1(x, b, a, xpast, ypast, *, nthreads: int = 0, lib=None):
    """y[B,T] in FP64 with direct-form initial conditions: past inputs xpast[B,N]
    (x[-1], x[-2], ...) and past outputs ypast[B,M] (y[-1], ...), the difference
    equation of Eq. rtf extended into negative time."""
    lib = lib or load()
    x, b, a, ypast = _f64(x), _f64(b), _f64(a), _f64(ypast)
    B, T = x.shape
    N, M = b.shape[1] - 1, a.shape[1]
    xpast = None if (xpast is None or N == 0) else _f64(xpast)
    y = np.zeros_like(x)
    lib.oracle_forward_df1(_ptr(x), _ptr(b), _ptr(a), _ptr(xpast), _ptr(ypast), _ptr(y), B, T,
                           N, M, int(nthreads))
    return y


def backward_df1(gy, x, y, b, a, xpast, ypast, *, nthreads: int = 0, lib=None):
    """(grad_x, grad_b, grad_a, grad_xpast, grad_ypast) in FP64 for forward_df1."""
    lib = lib or load()
    gy, x, y, b, a, ypast = _f64(gy), _f64(x), _f64(y), _f64(b), _f64(a), _f64(ypast)
    B, T = x.shape
    N, M = b.shape[1] - 1, a.shape[1]
    xpast = None if (xpast is None or N == 0) else _f64(xpast)
    gx = np.zeros_like(x)
    gb, ga = np.zeros((B, N + 1)), np.zeros((B, M))
    gxp, gyp = np.zeros((B, N)), np.zeros((B, M))
    rc = lib.oracle_backward_df1(_ptr(gy), _ptr(x), _ptr(y), _ptr(b), _ptr(a), _ptr(xpast),
                                 _ptr(ypast), _ptr(gx), _ptr(gb), _ptr(ga),
                                 _ptr(gxp) if N > 0 else None, _ptr(gyp), B, T, N, M,
                                 int(nthreads))
    if rc != 0:
        raise MemoryError("oracle backward_df1: allocation failed")
    return gx, gb, ga, gxp, gyp


def forward_tv(x, b, a, ypast=None, *, nthreads: int = 0, lib=None):
    """Parameter-varying direct form, FP64: x[B,T], b[B,T,N+1], a[B,T,M] (the
    coefficients of each output sample), ypast[B,M] (y[-1], ..., y[-M]) or None."""
    lib = lib or load()
    x, b, a = _f64(x), _f64(b), _f64(a)
    B, T = x.shape
    N, M = b.shape[2] - 1, a.shape[2]
    yp = None if ypast is None else _f64(ypast)
    y = np.zeros_like(x)
    lib.oracle_forward_tv(_ptr(x), _ptr(b), _ptr(a), _ptr(yp), _ptr(y), B, T, N, M, int(nthreads))
    return y


def backward_tv(gy, x, y, b, a, ypast=None, *, nthreads: int = 0, lib=None):
    """(grad_x [B,T], grad_b [B,T,N+1], grad_a [B,T,M], grad_ypast [B,M]) in FP64 for
    forward_tv."""
    lib = lib or load()
    gy, x, y, b, a = _f64(gy), _f64(x), _f64(y), _f64(b), _f64(a)
    B, T = x.shape
    N, M = b.shape[2] - 1, a.shape[2]
    yp = None if ypast is None else _f64(ypast)
    gx = np.zeros_like(x)
    gb, ga, gyp = np.zeros((B, T, N + 1)), np.zeros((B, T, M)), np.zeros((B, M))
    rc = lib.oracle_backward_tv(_ptr(gy), _ptr(x), _ptr(y), _ptr(b), _ptr(a), _ptr(yp), _ptr(gx),
                                _ptr(gb), _ptr(ga), _ptr(gyp), B, T, N, M, int(nthreads))
    if rc != 0:
        raise MemoryError("oracle backward_tv: allocation failed")
    return gx, gb, ga, gyp


# ----------------------------------------------------------------------------
# ragged batch: packed x[sum T_i], offs[B+1], Ms[B], Ns[B], b[B,Nmax+1], a[B,Mmax]
# ----------------------------------------------------------------------------

def forward_ragged(x, offs, Ms, Ns, b, a, zi=None, *, form: str = "tdf2",
                   nthreads: int = 0, lib=None):
    lib = lib or load()
    x, b, a = _f64(x), _f64(b), _f64(a)
    offs = np.ascontiguousarray(offs, dtype=np.int64)
    Ms = np.ascontiguousarray(Ms, dtype=np.int32)
    Ns = np.ascontiguousarray(Ns, dtype=np.int32)
    zi = None if zi is None else _f64(zi)
    B = len(Ms)
    Nmax, Mmax = b.shape[1] - 1, a.shape[1]
    y = np.zeros_like(x)
    rc = lib.oracle_forward_ragged(_ptr(x), _ptr(offs), _ptr(Ms), _ptr(Ns), _ptr(b), _ptr(a),
                                   _ptr(zi), _ptr(y), B, Nmax, Mmax,
                                   {"tdf2": 0, "injection": 1}[form], int(nthreads))
    if rc != 0:
        raise MemoryError("oracle forward: allocation failed")
    return y


def backward_ragged(gy, x, y, offs, Ms, Ns, b, a, *, nthreads: int = 0, lib=None):
    lib = lib or load()
    gy, x, y, b, a = _f64(gy), _f64(x), _f64(y), _f64(b), _f64(a)
    offs = np.ascontiguousarray(offs, dtype=np.int64)
    Ms = np.ascontiguousarray(Ms, dtype=np.int32)
    Ns = np.ascontiguousarray(Ns, dtype=np.int32)
    B = len(Ms)
    Nmax, Mmax = b.shape[1] - 1, a.shape[1]
    gx = np.zeros_like(x)
    gb = np.zeros((B, Nmax + 1))
    ga = np.zeros((B, Mmax))
    gzi = np.zeros((B, Mmax))
    rc = lib.oracle_backward_ragged(_ptr(gy), _ptr(x), _ptr(y), _ptr(offs), _ptr(Ms), _ptr(Ns),
                                    _ptr(b), _ptr(a), _ptr(gx), _ptr(gb), _ptr(ga), _ptr(gzi),
                                    B, Nmax, Mmax, int(nthreads))
    if rc != 0:
        raise MemoryError("oracle backward: allocation failed")
    return gx, gb, ga, gzi
