"""Thin Python binding of libdfilt.so (include/dfilt.h) plus a torch.autograd.Function.

Argument marshalling only: every step of the filter and its gradients runs in the
library's CUDA kernels.  PyTorch provides device memory and the current stream.
There is no fallback: if the library is missing or a call fails, this module raises.

Names follow the C ABI (``dfilt_forward``, ``dfilt_backward``, ...).  The operation
(paper: Eq. rtf; gradients Sec. 3.1) is, per channel,
    y[n] = sum_{k=0..N} b_k x[n-k] - sum_{k=1..M} a_k y[n-k]
with the initial state zi in the transposed-direct-form-II convention.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# DFILT_LIBRARY=debug loads the debug build (device-side index checks, build.py --debug)
LIB_PATH = os.path.join(_HERE, "libdfilt_debug.so" if os.environ.get("DFILT_LIBRARY") == "debug"
                        else "libdfilt.so")

ALGOS = {"auto": 0, "sequential": 1, "chunked": 2}
PRECISIONS = {"fp32": 0, "tf32": 1, "tf32x3": 3}
STATUS = {0: "DFILT_OK", 1: "DFILT_ERR_INVALID_ARG", 2: "DFILT_ERR_UNSUPPORTED",
          3: "DFILT_ERR_CUDA", 4: "DFILT_ERR_TIMEOUT", 5: "DFILT_ERR_NUMERIC",
          6: "DFILT_ERR_WORKSPACE", 7: "DFILT_ERR_BOUNDS"}
EXPORTS = ["dfilt_version", "dfilt_status_string", "dfilt_default_opts", "dfilt_workspace_size",
           "dfilt_forward", "dfilt_backward", "dfilt_workspace_size_ragged",
           "dfilt_forward_ragged", "dfilt_backward_ragged", "dfilt_sync_status",
           "dfilt_set_wait_limit", "dfilt_forward_noalloc", "dfilt_kernel_timing",
           "dfilt_kernel_timing_read", "dfilt_set_numeric_check", "dfilt_jvp_workspace_size",
           "dfilt_jvp", "dfilt_ss_workspace_size", "dfilt_ss_forward", "dfilt_ss_backward",
           "dfilt_ic_df1", "dfilt_ic_df1_backward", "dfilt_kernel_timing_read_classes",
           "dfilt_launch_count", "dfilt_tuning_set", "dfilt_tuning_get",
           "dfilt_diag_workspace_size", "dfilt_diag_forward", "dfilt_diag_backward",
           "dfilt_tv_workspace_size", "dfilt_tv_forward", "dfilt_tv_backward",
           "dfilt_debug_build", "dfilt_debug_set_limit"]


class DfiltError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, code)}")
        self.code = code


PATHS = {"auto": 0, "fused": 1, "decoupled": 2}


class Opts(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int), ("precision", ctypes.c_int),
                ("chunk_len", ctypes.c_int), ("fp64_scan", ctypes.c_int),
                ("path", ctypes.c_int), ("span_tiles", ctypes.c_int)]


def make_opts(algo="auto", precision="tf32x3", fp64_scan=-1, chunk_len=0, path="auto",
              span_tiles=0) -> Opts:
    if isinstance(algo, str):
        algo = ALGOS[algo]
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    if isinstance(path, str):
        path = PATHS[path]
    if algo == ALGOS["sequential"]:
        precision = PRECISIONS["fp32"]
    return Opts(int(algo), int(precision), int(chunk_len), int(fp64_scan), int(path),
                int(span_tiles))


_lib = None
_lock = threading.Lock()


def lib():
    """Load libdfilt.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -m paper_2511_14390_gb300.build`")
            L = ctypes.CDLL(LIB_PATH)
            P, i64, i32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
            PO = ctypes.POINTER(Opts)
            Psz = ctypes.POINTER(sz)
            L.dfilt_version.restype = i32
            L.dfilt_status_string.argtypes = [i32]
            L.dfilt_status_string.restype = ctypes.c_char_p
            L.dfilt_default_opts.argtypes = [PO]
            L.dfilt_workspace_size.argtypes = [i64, i64, i32, i32, PO, Psz, Psz, Psz]
            L.dfilt_workspace_size_ragged.argtypes = [i64, i64, i32, i32, PO, Psz, Psz, Psz]
            L.dfilt_forward.argtypes = [P, P, P, P, P, P, P, sz, i64, i64, i32, i32, PO, P]
            L.dfilt_backward.argtypes = [P, P, P, P, P, P, P, P, P, P, P, P, sz, i64, i64, i32,
                                         i32, PO, P]
            L.dfilt_forward_ragged.argtypes = [P, P, P, P, P, P, P, P, P, P, sz, i64, i64, i32,
                                               i32, PO, P]
            L.dfilt_backward_ragged.argtypes = [P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, sz,
                                                i64, i64, i32, i32, PO, P]
            L.dfilt_sync_status.argtypes = [P]
            L.dfilt_set_wait_limit.argtypes = [i64]
            L.dfilt_debug_build.restype = i32
            L.dfilt_debug_set_limit.argtypes = [i64]
            L.dfilt_set_numeric_check.argtypes = [i32]
            L.dfilt_forward_noalloc.argtypes = [P, P, P, P, P, i64, i64, i32, i32, PO, P]
            L.dfilt_kernel_timing.argtypes = [i32]
            L.dfilt_jvp_workspace_size.argtypes = [i64, i64, i32, i32, PO, Psz]
            L.dfilt_jvp.argtypes = [P, P, P, P, P, P, P, P, P, P, sz, i64, i64, i32, i32, PO, P]
            L.dfilt_ss_workspace_size.argtypes = [i64, i64, i32, Psz, Psz]
            L.dfilt_ss_forward.argtypes = [P, P, P, P, P, sz, i64, i64, i32, P]
            L.dfilt_ss_backward.argtypes = [P, P, P, P, P, P, P, P, sz, i64, i64, i32, P]
            L.dfilt_diag_workspace_size.argtypes = [i64, i64, i32, Psz, Psz]
            L.dfilt_diag_forward.argtypes = [P, P, P, P, P, P, P, sz, i64, i64, i32, P]
            L.dfilt_diag_backward.argtypes = [P, P, P, P, P, P, P, P, P, P, sz, i64, i64, i32, P]
            L.dfilt_tv_workspace_size.argtypes = [i64, i64, i32, i32, Psz]
            L.dfilt_tv_forward.argtypes = [P, P, P, P, P, P, sz, i64, i64, i32, i32, P]
            L.dfilt_tv_backward.argtypes = [P, P, P, P, P, P, P, P, P, P, P, sz, i64, i64, i32,
                                            i32, P]
            L.dfilt_ic_df1.argtypes = [P, P, P, P, P, i64, i32, i32, P]
            L.dfilt_ic_df1_backward.argtypes = [P, P, P, P, P, P, P, P, P, i64, i32, i32, P]
            PD, PI = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
            L.dfilt_kernel_timing_read.argtypes = [PD, PI, PD, PI]
            L.dfilt_kernel_timing_read_classes.argtypes = [PD, PI]
            L.dfilt_launch_count.argtypes = [ctypes.POINTER(ctypes.c_int64)]
            L.dfilt_tuning_set.argtypes = [i32, i32, i32]
            L.dfilt_tuning_get.argtypes = [i32, PI, PI]
            for name in EXPORTS:
                getattr(L, name).restype = getattr(L, name).restype or i32
            L.dfilt_status_string.restype = ctypes.c_char_p
            _lib = L
    return _lib


def _check(code: int, where: str):
    if code != 0:
        raise DfiltError(code, where)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _f32(t, name):
    if t is None:
        return None
    if not t.is_cuda or t.dtype != torch.float32:
        raise TypeError(f"{name} must be a CUDA float32 tensor")
    return t.contiguous()


# ---------------------------------------------------------------------------
# C-ABI wrappers (same names as include/dfilt.h)
# ---------------------------------------------------------------------------

def dfilt_workspace_size(B, T, N, M, opts: Opts | None = None):
    o = opts or make_opts()
    f, s, w = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().dfilt_workspace_size(B, T, N, M, ctypes.byref(o), ctypes.byref(f),
                                      ctypes.byref(s), ctypes.byref(w)), "dfilt_workspace_size")
    return f.value, s.value, w.value


def dfilt_workspace_size_ragged(B, total, Nmax, Mmax, opts: Opts | None = None):
    o = opts or make_opts()
    f, s, w = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().dfilt_workspace_size_ragged(B, total, Nmax, Mmax, ctypes.byref(o),
                                             ctypes.byref(f), ctypes.byref(s), ctypes.byref(w)),
           "dfilt_workspace_size_ragged")
    return f.value, s.value, w.value


def _buf(nbytes, device):
    return torch.empty(max(int(nbytes), 16), dtype=torch.uint8, device=device)


def dfilt_forward(x, b, a, zi=None, *, opts: Opts | None = None, y=None, saved=None, ws=None,
                  want_saved=True, stream=None):
    """y[B,T] (and the `saved` chunk-state buffer) for a fixed-shape batch."""
    x, b, a, zi = _f32(x, "x"), _f32(b, "b"), _f32(a, "a"), _f32(zi, "zi")
    B, T = x.shape
    N, M = b.shape[1] - 1, a.shape[1]
    o = opts or make_opts()
    fws, sv, _ = dfilt_workspace_size(B, T, N, M, o)
    y = torch.empty_like(x) if y is None else y
    if want_saved and sv and saved is None:
        saved = _buf(sv, x.device)
    ws = _buf(fws, x.device) if ws is None else ws
    _check(lib().dfilt_forward(_ptr(x), _ptr(b), _ptr(a), _ptr(zi), _ptr(y),
                               _ptr(saved) if want_saved else None, _ptr(ws), ws.numel(),
                               B, T, N, M, ctypes.byref(o), _stream(stream)), "dfilt_forward")
    return y, (saved if want_saved and sv else None)


def dfilt_backward(gy, x, y, b, a, zi=None, saved=None, *, opts: Opts | None = None,
                   needs=(True, True, True, True), ws=None, stream=None):
    """(grad_x, grad_b, grad_a, grad_zi); entries not in `needs` are None."""
    gy, x, y = _f32(gy, "gy"), _f32(x, "x"), _f32(y, "y")
    b, a = _f32(b, "b"), _f32(a, "a")
    B, T = x.shape
    N, M = b.shape[1] - 1, a.shape[1]
    o = opts or make_opts()
    _, _, bws = dfilt_workspace_size(B, T, N, M, o)
    gx = torch.empty_like(x) if needs[0] else None
    gb = torch.empty_like(b) if needs[1] else None
    ga = torch.empty_like(a) if needs[2] else None
    gzi = torch.empty((B, M), dtype=torch.float32, device=x.device) if needs[3] else None
    ws = _buf(bws, x.device) if ws is None else ws
    _check(lib().dfilt_backward(_ptr(gy), _ptr(x), _ptr(y), _ptr(b), _ptr(a), _ptr(zi),
                                _ptr(saved), _ptr(gx), _ptr(gb), _ptr(ga), _ptr(gzi), _ptr(ws),
                                ws.numel(), B, T, N, M, ctypes.byref(o), _stream(stream)),
           "dfilt_backward")
    return gx, gb, ga, gzi


def dfilt_forward_ragged(x, offsets, Ms, Ns, b, a, zi=None, *, opts: Opts | None = None,
                         y=None, saved=None, ws=None, want_saved=True, stream=None):
    x, b, a, zi = _f32(x, "x"), _f32(b, "b"), _f32(a, "a"), _f32(zi, "zi")
    B = Ms.shape[0]
    total = x.shape[0]
    Nmax, Mmax = b.shape[1] - 1, a.shape[1]
    o = opts or make_opts()
    fws, sv, _ = dfilt_workspace_size_ragged(B, total, Nmax, Mmax, o)
    y = torch.empty_like(x) if y is None else y
    if want_saved and sv and saved is None:
        saved = _buf(sv, x.device)
    ws = _buf(fws, x.device) if ws is None else ws
    _check(lib().dfilt_forward_ragged(_ptr(x), _ptr(offsets), _ptr(Ms), _ptr(Ns), _ptr(b),
                                      _ptr(a), _ptr(zi), _ptr(y),
                                      _ptr(saved) if want_saved else None, _ptr(ws), ws.numel(),
                                      B, total, Nmax, Mmax, ctypes.byref(o), _stream(stream)),
           "dfilt_forward_ragged")
    return y, (saved if want_saved and sv else None)


def dfilt_backward_ragged(gy, x, y, offsets, Ms, Ns, b, a, zi=None, saved=None, *,
                          opts: Opts | None = None, needs=(True, True, True, True), ws=None,
                          stream=None):
    gy, x, y = _f32(gy, "gy"), _f32(x, "x"), _f32(y, "y")
    b, a = _f32(b, "b"), _f32(a, "a")
    B = Ms.shape[0]
    total = x.shape[0]
    Nmax, Mmax = b.shape[1] - 1, a.shape[1]
    o = opts or make_opts()
    _, _, bws = dfilt_workspace_size_ragged(B, total, Nmax, Mmax, o)
    gx = torch.empty_like(x) if needs[0] else None
    gb = torch.zeros_like(b) if needs[1] else None
    ga = torch.zeros_like(a) if needs[2] else None
    gzi = torch.zeros((B, Mmax), dtype=torch.float32, device=x.device) if needs[3] else None
    ws = _buf(bws, x.device) if ws is None else ws
    _check(lib().dfilt_backward_ragged(_ptr(gy), _ptr(x), _ptr(y), _ptr(offsets), _ptr(Ms),
                                       _ptr(Ns), _ptr(b), _ptr(a), _ptr(zi), _ptr(saved),
                                       _ptr(gx), _ptr(gb), _ptr(ga), _ptr(gzi), _ptr(ws),
                                       ws.numel(), B, total, Nmax, Mmax, ctypes.byref(o),
                                       _stream(stream)), "dfilt_backward_ragged")
    return gx, gb, ga, gzi


def dfilt_forward_noalloc(x, b, a, zi=None, *, y, opts: Opts | None = None, stream=None):
    """Forward into the caller's `y` with the library's fixed internal scratch: no
    workspace and no device allocation by the library (see include/dfilt.h)."""
    x, b, a, zi = _f32(x, "x"), _f32(b, "b"), _f32(a, "a"), _f32(zi, "zi")
    B, T = x.shape
    o = opts or make_opts()
    _check(lib().dfilt_forward_noalloc(_ptr(x), _ptr(b), _ptr(a), _ptr(zi), _ptr(y), B, T,
                                       b.shape[1] - 1, a.shape[1], ctypes.byref(o),
                                       _stream(stream)), "dfilt_forward_noalloc")
    return y


def dfilt_jvp_workspace_size(B, T, N, M, opts: Opts | None = None) -> int:
    o = opts or make_opts()
    w = ctypes.c_size_t()
    _check(lib().dfilt_jvp_workspace_size(B, T, N, M, ctypes.byref(o), ctypes.byref(w)),
           "dfilt_jvp_workspace_size")
    return w.value


def dfilt_jvp(x, y, b, a, dx=None, db=None, da=None, dzi=None, *, opts: Opts | None = None,
              dy=None, ws=None, stream=None):
    """Forward-mode derivative dy[B,T] of the forward along the tangents (dx, db, da,
    dzi); a tangent left as None is zero.  x, y are the forward's input and output."""
    x, y, b, a = _f32(x, "x"), _f32(y, "y"), _f32(b, "b"), _f32(a, "a")
    dx, db, da, dzi = _f32(dx, "dx"), _f32(db, "db"), _f32(da, "da"), _f32(dzi, "dzi")
    B, T = x.shape
    N, M = b.shape[1] - 1, a.shape[1]
    o = opts or make_opts()
    nws = dfilt_jvp_workspace_size(B, T, N, M, o)
    dy = torch.empty_like(x) if dy is None else dy
    ws = _buf(nws, x.device) if ws is None else ws
    _check(lib().dfilt_jvp(_ptr(x), _ptr(y), _ptr(b), _ptr(a), _ptr(dx), _ptr(db), _ptr(da),
                           _ptr(dzi), _ptr(dy), _ptr(ws), ws.numel(), B, T, N, M,
                           ctypes.byref(o), _stream(stream)), "dfilt_jvp")
    return dy


def dfilt_ss_workspace_size(B, T, M):
    f, w = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().dfilt_ss_workspace_size(B, T, M, ctypes.byref(f), ctypes.byref(w)),
           "dfilt_ss_workspace_size")
    return f.value, w.value


def dfilt_ss_forward(A, v0, z, *, v=None, ws=None, stream=None):
    """v(1..T) [B,T,M] of the recurrence v(n+1) = A v(n) + z(n) (App. B), batched."""
    A, v0, z = _f32(A, "A"), _f32(v0, "v0"), _f32(z, "z")
    B, T, M = z.shape
    fws, _ = dfilt_ss_workspace_size(B, T, M)
    v = torch.empty_like(z) if v is None else v
    ws = _buf(fws, z.device) if ws is None else ws
    _check(lib().dfilt_ss_forward(_ptr(A), _ptr(v0), _ptr(z), _ptr(v), _ptr(ws), ws.numel(),
                                  B, T, M, _stream(stream)), "dfilt_ss_forward")
    return v


def dfilt_ss_backward(A, v0, v, gv, *, needs=(True, True), ws=None, stream=None):
    """(grad_A, grad_v0, grad_z) of the recurrence (App. A); entries of `needs` select
    grad_A and grad_v0."""
    A, v0, v, gv = _f32(A, "A"), _f32(v0, "v0"), _f32(v, "v"), _f32(gv, "gv")
    B, T, M = gv.shape
    _, bws = dfilt_ss_workspace_size(B, T, M)
    gA = torch.empty_like(A) if needs[0] else None
    gv0 = torch.empty((B, M), dtype=torch.float32, device=gv.device) if needs[1] else None
    gz = torch.empty_like(gv)
    ws = _buf(bws, gv.device) if ws is None else ws
    _check(lib().dfilt_ss_backward(_ptr(A), _ptr(v0), _ptr(v), _ptr(gv), _ptr(gA), _ptr(gv0),
                                   _ptr(gz), _ptr(ws), ws.numel(), B, T, M, _stream(stream)),
           "dfilt_ss_backward")
    return gA, gv0, gz


def _c64(t, name):
    """A contiguous complex64 CUDA tensor (complex arrays cross the C ABI as interleaved
    (re, im) float pairs)."""
    if not isinstance(t, torch.Tensor) or t.dtype != torch.complex64 or not t.is_cuda:
        raise TypeError(f"{name}: expected a complex64 CUDA tensor")
    return t.contiguous()


def dfilt_diag_workspace_size(B, T, M):
    f, w = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().dfilt_diag_workspace_size(B, T, M, ctypes.byref(f), ctypes.byref(w)),
           "dfilt_diag_workspace_size")
    return f.value, w.value


def dfilt_diag_forward(lam, V, Vinv, v0, z, *, v=None, ws=None, stream=None):
    """v(1..T) [B,T,M] of v(n+1) = A v(n) + z(n) with A = V diag(lam) V^-1 given by its
    eigendecomposition (lam [B,M], V and Vinv [B,M,M], complex64), run in the eigenbasis."""
    lam, V, Vinv = _c64(lam, "lam"), _c64(V, "V"), _c64(Vinv, "Vinv")
    v0, z = _f32(v0, "v0"), _f32(z, "z")
    B, T, M = z.shape
    fws, _ = dfilt_diag_workspace_size(B, T, M)
    v = torch.empty_like(z) if v is None else v
    ws = _buf(fws, z.device) if ws is None else ws
    _check(lib().dfilt_diag_forward(_ptr(lam), _ptr(V), _ptr(Vinv), _ptr(v0), _ptr(z), _ptr(v),
                                    _ptr(ws), ws.numel(), B, T, M, _stream(stream)),
           "dfilt_diag_forward")
    return v


def dfilt_diag_backward(lam, V, Vinv, v0, v, gv, *, needs=(True, True), ws=None, stream=None):
    """(grad_A, grad_v0, grad_z) of the diagonalised recurrence (the same gradients as the
    dense operator's); entries of `needs` select grad_A and grad_v0."""
    lam, V, Vinv = _c64(lam, "lam"), _c64(V, "V"), _c64(Vinv, "Vinv")
    v0, v, gv = _f32(v0, "v0"), _f32(v, "v"), _f32(gv, "gv")
    B, T, M = gv.shape
    _, bws = dfilt_diag_workspace_size(B, T, M)
    gA = torch.empty((B, M, M), dtype=torch.float32, device=gv.device) if needs[0] else None
    gv0 = torch.empty((B, M), dtype=torch.float32, device=gv.device) if needs[1] else None
    gz = torch.empty_like(gv)
    ws = _buf(bws, gv.device) if ws is None else ws
    _check(lib().dfilt_diag_backward(_ptr(lam), _ptr(V), _ptr(Vinv), _ptr(v0), _ptr(v), _ptr(gv),
                                     _ptr(gA), _ptr(gv0), _ptr(gz), _ptr(ws), ws.numel(), B, T, M,
                                     _stream(stream)), "dfilt_diag_backward")
    return gA, gv0, gz


def dfilt_tv_workspace_size(B, T, N, M):
    w = ctypes.c_size_t()
    _check(lib().dfilt_tv_workspace_size(B, T, N, M, ctypes.byref(w)), "dfilt_tv_workspace_size")
    return w.value


def dfilt_tv_forward(x, b, a, ypast=None, *, y=None, ws=None, stream=None):
    """Parameter-varying direct form: x [B,T], b [B,T,N+1], a [B,T,M] (coefficients of each
    output sample), ypast [B,M] (y[-1], ..., y[-M]) or None -> y [B,T]."""
    x, b, a, ypast = _f32(x, "x"), _f32(b, "b"), _f32(a, "a"), _f32(ypast, "ypast")
    B, T = x.shape
    N, M = b.shape[2] - 1, a.shape[2]
    nws = dfilt_tv_workspace_size(B, T, N, M)
    y = torch.empty_like(x) if y is None else y
    ws = _buf(nws, x.device) if ws is None else ws
    _check(lib().dfilt_tv_forward(_ptr(x), _ptr(b), _ptr(a), _ptr(ypast), _ptr(y), _ptr(ws),
                                  ws.numel(), B, T, N, M, _stream(stream)), "dfilt_tv_forward")
    return y


def dfilt_tv_backward(gy, x, y, b, a, ypast=None, *, needs=(True, True, True, True), ws=None,
                      stream=None):
    """(grad_x, grad_b, grad_a, grad_ypast) of dfilt_tv_forward; `needs` selects them
    (None where not wanted)."""
    gy, x, y = _f32(gy, "gy"), _f32(x, "x"), _f32(y, "y")
    b, a, ypast = _f32(b, "b"), _f32(a, "a"), _f32(ypast, "ypast")
    B, T = gy.shape
    N, M = b.shape[2] - 1, a.shape[2]
    nws = dfilt_tv_workspace_size(B, T, N, M)
    gx = torch.empty_like(gy) if needs[0] else None
    gb = torch.empty_like(b) if needs[1] else None
    ga = torch.empty_like(a) if needs[2] else None
    gyp = torch.empty((B, M), dtype=torch.float32, device=gy.device) if needs[3] else None
    ws = _buf(nws, gy.device) if ws is None else ws
    _check(lib().dfilt_tv_backward(_ptr(gy), _ptr(x), _ptr(y), _ptr(b), _ptr(a), _ptr(ypast),
                                   _ptr(gx), _ptr(gb), _ptr(ga), _ptr(gyp), _ptr(ws), ws.numel(),
                                   B, T, N, M, _stream(stream)), "dfilt_tv_backward")
    return gx, gb, ga, gyp


def dfilt_ic_df1(b, a, xpast, ypast, *, zi=None, stream=None):
    """TDF-II state zi[B,M] equivalent to past inputs xpast[B,N] and outputs ypast[B,M]."""
    b, a, xpast, ypast = _f32(b, "b"), _f32(a, "a"), _f32(xpast, "xpast"), _f32(ypast, "ypast")
    B, M = a.shape
    N = b.shape[1] - 1
    zi = torch.empty((B, M), dtype=torch.float32, device=a.device) if zi is None else zi
    _check(lib().dfilt_ic_df1(_ptr(b), _ptr(a), _ptr(xpast), _ptr(ypast), _ptr(zi), B, N, M,
                              _stream(stream)), "dfilt_ic_df1")
    return zi


def dfilt_ic_df1_backward(b, a, xpast, ypast, gzi, gb=None, ga=None, *,
                          needs=(True, True), stream=None):
    """(grad_xpast, grad_ypast) from grad_zi; adds the past values' terms to gb, ga
    (the filter backward's coefficient gradients) in place when given."""
    b, a, xpast, ypast = _f32(b, "b"), _f32(a, "a"), _f32(xpast, "xpast"), _f32(ypast, "ypast")
    gzi = _f32(gzi, "gzi")
    B, M = a.shape
    N = b.shape[1] - 1
    gxp = torch.empty((B, N), dtype=torch.float32, device=a.device) if needs[0] else None
    gyp = torch.empty((B, M), dtype=torch.float32, device=a.device) if needs[1] else None
    _check(lib().dfilt_ic_df1_backward(_ptr(b), _ptr(a), _ptr(xpast), _ptr(ypast), _ptr(gzi),
                                       _ptr(gxp), _ptr(gyp), _ptr(gb), _ptr(ga), B, N, M,
                                       _stream(stream)), "dfilt_ic_df1_backward")
    return gxp, gyp


def dfilt_sync_status(stream=None) -> int:
    """Synchronise the stream; return (and clear) the device status word."""
    return int(lib().dfilt_sync_status(_stream(stream)))


def dfilt_set_wait_limit(iters: int):
    _check(lib().dfilt_set_wait_limit(int(iters)), "dfilt_set_wait_limit")


def dfilt_debug_build() -> bool:
    """True when the loaded library is the debug build (device-side index checks)."""
    return bool(lib().dfilt_debug_build())


def dfilt_debug_set_limit(samples: int):
    """Debug build only: the index checks treat every signal as at most `samples` long
    (<= 0: no limit); later calls skip the work past it and report DFILT_ERR_BOUNDS."""
    _check(lib().dfilt_debug_set_limit(int(samples)), "dfilt_debug_set_limit")


def dfilt_set_numeric_check(enable: bool):
    """Scan every later call's outputs for non-finite values (DFILT_ERR_NUMERIC)."""
    _check(lib().dfilt_set_numeric_check(1 if enable else 0), "dfilt_set_numeric_check")


def dfilt_kernel_timing(enable: bool):
    """Start (True) or stop (False) event timing of each call's main kernel."""
    _check(lib().dfilt_kernel_timing(1 if enable else 0), "dfilt_kernel_timing")


def dfilt_kernel_timing_read():
    """Wait for the recorded calls; return ((fwd_ms_total, fwd_calls), (bwd_ms_total, bwd_calls))."""
    fm, bm = ctypes.c_double(), ctypes.c_double()
    fn, bn = ctypes.c_int(), ctypes.c_int()
    _check(lib().dfilt_kernel_timing_read(ctypes.byref(fm), ctypes.byref(fn), ctypes.byref(bm),
                                          ctypes.byref(bn)), "dfilt_kernel_timing_read")
    return (fm.value, fn.value), (bm.value, bn.value)


TIMING_CLASSES = ["forward", "backward", "scan", "e_pass", "y_pass", "u_pass", "span_transition",
                  "fused"]


def dfilt_kernel_timing_read_classes():
    """{class: (ms_total, records)} of the recorded event pairs (then discarded)."""
    ms = (ctypes.c_double * 8)()
    n = (ctypes.c_int * 8)()
    _check(lib().dfilt_kernel_timing_read_classes(ms, n), "dfilt_kernel_timing_read_classes")
    return {k: (ms[i], n[i]) for i, k in enumerate(TIMING_CLASSES)}


def dfilt_tuning_set(state_bucket: int, span_tiles: int = 0, chains_per_sm: int = 0):
    """Install a decoupled-path launch shape for a state bucket (0 = automatic)."""
    _check(lib().dfilt_tuning_set(int(state_bucket), int(span_tiles), int(chains_per_sm)),
           "dfilt_tuning_set")


def dfilt_tuning_get(state_bucket: int):
    """(span_tiles, chains_per_sm) installed for a state bucket (0 = automatic)."""
    s, c = ctypes.c_int(), ctypes.c_int()
    _check(lib().dfilt_tuning_get(int(state_bucket), ctypes.byref(s), ctypes.byref(c)),
           "dfilt_tuning_get")
    return s.value, c.value


def dfilt_launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    v = ctypes.c_int64()
    _check(lib().dfilt_launch_count(ctypes.byref(v)), "dfilt_launch_count")
    return v.value


# ---------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------

class DFilt(torch.autograd.Function):
    """y = DFilt.apply(x, b, a, zi, opts): batched direct-form filter whose backward
    is the library's closed-form adjoint (Sec. 3.1).  zi may be None."""

    @staticmethod
    def forward(ctx, x, b, a, zi=None, opts: Opts | None = None):
        opts = opts or make_opts()
        y, saved = dfilt_forward(x, b, a, zi, opts=opts)
        # y is kept for the backward (it is the output, so this costs no memory): the
        # decoupled high-order path reads it instead of recomputing it from the chunk
        # states, and the single-kernel path re-reads it when there are no chunk states
        ctx.opts = opts
        ctx.has_zi = zi is not None
        ctx.save_for_backward(x, b, a, zi if zi is not None else x.new_empty(0),
                              saved if saved is not None else x.new_empty(0), y)
        return y

    @staticmethod
    def backward(ctx, gy):
        x, b, a, zi, saved, y = ctx.saved_tensors
        needs = tuple(bool(v) for v in ctx.needs_input_grad[:4])
        gx, gb, ga, gzi = dfilt_backward(gy.contiguous(), x, y if y.numel() else None, b, a,
                                         zi if ctx.has_zi else None,
                                         saved if saved.numel() else None, opts=ctx.opts,
                                         needs=needs)
        return gx, gb, ga, (gzi if ctx.has_zi else None), None


def filt(x, b, a, zi=None, **opt_kwargs):
    """Differentiable batched direct-form filter (see DFilt)."""
    return DFilt.apply(x, b, a, zi, make_opts(**opt_kwargs) if opt_kwargs else None)


class DFiltDF1(torch.autograd.Function):
    """y = DFiltDF1.apply(x, b, a, xpast, ypast, opts): the filter started from
    direct-form initial conditions (past inputs xpast[B,N], past outputs ypast[B,M]),
    through the library's map to the TDF-II state and its adjoint."""

    @staticmethod
    def forward(ctx, x, b, a, xpast, ypast, opts: Opts | None = None):
        opts = opts or make_opts()
        zi = dfilt_ic_df1(b, a, xpast, ypast)
        y, saved = dfilt_forward(x, b, a, zi, opts=opts)
        ctx.opts = opts
        empty = x.new_empty(0)
        ctx.save_for_backward(x, b, a, xpast, ypast, zi, saved if saved is not None else empty,
                              y if saved is None else empty)
        return y

    @staticmethod
    def backward(ctx, gy):
        x, b, a, xpast, ypast, zi, saved, y = ctx.saved_tensors
        ng = ctx.needs_input_grad
        needs = (bool(ng[0]), bool(ng[1]), bool(ng[2]), True)
        gx, gb, ga, gzi = dfilt_backward(gy.contiguous(), x, y if y.numel() else None, b, a, zi,
                                         saved if saved.numel() else None, opts=ctx.opts,
                                         needs=needs)
        gxp, gyp = dfilt_ic_df1_backward(b, a, xpast, ypast, gzi, gb, ga,
                                         needs=(bool(ng[3]), bool(ng[4])))
        return gx, gb, ga, gxp, gyp, None


def filt_df1(x, b, a, xpast, ypast, **opt_kwargs):
    """Differentiable filter with direct-form initial conditions (see DFiltDF1)."""
    return DFiltDF1.apply(x, b, a, xpast, ypast, make_opts(**opt_kwargs) if opt_kwargs else None)


class DFiltRagged(torch.autograd.Function):
    """y = DFiltRagged.apply(x, offsets, Ms, Ns, b, a, zi, opts): a ragged batch packed
    into one signal (channel i is x[offsets[i]:offsets[i+1]] with orders Ms[i], Ns[i];
    b [B, Nmax+1], a [B, Mmax], zi [B, Mmax] zero-padded rows; zi may be None); the
    backward is the library's closed-form adjoint.  offsets, Ms and Ns get no gradient.
    The calls allocate through torch only, so a whole training step around it can be
    captured in a CUDA graph."""

    @staticmethod
    def forward(ctx, x, offsets, Ms, Ns, b, a, zi=None, opts: Opts | None = None):
        opts = opts or make_opts()
        y, saved = dfilt_forward_ragged(x, offsets, Ms, Ns, b, a, zi, opts=opts)
        ctx.opts = opts   # y is kept for the backward, as in DFilt
        ctx.has_zi = zi is not None
        empty = x.new_empty(0)
        ctx.save_for_backward(x, offsets, Ms, Ns, b, a, zi if zi is not None else empty,
                              saved if saved is not None else empty, y)
        return y

    @staticmethod
    def backward(ctx, gy):
        x, offsets, Ms, Ns, b, a, zi, saved, y = ctx.saved_tensors
        ng = ctx.needs_input_grad
        needs = (bool(ng[0]), bool(ng[4]), bool(ng[5]), bool(ng[6]) and ctx.has_zi)
        gx, gb, ga, gzi = dfilt_backward_ragged(gy.contiguous(), x, y if y.numel() else None,
                                                offsets, Ms, Ns, b, a,
                                                zi if ctx.has_zi else None,
                                                saved if saved.numel() else None,
                                                opts=ctx.opts, needs=needs)
        return gx, None, None, None, gb, ga, (gzi if ctx.has_zi else None), None


def filt_ragged(x, offsets, Ms, Ns, b, a, zi=None, **opt_kwargs):
    """Differentiable ragged batch of direct-form filters (see DFiltRagged)."""
    return DFiltRagged.apply(x, offsets, Ms, Ns, b, a, zi,
                             make_opts(**opt_kwargs) if opt_kwargs else None)
