"""The C-ABI library: builds for sm_103a, loads, exports every symbol include/dfilt.h
declares, and validates arguments on the host (no compute call without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2511_14390_gb300 import build as pkg_build
from paper_2511_14390_gb300 import dfilt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    pkg_build.build()
    return dfilt.lib()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "dfilt.h")).read()
    return sorted(set(re.findall(r"\b(dfilt_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    syms = declared_symbols()
    assert len(syms) >= 11
    for s in syms:
        assert hasattr(L, s), s
    assert set(syms) == set(dfilt.EXPORTS)


def test_host_only_calls(L):
    assert L.dfilt_version() == 100
    assert L.dfilt_status_string(4) == b"DFILT_ERR_TIMEOUT"
    o = dfilt.Opts()
    assert L.dfilt_default_opts(ctypes.byref(o)) == 0
    assert (o.algo, o.precision, o.chunk_len, o.fp64_scan) == (0, 3, 0, -1)


def test_kernel_timing_without_calls(L):
    """Timing switch and read are host-side; with no recorded call the sums are zero."""
    dfilt.dfilt_kernel_timing(True)
    assert dfilt.dfilt_kernel_timing_read() == ((0.0, 0), (0.0, 0))
    dfilt.dfilt_kernel_timing(False)
    assert dfilt.dfilt_kernel_timing_read() == ((0.0, 0), (0.0, 0))


def test_workspace_sizes(L):
    f, s, w = dfilt.dfilt_workspace_size(1024, 48000, 2, 2)
    assert f > 0 and w > 0 and s >= 1024 * 48000 // 64 * 2 * 4
    f, s, w = dfilt.dfilt_workspace_size(1024, 48000, 2, 2, dfilt.make_opts("sequential"))
    assert (f, s, w) == (0, 0, 0)
    f, s, w = dfilt.dfilt_workspace_size_ragged(4096, 10 ** 6, 32, 32)
    assert f > 0 and s > 0 and w > 0


@pytest.mark.parametrize("B,T,N,M,code", [(4, 10, 0, 65, 2), (4, 10, 3, 2, 1), (4, 10, 0, 0, 1),
                                          (-1, 10, 0, 2, 1), (4, -5, 0, 2, 1)])
def test_argument_errors(L, B, T, N, M, code):
    o = dfilt.make_opts()
    sz = ctypes.c_size_t()
    assert L.dfilt_workspace_size(B, T, N, M, ctypes.byref(o), ctypes.byref(sz), None, None) == code
    assert L.dfilt_forward(None, None, None, None, None, None, None, 0, B, T, N, M,
                           ctypes.byref(o), None) == code


def test_bad_options(L):
    o = dfilt.make_opts(chunk_len=32)
    sz = ctypes.c_size_t()
    assert L.dfilt_workspace_size(4, 10, 0, 2, ctypes.byref(o), ctypes.byref(sz), None, None) == 2
    o = dfilt.Opts(7, 3, 0, -1)
    assert L.dfilt_workspace_size(4, 10, 0, 2, ctypes.byref(o), ctypes.byref(sz), None, None) == 1


def test_missing_pointers_rejected(L):
    o = dfilt.make_opts()
    assert L.dfilt_forward(None, None, None, None, None, None, None, 0, 4, 10, 0, 2,
                           ctypes.byref(o), None) == 1


def test_jvp_host_checks(L):
    """Forward-mode entry point: workspace size (holds v, B*T floats, plus the forward's
    workspace), argument errors and the empty batch, all decided on the host."""
    o = dfilt.make_opts()
    nws = dfilt.dfilt_jvp_workspace_size(1024, 48000, 2, 2, o)
    f, _, _ = dfilt.dfilt_workspace_size(1024, 48000, 0, 2, o)
    assert nws >= 1024 * 48000 * 4 + 1024 * 4 + f
    sz = ctypes.c_size_t()
    for B, T, N, M, code in [(4, 10, 0, 65, 2), (4, 10, 3, 2, 1), (4, 10, 0, 0, 1),
                             (-1, 10, 0, 2, 1), (4, -5, 0, 2, 1)]:
        assert L.dfilt_jvp_workspace_size(B, T, N, M, ctypes.byref(o), ctypes.byref(sz)) == code
        assert L.dfilt_jvp(None, None, None, None, None, None, None, None, None, None, 0, B, T,
                           N, M, ctypes.byref(o), None) == code
    # missing a / dy, a tangent without the input it multiplies, too small a workspace
    assert L.dfilt_jvp(None, None, None, None, None, None, None, None, None, None, 0, 4, 10, 2,
                       2, ctypes.byref(o), None) == 1
    fake = ctypes.c_void_p(4096)    # never dereferenced: the call fails before any launch
    assert L.dfilt_jvp(None, None, None, fake, fake, None, None, None, fake, fake, 1 << 30, 4,
                       10, 2, 2, ctypes.byref(o), None) == 1          # dx without b
    assert L.dfilt_jvp(None, None, fake, fake, None, None, fake, None, fake, fake, 1 << 30, 4,
                       10, 2, 2, ctypes.byref(o), None) == 1          # da without y
    assert L.dfilt_jvp(None, None, fake, fake, None, None, None, None, fake, fake, 16, 4, 10, 2,
                       2, ctypes.byref(o), None) == 6                 # workspace too small
    assert L.dfilt_jvp(None, None, None, None, None, None, None, None, None, None, 0, 0, 10, 2,
                       2, ctypes.byref(o), None) == 0                 # empty batch


def test_ss_host_checks(L):
    """State-space operator: workspace sizes and argument errors decided on the host."""
    f, w = dfilt.dfilt_ss_workspace_size(64, 1 << 20, 2)
    assert f > 0 and w > f
    sz = ctypes.c_size_t()
    assert L.dfilt_ss_workspace_size(4, 10, 5, ctypes.byref(sz), None) == 2    # M > 4
    assert L.dfilt_ss_workspace_size(4, 10, 0, ctypes.byref(sz), None) == 1
    assert L.dfilt_ss_workspace_size(-1, 10, 2, ctypes.byref(sz), None) == 1
    assert L.dfilt_ss_forward(None, None, None, None, None, 0, 4, 10, 2, None) == 1
    assert L.dfilt_ss_forward(None, None, None, None, None, 0, 0, 10, 2, None) == 0
    assert L.dfilt_ss_backward(None, None, None, None, None, None, None, None, 0, 4, 10, 2,
                               None) == 1
    fake = ctypes.c_void_p(4096)    # never dereferenced: the call fails before any launch
    assert L.dfilt_ss_forward(fake, None, fake, fake, fake, 16, 4, 10, 2, None) == 6


def test_diag_host_checks(L):
    """Diagonalised state-space operator: workspace sizes and argument errors decided on
    the host (no launch)."""
    f, w = dfilt.dfilt_diag_workspace_size(64, 1 << 20, 2)
    assert f > 0 and w > f
    sz = ctypes.c_size_t()
    assert L.dfilt_diag_workspace_size(4, 10, 5, ctypes.byref(sz), None) == 2    # M > 4
    assert L.dfilt_diag_workspace_size(4, 10, 0, ctypes.byref(sz), None) == 1
    assert L.dfilt_diag_forward(None, None, None, None, None, None, None, 0, 4, 10, 2, None) == 1
    assert L.dfilt_diag_forward(None, None, None, None, None, None, None, 0, 0, 10, 2, None) == 0
    assert L.dfilt_diag_backward(None, None, None, None, None, None, None, None, None, None, 0,
                                 4, 10, 2, None) == 1
    fake, odd = ctypes.c_void_p(4096), ctypes.c_void_p(4100)
    assert L.dfilt_diag_forward(fake, fake, fake, None, fake, fake, fake, 16, 4, 10, 2, None) == 6
    assert L.dfilt_diag_forward(odd, fake, fake, None, fake, fake, fake, 1 << 20, 4, 10, 2,
                                None) == 1    # complex arrays must be 8-byte aligned


def test_tv_host_checks(L):
    """Parameter-varying filter: workspace sizes and argument errors decided on the host."""
    assert dfilt.dfilt_tv_workspace_size(8, 4096, 2, 2) > 0
    sz = ctypes.c_size_t()
    assert L.dfilt_tv_workspace_size(4, 10, 2, 5, ctypes.byref(sz)) == 2     # M > 4
    assert L.dfilt_tv_workspace_size(4, 10, 3, 2, ctypes.byref(sz)) == 1     # N > M
    assert L.dfilt_tv_workspace_size(4, 10, 0, 0, ctypes.byref(sz)) == 1
    assert L.dfilt_tv_forward(None, None, None, None, None, None, 0, 4, 10, 2, 2, None) == 1
    assert L.dfilt_tv_forward(None, None, None, None, None, None, 0, 0, 10, 2, 2, None) == 0
    fake = ctypes.c_void_p(4096)
    assert L.dfilt_tv_forward(fake, fake, fake, None, fake, fake, 16, 4, 10, 2, 2, None) == 6
    assert L.dfilt_tv_backward(None, None, None, None, None, None, None, None, None, None, None,
                               0, 4, 10, 2, 2, None) == 1


def test_ic_df1_host_checks(L):
    """Direct-form initial conditions: argument errors and the empty batch on the host."""
    assert L.dfilt_ic_df1(None, None, None, None, None, 4, 2, 65, None) == 2
    assert L.dfilt_ic_df1(None, None, None, None, None, 4, 3, 2, None) == 1
    assert L.dfilt_ic_df1(None, None, None, None, None, 4, 2, 2, None) == 1     # zi missing
    assert L.dfilt_ic_df1(None, None, None, None, None, 0, 2, 2, None) == 0
    assert L.dfilt_ic_df1_backward(None, None, None, None, None, None, None, None, None, 4, 2,
                                   2, None) == 1                                  # gzi missing
    assert L.dfilt_ic_df1_backward(None, None, None, None, None, None, None, None, None, 0, 2,
                                   2, None) == 0


@pytest.mark.parametrize("precision", [2, 4])
def test_bf16_precisions_unsupported(L, precision):
    """BF16 and split-BF16 operands are not built: the chunked path reports
    DFILT_ERR_UNSUPPORTED for them, decided on the host."""
    o = dfilt.Opts(2, precision, 0, -1)
    sz = ctypes.c_size_t()
    assert L.dfilt_workspace_size(4, 100, 2, 2, ctypes.byref(o), ctypes.byref(sz), None,
                                  None) == 2


def test_binding_fails_loudly_without_the_library(tmp_path, monkeypatch):
    """No fallback: with libdfilt.so absent the binding raises instead of computing
    anything another way."""
    monkeypatch.setattr(dfilt, "LIB_PATH", str(tmp_path / "libdfilt.so"))
    monkeypatch.setattr(dfilt, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        dfilt.lib()


def test_debug_entry_points_in_release(L):
    """The release library compiles the device-side index checks out: it says so, and
    refuses the debug limit."""
    assert L.dfilt_debug_build() == 0
    assert L.dfilt_debug_set_limit(ctypes.c_int64(1000)) == 2   # DFILT_ERR_UNSUPPORTED
    assert L.dfilt_status_string(7) == b"DFILT_ERR_BOUNDS"


def test_debug_library_builds_and_exports():
    """build.py --debug links libdfilt_debug.so (the checked units recompiled with
    -DDFILT_DEBUG); it loads without a GPU, exports every declared symbol, reports
    itself as the debug build and accepts the limit."""
    path = pkg_build.build_debug()
    D = ctypes.CDLL(path)
    for s in declared_symbols():
        assert hasattr(D, s), s
    D.dfilt_debug_set_limit.argtypes = [ctypes.c_int64]
    assert D.dfilt_debug_build() == 1
    assert D.dfilt_debug_set_limit(1000) == 0
    assert D.dfilt_debug_set_limit(0) == 0
