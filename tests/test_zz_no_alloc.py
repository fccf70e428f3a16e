"""dfilt_forward_noalloc: the forward for callers that cannot allocate device memory
while they run (for example a real-time audio callback, where cudaMalloc can stall on
device synchronisation, or a host without a device allocator).  It keeps its scratch
in a fixed array inside the library, so it must give the same y as dfilt_forward with
a caller workspace -- also on a second call, when the array still holds the previous
call's tables.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2511_14390_gb300 import dfilt, inputs

pytestmark = pytest.mark.gpu


def _rel(got, ref):
    got = got.double().cpu().numpy()
    ref = ref.double().cpu().numpy()
    return float((np.abs(got - ref).max(1) / np.abs(ref).max(1)).max())


def test_noalloc_forward_matches_workspace_forward_on_consecutive_calls():
    L = dfilt.lib()
    o = dfilt.make_opts(algo="chunked", precision="tf32x3")
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [inputs.make("biquad_1024x48000", B=96, T=3 * 8192 + 101, seed=41),
             inputs.make("biquad_1024x48000", B=40, T=20000, M=6, N=3, seed=42)]
    for w in cases:   # two calls in a row through the C ABI
        x, b, a, zi = dev(w.x), dev(w.b), dev(w.a), dev(w.zi)
        B, T = w.x.shape
        y_ref, _ = dfilt.dfilt_forward(x, b, a, zi, opts=o, want_saved=False)
        y = torch.full_like(x, float("nan"))
        rc = L.dfilt_forward_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                     ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(zi.data_ptr()),
                                     ctypes.c_void_p(y.data_ptr()), B, T, w.N, w.M,
                                     ctypes.byref(o), stream)
        assert rc == 0, dfilt.STATUS.get(rc, rc)
        assert dfilt.dfilt_sync_status() == 0
        assert torch.isfinite(y).all()
        assert _rel(y, y_ref) < 1e-5


def test_noalloc_rejects_batches_beyond_its_scratch():
    L = dfilt.lib()
    o = dfilt.make_opts(algo="chunked")
    # 64th-order tables for 4096 channels need far more than the fixed scratch
    B, T, M = 4096, 100, 64
    x = torch.zeros(B, T, device="cuda:0")
    b = torch.zeros(B, M + 1, device="cuda:0")
    a = torch.zeros(B, M, device="cuda:0")
    y = torch.zeros(B, T, device="cuda:0")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = L.dfilt_forward_noalloc(p(x), p(b), p(a), None, p(y), B, T, M, M, ctypes.byref(o), None)
    assert rc == 6   # DFILT_ERR_WORKSPACE, returned before any launch
    assert not y.any()
