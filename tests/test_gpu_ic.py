"""Direct-form initial conditions (past inputs and outputs) through the C ABI
(dfilt_ic_df1 + the filter + dfilt_ic_df1_backward, composed by DFiltDF1) against the
FP64 oracle's difference equation extended into negative time, element by element:
the output and the gradients of x, b, a and both past-value arrays, on the chunked
and sequential paths, for several orders including N = 0."""
import numpy as np
import pytest
import scipy.signal as ss
import torch

import oracle
from paper_2511_14390_gb300 import dfilt, inputs

from tol import U32, coef_err, kappa, log_errors, rel_rows

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def dev(a, grad=False):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)
    return t.requires_grad_() if grad else t


def case(M, N, B, T, seed):
    w = inputs.make("biquad_1024x48000", B=B, T=T, M=M, N=N, seed=seed)
    rng = np.random.default_rng(seed + 1)
    if M > 2:
        for i in range(B):
            w.a[i], _, _ = inputs.draw_denominator(rng, M, 0.3, 0.8)
    xp = rng.standard_normal((B, N)).astype(np.float32)
    yp = rng.standard_normal((B, M)).astype(np.float32)
    return w, xp, yp


@pytest.mark.parametrize("algo", ["chunked", "sequential"])
@pytest.mark.parametrize("M,N", [(2, 2), (5, 3), (3, 0), (16, 16)])
def test_df1_forward_and_gradients(algo, M, N):
    B, T = 4, 2 * 8192 + 123
    w, xp, yp = case(M, N, B, T, 90 + 7 * M + N)
    x, b, a = dev(w.x, True), dev(w.b, True), dev(w.a, True)
    xpd, ypd = dev(xp, True), dev(yp, True)
    y = dfilt.filt_df1(x, b, a, xpd, ypd, algo=algo)
    (y * dev(w.gy)).sum().backward()
    torch.cuda.synchronize()
    assert dfilt.dfilt_sync_status() == 0
    yr = oracle.forward_df1(w.x, w.b, w.a, xp, yp)
    gx, gb, ga, gxp, gyp = oracle.backward_df1(w.gy, w.x, yr, w.b, w.a, xp, yp)
    h = lambda t: t.detach().cpu().numpy().astype(np.float64)
    tol = np.maximum(1e-5, 16 * U32 * kappa(w.a, T))
    # each coefficient / past-value gradient against the sum of its terms' magnitudes
    u = np.abs(oracle.backward(w.gy, w.x, yr, np.ones((B, 1)), w.a)[0])
    xe = np.abs(np.concatenate([xp[:, ::-1], w.x], 1))     # xe[:, N + i] = |x[i]|, i >= -N
    ye = np.abs(np.concatenate([yp[:, ::-1], yr], 1))      # ye[:, M + i] = |y[i]|, i >= -M
    Sb = np.stack([(u * xe[:, N - k: N - k + T]).sum(1) for k in range(N + 1)], 1)
    Sa = np.stack([(u * ye[:, M - k: M - k + T]).sum(1) for k in range(1, M + 1)], 1)
    ab, aa = np.abs(w.b).astype(np.float64), np.abs(w.a).astype(np.float64)
    Syp = np.stack([sum(aa[:, k - 1] * u[:, k - j] for k in range(j, M + 1))
                    for j in range(1, M + 1)], 1)
    errs = {"y": rel_rows(h(y), yr), "gx": rel_rows(h(x.grad), gx),
            "gb": coef_err(h(b.grad), gb, Sb), "ga": coef_err(h(a.grad), ga, Sa),
            "gypast": coef_err(h(ypd.grad), gyp, Syp)}
    if N:
        Sxp = np.stack([sum(ab[:, k] * u[:, k - j] for k in range(j, N + 1))
                        for j in range(1, N + 1)], 1)
        errs["gxpast"] = coef_err(h(xpd.grad), gxp, Sxp)
    log_errors(f"df1_{algo}_M{M}_N{N}", **errs)
    for k, e in errs.items():
        assert (e < tol).all(), (k, e, tol)


def test_df1_state_matches_lfiltic():
    """The library's map to the TDF-II state equals SciPy's lfiltic (library routine)."""
    w, xp, yp = case(6, 4, 5, 100, 123)
    zi = dfilt.dfilt_ic_df1(dev(w.b), dev(w.a), dev(xp), dev(yp)).cpu().numpy()
    for i in range(5):
        ref = ss.lfiltic(w.b[i].astype(np.float64), np.concatenate([[1.0], w.a[i]]),
                         yp[i].astype(np.float64), xp[i].astype(np.float64))
        assert np.abs(zi[i] - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max()), (zi[i], ref)
