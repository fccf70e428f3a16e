"""The parameter-varying direct form (dfilt_tv_forward / dfilt_tv_backward: coefficients
per output sample) through the C ABI against the FP64 oracle (oracle.forward_tv /
backward_tv), element by element: every supported M with numerators 0..M, lengths around
the 32-step chunks and 1024-step segments, more than 32 segments, with and without past
outputs, and against the fixed-coefficient chunked path when the coefficients are
constant.

Coefficients: each channel's poles (conjugate pairs, radius 0.5-0.95, one real pole for
odd orders) move smoothly over time (radius and angle modulated by slow sinusoids), the
numerator likewise; the filter stays stable at every sample.  Tolerance per channel
max(1e-5, 32 u32 kappa), kappa = sum_n |h[n]| (1 + max_n sum_k |a[n][k]|) with h the
impulse response of the time-varying all-pole part from time 0 (oracle), the first-order
bound of a rounded linear recursion as for the fixed-coefficient filter."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_14390_gb300 import dfilt

from tol import U32, log_errors, rel_rows

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


def varying_coefficients(rng, B, T, N, M, rlo=0.5, rhi=0.95):
    """a [B,T,M], b [B,T,N+1] from poles / zeros modulated slowly over time (FP64)."""
    n = np.arange(T)[:, None]
    a = np.zeros((B, T, M)); b = np.zeros((B, T, N + 1))
    for i in range(B):
        npair = M // 2
        r0 = rng.uniform(rlo, rhi, npair); th0 = rng.uniform(0.1, 3.0, npair)
        wr, wt = rng.uniform(1e-3, 2e-2, npair), rng.uniform(1e-3, 2e-2, npair)
        r = r0 * (1 - 0.04 * (1 + np.sin(wr * n)))            # stays below r0
        th = th0 + 0.2 * np.sin(wt * n)
        poles = np.concatenate([r * np.exp(1j * th), r * np.exp(-1j * th)], axis=1)
        if M % 2:
            pr = rng.uniform(rlo, rhi) * rng.choice([-1, 1]) * (1 - 0.04 * (1 + np.sin(0.005 * n)))
            poles = np.concatenate([poles, pr], axis=1)
        for t in range(T):
            a[i, t] = np.real(np.poly(poles[t]))[1:]
        zb = rng.standard_normal(N + 1)
        b[i] = zb[None, :] * (1 + 0.1 * np.sin(0.003 * n))
    return a.astype(np.float32), b.astype(np.float32)


def kappa(a):
    B, T, M = a.shape
    imp = np.zeros((B, T)); imp[:, 0] = 1.0
    h = oracle.forward_tv(imp, np.ones((B, T, 1)), a)
    return np.abs(h).sum(1) * (1 + np.abs(a).sum(2).max(1))


def run_and_check(name, x, b, a, yp, gy):
    B, T = x.shape
    xd, bd, ad, ypd, gyd = dev(x), dev(b), dev(a), dev(yp), dev(gy)
    y = dfilt.dfilt_tv_forward(xd, bd, ad, ypd)
    gx, gb, ga, gyp = dfilt.dfilt_tv_backward(gyd, xd, y, bd, ad, ypd)
    st = dfilt.dfilt_sync_status()
    assert st == 0, dfilt.STATUS[st]
    y, gx, gb, ga, gyp = (t.cpu().numpy().astype(np.float64) for t in (y, gx, gb, ga, gyp))
    yr = oracle.forward_tv(x, b, a, yp)
    rx, rb, ra, ryp = oracle.backward_tv(gy, x, yr, b, a, yp)
    u = oracle.backward_tv(gy, x, yr, np.ones((B, T, 1)), a, yp)[0]   # the adjoint itself
    errs = {"y": rel_rows(y, yr), "gx": rel_rows(gx, rx),
            "gb": rel_rows(gb.reshape(B, -1), rb.reshape(B, -1)),
            "ga": rel_rows(ga.reshape(B, -1), ra.reshape(B, -1)),
            "gyp": np.abs(gyp - ryp).max(1) / np.maximum(np.abs(u).max(1) * np.abs(a).sum(2).max(1), 1e-30)}
    tol = np.maximum(1e-5, 32 * U32 * kappa(a))
    log_errors(f"tv_{name}", **errs)
    for k, e in errs.items():
        assert (e < tol).all(), (name, k, e, tol)


@pytest.mark.parametrize("M,N", [(1, 0), (1, 1), (2, 0), (2, 2), (3, 1), (3, 3), (4, 2), (4, 4)])
@pytest.mark.parametrize("T", [1, 31, 33, 1024, 1025, 5000])
def test_tv_shapes(M, N, T):
    rng = np.random.default_rng(100 * M + 10 * N + T)
    B = 3
    a, b = varying_coefficients(rng, B, T, N, M)
    x = rng.standard_normal((B, T)).astype(np.float32)
    yp = (0.1 * rng.standard_normal((B, M))).astype(np.float32)
    gy = rng.standard_normal((B, T)).astype(np.float32)
    run_and_check(f"M{M}N{N}_T{T}", x, b, a, yp, gy)


def test_tv_many_segments_no_past():
    """40000 steps = 40 segments; no past outputs; poles up to radius 0.99."""
    rng = np.random.default_rng(5)
    B, T, N, M = 2, 40000, 2, 2
    a, b = varying_coefficients(rng, B, T, N, M, 0.9, 0.99)
    x = rng.standard_normal((B, T)).astype(np.float32)
    gy = rng.standard_normal((B, T)).astype(np.float32)
    run_and_check("many_segments", x, b, a, None, gy)


def test_tv_constant_coefficients_match_fixed_filter():
    """Constant per-sample coefficients and no past: the same filter as the
    fixed-coefficient chunked path with a zero initial state (y, grad_x; the per-sample
    coefficient gradients summed over time give its grad_b, grad_a)."""
    rng = np.random.default_rng(6)
    B, T, N, M = 4, 3 * 8192 + 99, 2, 2
    a0, b0 = varying_coefficients(rng, B, 1, N, M)
    a = np.repeat(a0, T, axis=1); b = np.repeat(b0, T, axis=1)
    x = rng.standard_normal((B, T)).astype(np.float32)
    gy = rng.standard_normal((B, T)).astype(np.float32)
    xd, gyd = dev(x), dev(gy)
    y = dfilt.dfilt_tv_forward(xd, dev(b), dev(a))
    gx, gb, ga, _ = dfilt.dfilt_tv_backward(gyd, xd, y, dev(b), dev(a), needs=(True, True, True, False))
    zi = torch.zeros((B, M), device=DEV)
    yf, saved = dfilt.dfilt_forward(xd, dev(b0[:, 0]), dev(a0[:, 0]), zi, opts=dfilt.make_opts(algo="chunked"))
    gf = dfilt.dfilt_backward(gyd, xd, None, dev(b0[:, 0]), dev(a0[:, 0]), zi, saved,
                              opts=dfilt.make_opts(algo="chunked"))
    assert dfilt.dfilt_sync_status() == 0
    assert (rel_rows(y.cpu().numpy(), yf.cpu().numpy()) < 1e-5).all()
    assert (rel_rows(gx.cpu().numpy(), gf[0].cpu().numpy()) < 1e-5).all()
    assert (rel_rows(gb.sum(1).cpu().numpy(), gf[1].cpu().numpy()) < 1e-4).all()
    assert (rel_rows(ga.sum(1).cpu().numpy(), gf[2].cpu().numpy()) < 1e-4).all()


def test_tv_empty_and_selected_gradients():
    e = torch.empty(0, 7, device=DEV)
    assert dfilt.dfilt_tv_forward(e, torch.empty(0, 7, 3, device=DEV), torch.empty(0, 7, 2, device=DEV)).shape == (0, 7)
    rng = np.random.default_rng(7)
    B, T, N, M = 2, 3000, 1, 3
    a, b = varying_coefficients(rng, B, T, N, M)
    x = dev(rng.standard_normal((B, T))); gy = dev(rng.standard_normal((B, T)))
    yp = dev(0.1 * rng.standard_normal((B, M)))
    y = dfilt.dfilt_tv_forward(x, dev(b), dev(a), yp)
    full = dfilt.dfilt_tv_backward(gy, x, y, dev(b), dev(a), yp)
    part = dfilt.dfilt_tv_backward(gy, x, y, dev(b), dev(a), yp, needs=(False, True, False, True))
    assert part[0] is None and part[2] is None
    assert torch.equal(part[1], full[1]) and torch.equal(part[3], full[3])
    assert dfilt.dfilt_sync_status() == 0
