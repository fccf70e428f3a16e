"""Forward mode (dfilt_jvp) through the C ABI against the FP64 oracle's JVP, element by
element: every tangent alone and all together, the sequential and chunked recursions,
segment and tile boundaries with ragged tails, orders up to 16, short signals, and the
benchmark's full-size workload on sampled channels."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_14390_gb300 import dfilt, inputs

from tol import U32, kappa, log_errors, rel_rows

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
OPTS = {"seq": dict(algo="sequential"), "chunk3": dict(algo="chunked", precision="tf32x3")}
ALL = ("dx", "db", "da", "dzi")


def dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def tangents(w, seed, which=ALL):
    """Seeded tangent directions (float32): signals ~ N(0, 1), coefficients ~ N(0, 0.1^2)."""
    rng = np.random.default_rng(seed)
    t = {"dx": rng.standard_normal(w.x.shape),
         "db": 0.1 * rng.standard_normal(w.b.shape),
         "da": 0.1 * rng.standard_normal(w.a.shape),
         "dzi": rng.standard_normal(w.a.shape)}
    return {k: (v.astype(np.float32) if k in which else None) for k, v in t.items()}


def run(w, t, mode):
    o = dfilt.make_opts(**OPTS[mode])
    x, b, a, zi = dev(w.x), dev(w.b), dev(w.a), dev(w.zi)
    y, _ = dfilt.dfilt_forward(x, b, a, zi, opts=o, want_saved=False)
    dy = dfilt.dfilt_jvp(x, y, b, a, dev(t["dx"]), dev(t["db"]), dev(t["da"]), dev(t["dzi"]),
                         opts=o)
    st = dfilt.dfilt_sync_status()
    assert st == 0, dfilt.STATUS[st]
    return dy.cpu().numpy()


def reference(w, t):
    return oracle.jvp(w.x, w.b, w.a, w.zi, t["dx"], t["db"], t["da"], t["dzi"])[1]


def check(name, w, t, mode, tol):
    got = run(w, t, mode)
    err = rel_rows(got, reference(w, t))
    log_errors(f"jvp_{name}/{mode}", dy=err)
    tol = np.broadcast_to(tol, err.shape)
    assert (err < tol).all(), (name, mode, err, tol)


@pytest.mark.parametrize("mode", ["seq", "chunk3"])
def test_jvp_biquad_all_tangents(mode):
    w = inputs.make("biquad_1024x48000", B=40, T=2 * 8192 + 4321)
    check("biquad", w, tangents(w, 1), mode, 1e-5)


@pytest.mark.parametrize("which", ALL)
def test_jvp_single_tangent(which):
    """Each tangent alone (the others passed as NULL), on segment and tile tails."""
    w = inputs.make("biquad_1024x48000", B=6, T=3 * 2048 + 8192 + 17)
    check(f"only_{which}", w, tangents(w, 2, (which,)), "chunk3", 1e-5)


@pytest.mark.parametrize("M", [1, 3, 8, 16])
def test_jvp_orders(M):
    """Several state buckets (N = M, halo of the input step up to 16), poles r <= 0.7."""
    w = inputs.make("biquad_1024x48000", B=3, T=8192 + 2048 + 333, M=M, N=M, seed=40 + M)
    rng = np.random.default_rng(500 + M)
    for i in range(w.B):
        a, _, _ = inputs.draw_denominator(rng, M, 0.3, 0.7)
        w.a[i] = a
        w.b[i] = inputs.draw_numerator(rng, M, True)
    tol = np.maximum(1e-5, 16 * U32 * kappa(w.a, w.x.shape[1]))
    check(f"M{M}", w, tangents(w, 3), "chunk3", tol)


@pytest.mark.parametrize("T", [1, 5, 63, 2049])
def test_jvp_short_signals(T):
    """Signals shorter than the order, one chunk, one segment plus one sample."""
    w = inputs.make("biquad_1024x48000", B=5, T=T, M=8, N=6, seed=60 + T)
    rng = np.random.default_rng(600 + T)
    for i in range(w.B):
        a, _, _ = inputs.draw_denominator(rng, 8, 0.3, 0.7)
        w.a[i] = a
    check(f"T{T}", w, tangents(w, 4), "chunk3", 1e-5)


@pytest.mark.parametrize("M,N", [(1, 0), (2, 2), (3, 1), (4, 4)])
def test_jvp_low_order_streaming_path(M, N):
    """Orders <= 4 on rows of a multiple of 4 samples (the float4 streaming input step):
    all tangents, then each alone; rows spanning several blocks with a partial last one."""
    w = inputs.make("biquad_1024x48000", B=5, T=2 * 8192 + 2048 + 20, M=M, N=N, seed=70 + M)
    for which in (ALL,) + tuple((k,) for k in ALL):
        check(f"vec4_M{M}_{'_'.join(which)}", w, tangents(w, 7, which), "chunk3", 1e-5)


@pytest.mark.parametrize("B,T", [(7, 4), (70000, 8)])
def test_jvp_low_order_short_rows(B, T):
    """One or two quads per row, and more rows than one grid dimension holds (the
    streaming input step strides over rows)."""
    w = inputs.make("biquad_1024x48000", B=B, T=T, seed=80 + T)
    check(f"vec4_rows_B{B}_T{T}", w, tangents(w, 8), "chunk3", 1e-5)


def test_jvp_zero_tangents_and_empty():
    """No tangent at all gives dy = 0; an empty batch is a no-op."""
    w = inputs.make("biquad_1024x48000", B=3, T=5000)
    got = run(w, tangents(w, 5, ()), "chunk3")
    assert np.array_equal(got, np.zeros_like(got))
    e = torch.empty(0, 7, device=DEV)
    dy = dfilt.dfilt_jvp(e, e, torch.ones(0, 3, device=DEV), torch.zeros(0, 2, device=DEV),
                         dx=e)
    assert dy.shape == (0, 7) and dfilt.dfilt_sync_status() == 0


def test_jvp_full_size_biquad_sampled():
    """The benchmark's workload (1024 x 48000 biquads), all tangents; sampled channels
    recomputed by the oracle, and the adjoint identity <g, dy> = <J^T g, d> over the
    whole batch against the library's own backward."""
    w = inputs.make("biquad_1024x48000")
    t = tangents(w, 6)
    got = run(w, t, "chunk3")
    idx = np.array([0, 1, 77, 255, 511, 767, 1000, 1023])
    sub = inputs.Workload(x=w.x[idx], b=w.b[idx], a=w.a[idx], zi=w.zi[idx], gy=w.gy[idx],
                          M=w.M, N=w.N, radius=w.radius[idx])
    ts = {k: v[idx] for k, v in t.items()}
    err = rel_rows(got[idx], reference(sub, ts))
    log_errors("jvp_biquad_full_sampled/chunk3", dy=err)
    assert err.max() < 1e-5, err

    o = dfilt.make_opts(algo="chunked")
    x, b, a, zi, gy = dev(w.x), dev(w.b), dev(w.a), dev(w.zi), dev(w.gy)
    y, saved = dfilt.dfilt_forward(x, b, a, zi, opts=o)
    gx, gb, ga, gzi = dfilt.dfilt_backward(gy, x, None, b, a, zi, saved, opts=o)
    # both sides in FP64 over FP32 data; the bound is the sum of the terms' magnitudes
    # (relative rounding of every term by 1e-5 moves each side by at most that much)
    pl = gy.double() * torch.from_numpy(got).to(DEV).double()
    pr = [g.double() * dev(t[k]).double()
          for g, k in [(gx, "dx"), (gb, "db"), (ga, "da"), (gzi, "dzi")]]
    lhs, rhs = float(pl.sum()), float(sum(p.sum() for p in pr))
    scale = float(pl.abs().sum()) + float(sum(p.abs().sum() for p in pr))
    assert abs(lhs - rhs) <= 1e-5 * scale, (lhs, rhs, scale)
