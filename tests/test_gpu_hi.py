"""The decoupled high-order path (orders above 8, state buckets 16/32/64: tensor-core E
pass, double-word chunk-state scan over spans joined by a bounded look-back, tensor-core
output passes) against the FP64 oracle, through the C ABI; and the workloads of the
high-order configurations (order 16 x 2^18, orders 64/64 x 2^20 at pole radius up to
0.999, the ragged 4096-channel batch) on sampled channels at full size.

Tolerances: per channel max(1e-5, 16 u32 kappa) (tests/tol.py), kappa the first-order
condition number of the recursion, and -- "equal accuracy" -- the chunked path's error
against the sequential FP32 kernel's on the same channels."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_14390_gb300 import dfilt, inputs

from tol import U32, coef_err, coef_scales, kappa, log_errors, rel_rows

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
# "Equal accuracy" of the chunked path against the sequential FP32 kernel, per channel:
# chunked error <= max(EQ x sequential error, 1e-5).  Both errors are FP32 rounding in
# the recursion amplified by the same condition number; the chunked path adds the
# split-TF32 Toeplitz products (11-bit operand pieces, the lo x lo product dropped), so
# its error may sit a small factor above the sequential kernel's on some channels.
# Measured in these tests: at most 1.8x (order 2 at radius 0.99-0.9995, grad_x); ratios
# up to 4.5x occur only on channels whose errors are both below the 1e-5 floor.
EQ = 3.0


def dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def run_fixed(w, **opt):
    o = dfilt.make_opts(**opt)
    x, b, a, zi, gy = dev(w.x), dev(w.b), dev(w.a), dev(w.zi), dev(w.gy)
    y, saved = dfilt.dfilt_forward(x, b, a, zi, opts=o)
    grads = dfilt.dfilt_backward(gy, x, None if saved is not None else y, b, a, zi, saved, opts=o)
    st = dfilt.dfilt_sync_status()
    assert st == 0, dfilt.STATUS[st]
    return y.cpu().numpy(), [g.cpu().numpy() for g in grads]


def oracle_fixed(w):
    y = oracle.forward(w.x, w.b, w.a, w.zi)
    return y, oracle.backward(w.gy, w.x, y, w.b, w.a)


def errors(w, y, grads, yr, gref):
    Sb, Sa, Su = coef_scales(w.gy, w.x, yr, w.b, w.a)
    gx, gb, ga, gz = grads
    return {"y": rel_rows(y, yr), "gx": rel_rows(gx, gref[0]), "gb": coef_err(gb, gref[1], Sb),
            "ga": coef_err(ga, gref[2], Sa), "gzi": coef_err(gz, gref[3], Su),
            # plain normwise errors of the coefficient gradients, reported beside
            "gb_norm": rel_rows(gb, gref[1]), "ga_norm": rel_rows(ga, gref[2]),
            "gzi_norm": rel_rows(gz, gref[3])}


def redraw(w, rlo, rhi, seed):
    rng = np.random.default_rng(seed)
    for i in range(w.B):
        w.a[i], w.radius[i], _ = inputs.draw_denominator(rng, w.M, rlo, rhi)
        if w.N:
            w.b[i] = inputs.draw_numerator(rng, w.N, True)


@pytest.mark.parametrize("span", [1, 4])
@pytest.mark.parametrize("M", [9, 16, 17, 32, 33, 64])
def test_decoupled_orders(M, span):
    """Every high-order state bucket and its edges, 5 tiles and a tail per channel,
    spans of 1 tile (five CTAs per channel joined by the look-back) or 4."""
    w = inputs.make("biquad_1024x48000", B=3, T=5 * 8192 + 333, M=M, N=M, seed=500 + M)
    redraw(w, 0.3, 0.7, 600 + M)
    y, g = run_fixed(w, algo="chunked", path="decoupled", span_tiles=span)
    yr, gr = oracle_fixed(w)
    e = errors(w, y, g, yr, gr)
    log_errors(f"hi_orders_M{M}_s{span}", **e)
    tol = np.maximum(1e-5, 16 * U32 * kappa(w.a, w.x.shape[1]))
    for nm in ("y", "gx", "gb", "ga", "gzi"):
        assert (e[nm] < tol).all(), (M, span, nm, e[nm], tol)


@pytest.mark.parametrize("M", [16, 32, 64])
def test_decoupled_high_radius(M):
    """Poles at radius 0.9-0.99 carried across 6 tiles in 6 spans: the states cross
    every span boundary through the look-back."""
    w = inputs.make("biquad_1024x48000", B=3, T=6 * 8192 + 77, M=M, N=M // 2, seed=700 + M)
    redraw(w, 0.9, 0.99, 710 + M)
    yr, gr = oracle_fixed(w)
    y, g = run_fixed(w, algo="chunked", path="decoupled", span_tiles=1)
    e = errors(w, y, g, yr, gr)
    ys, gs = run_fixed(w, algo="sequential")
    es = errors(w, ys, gs, yr, gr)
    log_errors(f"hi_highr_M{M}/decoupled", **e)
    log_errors(f"hi_highr_M{M}/seq", **es)
    bound = np.maximum(1e-5, 16 * U32 * kappa(w.a, w.x.shape[1]))
    for nm in ("y", "gx", "gb", "ga", "gzi"):
        assert (e[nm] < bound).all(), (M, nm, e[nm], bound)
    # the outputs at the sequential FP32 kernel's accuracy, channel by channel, within
    # the spread of two rounding orders over three channels (measured ratios 0.36-2.8)
    for nm in ("y", "gx"):
        assert (e[nm] < np.maximum(4 * es[nm], 1e-6)).all(), (M, nm, e[nm], es[nm])


def long_memory_filters(B, M, N, seed, r_long=0.999):
    """Denominators with one conjugate pole pair at radius r_long (a state that still
    carries ~0.8% of itself across a 8192-sample span) and the rest well damped
    (radius 0.3-0.6), so the look-back's span transition matters and the recursion stays
    well conditioned."""
    rng = np.random.default_rng(seed)
    a = np.zeros((B, M), dtype=np.float32)
    b = np.zeros((B, N + 1), dtype=np.float32)
    for i in range(B):
        th = rng.uniform(0.1, 3.0)
        poles = np.concatenate([[r_long * np.exp(1j * th), r_long * np.exp(-1j * th)],
                                inputs._draw_roots(rng, M - 2, 0.3, 0.6)])
        a[i] = np.real(np.poly(poles))[1:].astype(np.float32)
        assert np.abs(np.roots(np.concatenate([[1.0], a[i].astype(np.float64)]))).max() < 0.9995
        b[i] = inputs.draw_numerator(rng, N, True)
    return a, b


@pytest.mark.parametrize("M", [16, 32, 64])
def test_span_split_agrees(M):
    """Channels scanned in one span and in 1-tile spans (eight CTAs per channel joined by
    the look-back): only the span transitions and entry states differ, so the outputs
    agree to the level of FP32 rounding, and both meet the oracle."""
    w = inputs.make("biquad_1024x48000", B=4, T=8 * 8192 + 5, M=M, N=8, seed=801 + M)
    w.a, w.b = long_memory_filters(w.B, M, 8, 802 + M)
    y1, g1 = run_fixed(w, algo="chunked", path="decoupled", span_tiles=16)
    y2, g2 = run_fixed(w, algo="chunked", path="decoupled", span_tiles=1)
    yr, gr = oracle_fixed(w)
    e1, e2 = errors(w, y1, g1, yr, gr), errors(w, y2, g2, yr, gr)
    log_errors(f"span_split_M{M}/one_span", **e1)
    log_errors(f"span_split_M{M}/tile_spans", **e2)
    # the two scans differ by far less than either's error against the oracle, and the
    # split one is as accurate as the single span: both errors are the same
    # conditioning-limited rounding with independent patterns (the span transitions and
    # entry states round differently), so their per-channel maxima differ by an O(1)
    # factor (measured up to 1.65x, on grad_b at order 64)
    for nm, a1, a2 in (("y", y1, y2), ("gx", g1[0], g2[0])):
        assert (rel_rows(a2, a1) <= np.maximum(1e-5, e1[nm])).all(), (M, nm)
    for nm in ("y", "gx", "gb", "ga", "gzi"):
        assert (e2[nm] <= np.maximum(1e-5, 2.0 * e1[nm])).all(), (M, nm, e2[nm], e1[nm])


def test_decoupled_matches_fused():
    """The decoupled and single-kernel paths are the same chunk algebra: on an order-16
    batch both meet the oracle bound, and they agree with each other to the same level."""
    w = inputs.make("allpole16_256x262144", B=4, T=4 * 8192 + 999, seed=811)
    yr, gr = oracle_fixed(w)
    yd, gd = run_fixed(w, algo="chunked", path="decoupled", span_tiles=1)
    yf, gf = run_fixed(w, algo="chunked", path="fused")
    bound = np.maximum(1e-5, 16 * U32 * kappa(w.a, w.x.shape[1]))
    for tag, (y, g) in (("decoupled", (yd, gd)), ("fused", (yf, gf))):
        e = errors(w, y, g, yr, gr)
        log_errors(f"hi_vs_fused/{tag}", **e)
        for nm in ("y", "gx", "ga", "gzi"):
            assert (e[nm] < bound).all(), (tag, nm, e[nm], bound)
    assert (rel_rows(yd, yf) < 2 * bound).all()


def test_decoupled_deterministic():
    """Work items are taken from counters in a run-dependent order, but every reduction
    runs in a fixed order: two backward calls give bit-identical gradients."""
    w = inputs.make("biquad_1024x48000", B=6, T=7 * 8192 + 901, M=32, N=32, seed=821)
    redraw(w, 0.5, 0.95, 822)
    o = dfilt.make_opts(algo="chunked", path="decoupled", span_tiles=2)
    x, b, a, zi, gy = dev(w.x), dev(w.b), dev(w.a), dev(w.zi), dev(w.gy)
    y, saved = dfilt.dfilt_forward(x, b, a, zi, opts=o)
    g1 = [t.clone() for t in dfilt.dfilt_backward(gy, x, None, b, a, zi, saved, opts=o)]
    g2 = dfilt.dfilt_backward(gy, x, None, b, a, zi, saved, opts=o)
    g3 = dfilt.dfilt_backward(gy, x, y, b, a, zi, saved, opts=o)   # y given: no recompute
    assert dfilt.dfilt_sync_status() == 0
    for t1, t2 in zip(g1, g2):
        assert torch.equal(t1, t2)
    yr, gr = oracle_fixed(w)
    tol = np.maximum(1e-5, 16 * U32 * kappa(w.a, w.x.shape[1]))
    e3 = errors(w, y.cpu().numpy(), [t.cpu().numpy() for t in g3], yr, gr)
    for nm in ("gx", "gb", "ga", "gzi"):
        assert (e3[nm] < tol).all(), (nm, e3[nm])


def test_fused_low_order_deterministic():
    """The single-kernel backward (orders <= 8) sums its lag products in fixed slots:
    repeated calls over a batch whose channels land on different CTAs from run to run
    give bit-identical coefficient gradients."""
    w = inputs.make("biquad_1024x48000", B=300, T=3 * 8192 + 17, M=8, N=8, seed=831)
    redraw(w, 0.5, 0.95, 832)
    o = dfilt.make_opts(algo="chunked")
    x, b, a, zi, gy = dev(w.x), dev(w.b), dev(w.a), dev(w.zi), dev(w.gy)
    y, saved = dfilt.dfilt_forward(x, b, a, zi, opts=o)
    ref = [t.clone() for t in dfilt.dfilt_backward(gy, x, None, b, a, zi, saved, opts=o)]
    for _ in range(3):
        g = dfilt.dfilt_backward(gy, x, None, b, a, zi, saved, opts=o)
        for t1, t2 in zip(ref, g):
            assert torch.equal(t1, t2)
    assert dfilt.dfilt_sync_status() == 0


def _placement_run(w, opts, reps=1, tuning=None):
    """fwd + bwd of a batch whose channels are w's channels repeated `reps` times."""
    rep = lambda v: None if v is None else np.concatenate([v] * reps, axis=0)
    x, b, a, zi, gy = dev(rep(w.x)), dev(rep(w.b)), dev(rep(w.a)), dev(rep(w.zi)), dev(rep(w.gy))
    o = dfilt.make_opts(**opts)
    if tuning:
        dfilt.dfilt_tuning_set(*tuning)
    try:
        y, saved = dfilt.dfilt_forward(x, b, a, zi, opts=o)
        g = dfilt.dfilt_backward(gy, x, None, b, a, zi, saved, opts=o)
    finally:
        if tuning:
            dfilt.dfilt_tuning_set(tuning[0], 0, 0)
    assert dfilt.dfilt_sync_status() == 0
    return [t.cpu() for t in (y, *g)]


@pytest.mark.parametrize("M,opts,tune", [
    (2, dict(algo="chunked"), None),
    (8, dict(algo="chunked", path="fused"), None),
    (16, dict(algo="chunked", path="decoupled", span_tiles=2), (16, 2, 4)),
    (32, dict(algo="chunked", path="decoupled", span_tiles=2), (32, 2, 16)),
])
def test_results_independent_of_channel_placement(M, opts, tune):
    """Every reduction runs in a fixed order, so a channel's outputs and gradients do not
    depend on which CTA, tile group or work item it lands on: the same channels filtered
    alone, as the second copy in a doubled batch (other CTAs, other tile parities, other
    work-item order) and, on the decoupled path, with another number of scan chains per
    SM give bit-identical y, grad_x, grad_b, grad_a and grad_zi."""
    w = inputs.make("biquad_1024x48000", B=37, T=3 * 8192 + 1234, M=M, N=M, seed=860 + M)
    redraw(w, 0.5, 0.97, 870 + M)
    base = _placement_run(w, opts)
    dbl = _placement_run(w, opts, reps=2)
    B = w.B
    for t0, t2 in zip(base, dbl):
        assert torch.equal(t2[:B], t0) and torch.equal(t2[B:], t0)
    if tune:
        other = _placement_run(w, opts, tuning=tune)
        for t0, t1 in zip(base, other):
            assert torch.equal(t1, t0)


def test_decoupled_ragged():
    """Ragged batch over every bucket (orders 1..64; 16, 32 and 64 take the decoupled
    path), lengths up to 9 tiles split into 2-tile spans, empty channels."""
    w = inputs.make_ragged(B=30, T_range=(1, 70000), M_range=(1, 64), seed=841)
    lens = np.diff(w.offsets)
    lens[[4, 11]] = 0
    offs = np.zeros_like(w.offsets)
    offs[1:] = np.cumsum(lens)
    w.x = np.concatenate([w.x[w.offsets[i]:w.offsets[i] + lens[i]] for i in range(w.B)])
    w.gy = np.concatenate([w.gy[w.offsets[i]:w.offsets[i] + lens[i]] for i in range(w.B)])
    w.offsets = offs
    o = dfilt.make_opts(algo="chunked", path="decoupled", span_tiles=2)
    dx, dgy = dev(w.x), dev(w.gy)
    doffs, dMs, dNs = dev(w.offsets), dev(w.Ms), dev(w.Ns)
    db, da, dzi = dev(w.b), dev(w.a), dev(w.zi)
    y, saved = dfilt.dfilt_forward_ragged(dx, doffs, dMs, dNs, db, da, dzi, opts=o)
    g = dfilt.dfilt_backward_ragged(dgy, dx, None, doffs, dMs, dNs, db, da, dzi, saved, opts=o)
    assert dfilt.dfilt_sync_status() == 0
    y = y.cpu().numpy()
    gx, gb, ga, gz = [t.cpu().numpy() for t in g]
    yr = oracle.forward_ragged(w.x, w.offsets, w.Ms, w.Ns, w.b, w.a, w.zi)
    gr = oracle.backward_ragged(w.gy, w.x, yr, w.offsets, w.Ms, w.Ns, w.b, w.a)
    for i in range(w.B):
        s, e = w.offsets[i], w.offsets[i + 1]
        M, N = int(w.Ms[i]), int(w.Ns[i])
        if e == s:
            assert not gb[i].any() and not ga[i].any() and not gz[i].any()
            continue
        tol = max(1e-5, 16 * U32 * float(kappa(w.a[i:i + 1, :M], e - s)[0]))
        Sb, Sa, Su = coef_scales(w.gy[s:e], w.x[s:e], yr[s:e], w.b[i, :N + 1], w.a[i, :M])
        assert rel_rows(y[s:e], yr[s:e])[0] < tol, (i, M)
        assert rel_rows(gx[s:e], gr[0][s:e])[0] < tol, (i, M)
        assert coef_err(gb[i, :N + 1], gr[1][i, :N + 1], Sb)[0] < tol, (i, M)
        assert coef_err(ga[i, :M], gr[2][i, :M], Sa)[0] < tol, (i, M)
        assert coef_err(gz[i, :M], gr[3][i, :M], Su)[0] < tol, (i, M)


def test_order64_config():
    """The orders-64/64 configuration's filters (poles at radius 0.9-0.999, numerator
    scaled to max |b| = 1, random initial state) over 6 tiles: decoupled path (3 spans),
    single-kernel path and sequential kernel against the oracle.  Both chunked paths
    stay within the first-order bound and within EQ x the sequential FP32 kernel's
    error on every channel."""
    w = inputs.make("df64_64x1048576", B=4, T=6 * 8192 + 111)
    yr, gr = oracle_fixed(w)
    res = {"decoupled": run_fixed(w, algo="chunked", path="decoupled", span_tiles=2),
           "fused": run_fixed(w, algo="chunked", path="fused"),
           "seq": run_fixed(w, algo="sequential")}
    e = {k: errors(w, y, g, yr, gr) for k, (y, g) in res.items()}
    for k in e:
        log_errors(f"c4_6tiles/{k}", radius=w.radius, **e[k])
    bound = np.maximum(1e-5, 16 * U32 * kappa(w.a, w.x.shape[1]))
    for k in ("decoupled", "fused"):
        for nm in ("y", "gx", "gb", "ga", "gzi"):
            assert (e[k][nm] < bound).all(), (k, nm, e[k][nm], bound)
        for nm in ("y", "gx"):
            assert (e[k][nm] <= np.maximum(EQ * e["seq"][nm], 1e-5)).all(), (k, nm, e[k][nm],
                                                                              e["seq"][nm])


def test_order64_full_length_sampled():
    """The orders-64/64 workload at full size (64 x 2^20) in the benchmark's launch
    configuration; three channels recomputed by the oracle over their whole length."""
    w = inputs.make("df64_64x1048576")
    y, g = run_fixed(w, algo="chunked")
    idx = np.array([0, 31, 63])
    sub = inputs.Workload(x=w.x[idx], b=w.b[idx], a=w.a[idx], zi=w.zi[idx], gy=w.gy[idx],
                          M=w.M, N=w.N, radius=w.radius[idx])
    yr, gr = oracle_fixed(sub)
    e = errors(sub, y[idx], [t[idx] for t in g], yr, gr)
    log_errors("c4_full_sampled", radius=sub.radius, **e)
    bound = np.maximum(1e-5, 16 * U32 * kappa(sub.a, 1 << 16))
    for nm in ("y", "gx", "gb", "ga", "gzi"):
        assert (e[nm] < bound).all(), (nm, e[nm], bound)


def test_order16_full_size_sampled():
    """The order-16 workload at full size (256 x 2^18); four channels recomputed."""
    w = inputs.make("allpole16_256x262144")
    y, g = run_fixed(w, algo="chunked")
    idx = np.array([0, 100, 200, 255])
    sub = inputs.Workload(x=w.x[idx], b=w.b[idx], a=w.a[idx], zi=None, gy=w.gy[idx],
                          M=w.M, N=w.N, radius=w.radius[idx])
    yr, gr = oracle_fixed(sub)
    gx, gb, ga, gz = [t[idx] for t in g]
    e = errors(sub, y[idx], [gx, gb, ga, gz], yr, gr)
    log_errors("c3_full_sampled", radius=sub.radius, **e)
    bound = np.maximum(1e-5, 16 * U32 * kappa(sub.a, 1 << 16))
    for nm in ("y", "gx", "ga", "gzi"):
        assert (e[nm] < bound).all(), (nm, e[nm], bound)


def test_ragged4096_full_size_sampled():
    """The ragged workload at full size (4096 filters, orders 1..32, lengths 1e3..1e6,
    about 594M samples) in the benchmark's configuration; eight channels from every
    state bucket recomputed by the oracle."""
    w = inputs.make_ragged("ragged4096")
    o = dfilt.make_opts(algo="chunked")
    dx, dgy = dev(w.x), dev(w.gy)
    doffs, dMs, dNs = dev(w.offsets), dev(w.Ms), dev(w.Ns)
    db, da, dzi = dev(w.b), dev(w.a), dev(w.zi)
    y, saved = dfilt.dfilt_forward_ragged(dx, doffs, dMs, dNs, db, da, dzi, opts=o)
    g = dfilt.dfilt_backward_ragged(dgy, dx, y, doffs, dMs, dNs, db, da, dzi, saved, opts=o)
    assert dfilt.dfilt_sync_status() == 0
    lens = np.diff(w.offsets)
    pick = []
    for lo, hi in ((1, 2), (3, 4), (5, 8), (9, 16), (17, 32)):
        cand = np.where((w.Ms >= lo) & (w.Ms <= hi) & (lens < 300_000))[0]
        pick += list(cand[:2]) if hi >= 16 else list(cand[:1])
    longest = int(np.argmax(lens))
    pick.append(longest)
    for i in pick:
        s, e = int(w.offsets[i]), int(w.offsets[i + 1])
        M, N = int(w.Ms[i]), int(w.Ns[i])
        xs, gys = w.x[s:e][None], w.gy[s:e][None]
        bs, as_, zs = w.b[i:i + 1, :N + 1], w.a[i:i + 1, :M], w.zi[i:i + 1, :M]
        yr = oracle.forward(xs, bs, as_, zs)
        gr = oracle.backward(gys, xs, yr, bs, as_)
        ys = y[s:e].cpu().numpy()[None]
        gx = g[0][s:e].cpu().numpy()[None]
        gb = g[1][i:i + 1, :N + 1].cpu().numpy()
        ga = g[2][i:i + 1, :M].cpu().numpy()
        gz = g[3][i:i + 1, :M].cpu().numpy()
        Sb, Sa, Su = coef_scales(gys, xs, yr, bs, as_)
        tol = max(1e-5, 16 * U32 * float(kappa(as_, min(e - s, 1 << 16))[0]))
        errs = {"y": rel_rows(ys, yr)[0], "gx": rel_rows(gx, gr[0])[0],
                "gb": coef_err(gb, gr[1], Sb)[0], "ga": coef_err(ga, gr[2], Sa)[0],
                "gzi": coef_err(gz, gr[3], Su)[0]}
        log_errors(f"c5_full_sampled/ch{i}_M{M}_T{e - s}", **errs)
        for nm, v in errs.items():
            assert v < tol, (i, M, e - s, nm, v, tol)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_low_order_near_unit_circle(M):
    """Orders <= 4 with poles at radius 0.99-0.9995 over 16 tiles.  The automatic scan
    choice (FP32 two-level scan for orders <= 2, double words above) must meet the same
    per-channel bound as the forced double-word scan and stay within EQ x the
    sequential FP32 kernel's error.  (At order 4 an FP32 scan measured 21x the
    double-word scan's error on one such channel, which is why orders 3 and 4 take the
    double-word scan.)"""
    w = inputs.make("biquad_1024x48000", B=16, T=16 * 8192 + 3, M=M, N=M, seed=900 + M)
    redraw(w, 0.99, 0.9995, 910 + M)
    yr, gr = oracle_fixed(w)
    res = {"auto": run_fixed(w, algo="chunked"),
           "dw": run_fixed(w, algo="chunked", fp64_scan=1),
           "seq": run_fixed(w, algo="sequential")}
    e = {k: errors(w, y, g, yr, gr) for k, (y, g) in res.items()}
    for k in e:
        log_errors(f"lowM{M}_unit/{k}", radius=w.radius, **e[k])
    bound = np.maximum(1e-5, 16 * U32 * kappa(w.a, w.x.shape[1]))
    for k in ("auto", "dw"):
        for nm in ("y", "gx", "gb", "ga", "gzi"):
            assert (e[k][nm] < bound).all(), (k, nm, e[k][nm], bound)
        for nm in ("y", "gx"):
            assert (e[k][nm] <= np.maximum(EQ * e["seq"][nm], 1e-5)).all(), (k, nm, e[k][nm],
                                                                              e["seq"][nm])
