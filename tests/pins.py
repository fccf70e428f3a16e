"""Pins for the FP64 oracle: checks against things the paper and the mathematics
fix, independent of the oracle's own code.  Each function raises AssertionError
on failure and takes an optional ``lib`` (a loaded oracle variant), so the same
pins can be run against a copy of the oracle with a planted mistake.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

import oracle
from oracle import pyref


def _rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    if not (np.iscomplexobj(a) or np.iscomplexobj(b)):
        a = a.astype(np.float64)
        b = b.astype(np.float64)
    den = max(np.abs(b).max(), 1e-300)
    return float(np.abs(a - b).max() / den)


# --------------------------------------------------------------------------
# forward pins
# --------------------------------------------------------------------------

def pin_single_pole(lib=None):
    """a = [-p], b = [c]: impulse response c p^n (geometric series)."""
    for p, c in [(0.9, 1.0), (-0.75, 2.5), (0.5, -1.0)]:
        T = 200
        x = np.zeros((1, T)); x[0, 0] = 1.0
        y = oracle.forward(x, [[c]], [[-p]], lib=lib)
        ref = c * p ** np.arange(T)
        assert _rel(y[0], ref) < 1e-13, ("single pole", p)


def pin_biquad_allpole(lib=None):
    """Poles r e^{+-i th}: a = [-2 r cos th, r^2], h[n] = r^n sin((n+1) th) / sin th."""
    for r, th in [(0.95, 0.3), (0.6, 2.0), (0.99, 1.1)]:
        T = 500
        x = np.zeros((1, T)); x[0, 0] = 1.0
        y = oracle.forward(x, [[1.0]], [[-2 * r * np.cos(th), r * r]], lib=lib)
        n = np.arange(T)
        ref = r ** n * np.sin((n + 1) * th) / np.sin(th)
        assert _rel(y[0], ref) < 1e-12, ("biquad", r, th)


def _random_filter(rng, M, N, rmax=0.9):
    poles = []
    for _ in range(M // 2):
        r, th = rng.uniform(0.3, rmax), rng.uniform(0, np.pi)
        poles += [r * np.exp(1j * th), r * np.exp(-1j * th)]
    if M % 2:
        poles.append(rng.uniform(-rmax, rmax))
    a = np.real(np.poly(poles))[1:]
    b = rng.standard_normal(N + 1)
    return b, a


def pin_transfer_function(lib=None):
    """The DFT of a long impulse response equals B(e^{jw}) / A(e^{jw}) at w = 2 pi k / K
    (Eq. rtf), up to the truncation r^K."""
    rng = np.random.default_rng(11)
    for M, N in [(1, 0), (2, 2), (5, 3), (8, 8)]:
        b, a = _random_filter(rng, M, N, rmax=0.9)
        K = 4096
        x = np.zeros((1, K)); x[0, 0] = 1.0
        h = oracle.forward(x, b[None], a[None], lib=lib)[0]
        Hfft = np.fft.fft(h)
        zinv = np.exp(-2j * np.pi * np.arange(K) / K)
        num = np.polyval(b[::-1], zinv)
        den = np.polyval(np.concatenate([[1.0], a])[::-1], zinv)
        assert _rel(Hfft, num / den) < 1e-10, ("transfer function", M, N)


def pin_lfilter(lib=None):
    """Library cross-check: SciPy lfilter (TDF-II with zi), called, never copied."""
    import scipy.signal as ss
    rng = np.random.default_rng(12)
    for M, N, T in [(1, 0, 50), (2, 2, 300), (3, 1, 257), (6, 6, 400), (9, 4, 130)]:
        b, a = _random_filter(rng, M, N, rmax=0.95)
        x = rng.standard_normal(T)
        zi = rng.standard_normal(M)
        y = oracle.forward(x[None], b[None], a[None], zi[None], lib=lib)[0]
        bp = np.zeros(M + 1); bp[: N + 1] = b
        ref, _ = ss.lfilter(bp, np.concatenate([[1.0], a]), x, zi=zi)
        assert _rel(y, ref) < 1e-12, ("lfilter", M, N)


def pin_injection_form(lib=None):
    """TDF-II initial state == injecting zi into the all-pole input at times 0..M-1."""
    rng = np.random.default_rng(13)
    for M, N, T in [(1, 1, 20), (4, 2, 100), (7, 7, 3), (3, 0, 64)]:
        b, a = _random_filter(rng, M, N)
        x = rng.standard_normal((2, T))
        zi = rng.standard_normal((2, M))
        B2 = np.stack([b, b]); A2 = np.stack([a, a])
        y1 = oracle.forward(x, B2, A2, zi, form="tdf2", lib=lib)
        y2 = oracle.forward(x, B2, A2, zi, form="injection", lib=lib)
        assert _rel(y1, y2) < 1e-12, ("injection", M, N, T)


def pin_linearity_shift(lib=None):
    """y(x, zi) = y(x, 0) + y(0, zi); zero-state response is shift invariant."""
    rng = np.random.default_rng(14)
    M, N, T = 4, 3, 120
    b, a = _random_filter(rng, M, N)
    x = rng.standard_normal((1, T)); zi = rng.standard_normal((1, M))
    f = lambda xx, zz: oracle.forward(xx, b[None], a[None], zz, lib=lib)
    assert _rel(f(x, zi), f(x, None) + f(np.zeros_like(x), zi)) < 1e-12
    s = 17
    xs = np.zeros_like(x); xs[0, s:] = x[0, : T - s]
    assert _rel(f(xs, None)[0, s:], f(x, None)[0, : T - s]) < 1e-12


def _exact_forward(x, b, a, zi):
    return pyref.forward(x, b, a, zi)


def pin_exact_forward(lib=None):
    """Exact rational arithmetic (Fractions) through the difference equation."""
    b = [Fraction(1), Fraction(1, 2)]
    a = [Fraction(-1, 2)]
    x = [Fraction(1), Fraction(2), Fraction(0), Fraction(0)]
    zi = [Fraction(1, 4)]
    y = _exact_forward(x, b, a, zi)
    # by hand: y0 = 1 + 1/4; y1 = 2 + 1/2*1 + 1/2*y0; y2 = 1/2*2 + 1/2*y1; y3 = 1/2*y2
    assert y == [Fraction(5, 4), Fraction(25, 8), Fraction(41, 16), Fraction(41, 32)]
    yo = oracle.forward(np.array([[1.0, 2, 0, 0]]), [[1.0, 0.5]], [[-0.5]], [[0.25]], lib=lib)
    assert np.array_equal(yo[0], np.array([float(v) for v in y]))


# --------------------------------------------------------------------------
# backward pins
# --------------------------------------------------------------------------

def _rat_filter(rng, M, N):
    """Small random stable rational coefficients."""
    b = [Fraction(int(rng.integers(-8, 9)), 8) for _ in range(N + 1)]
    a = [Fraction(int(rng.integers(-3, 4)), 16) for _ in range(M)]
    return b, a


def pin_exact_gradients(lib=None):
    """Brute force in exact rationals.

    The filter is linear in (x, zi): column j of the Jacobian is the response to a
    unit impulse, so grad_x = J_x^T g and grad_zi = J_zi^T g exactly.  It is
    nonlinear in (a, b): there the exact directional derivatives come from
    forward-mode tangents of the difference equation,
        dy/db_k = (1/A) [x delayed by k],
        dy/da_k = (1/A) [-(y delayed by k)],
    (differentiate y[n] + sum a_k y[n-k] = sum b_k x[n-k] + zi-injection), and
    grad_theta = <g, dy/dtheta>.  The oracle's FP64 adjoint must agree to rounding.
    """
    rng = np.random.default_rng(21)
    for M, N, T in [(1, 0, 5), (2, 2, 7), (3, 1, 9), (4, 4, 6), (3, 3, 2)]:
        b, a = _rat_filter(rng, M, N)
        x = [Fraction(int(rng.integers(-9, 10)), 4) for _ in range(T)]
        zi = [Fraction(int(rng.integers(-9, 10)), 4) for _ in range(M)]
        g = [Fraction(int(rng.integers(-9, 10)), 4) for _ in range(T)]
        zero = [Fraction(0)] * T
        y = pyref.forward(x, b, a, zi)
        gx = []
        for j in range(T):
            e = [Fraction(0)] * T; e[j] = Fraction(1)
            col = pyref.forward(e, b, a, None)
            gx.append(sum(gi * ci for gi, ci in zip(g, col)))
        gzi = []
        for k in range(M):
            e = [Fraction(0)] * M; e[k] = Fraction(1)
            col = pyref.forward(zero, b, a, e)
            gzi.append(sum(gi * ci for gi, ci in zip(g, col)))
        allpole = lambda s: pyref.forward(s, [Fraction(1)], a, None)
        gb = []
        for k in range(N + 1):
            xd = [x[n - k] if n - k >= 0 else Fraction(0) for n in range(T)]
            gb.append(sum(gi * ti for gi, ti in zip(g, allpole(xd))))
        ga = []
        for k in range(1, M + 1):
            yd = [-y[n - k] if n - k >= 0 else Fraction(0) for n in range(T)]
            ga.append(sum(gi * ti for gi, ti in zip(g, allpole(yd))))
        f = lambda v: np.array([float(t) for t in v])[None]
        ox, ob, oa, oz = oracle.backward(f(g), f(x), f(y), f(b), f(a), lib=lib)
        for got, ref, nm in [(ox, gx, "x"), (ob, gb, "b"), (oa, ga, "a"), (oz, gzi, "zi")]:
            ref = np.array([float(t) for t in ref])
            assert _rel(got[0], ref) < 1e-12 or np.abs(got[0] - ref).max() < 1e-13, \
                ("exact gradient", nm, M, N, T)


def pin_finite_differences(lib=None):
    """FP64 central differences of L = <g, y> with respect to a, b, zi, x."""
    rng = np.random.default_rng(22)
    for M, N, T in [(2, 2, 64), (5, 3, 48), (1, 0, 30)]:
        b, a = _random_filter(rng, M, N, rmax=0.8)
        x = rng.standard_normal(T); zi = rng.standard_normal(M); g = rng.standard_normal(T)
        L = lambda bb, aa, zz, xx: float(g @ oracle.forward(xx[None], bb[None], aa[None],
                                                            zz[None], lib=lib)[0])
        y = oracle.forward(x[None], b[None], a[None], zi[None], lib=lib)
        gx, gb, ga, gz = oracle.backward(g[None], x[None], y, b[None], a[None], lib=lib)
        h = 1e-6
        def fd(vec, which):
            out = np.zeros_like(vec)
            for i in range(vec.size):
                vp, vm = vec.copy(), vec.copy(); vp[i] += h; vm[i] -= h
                args_p = dict(bb=b, aa=a, zz=zi, xx=x); args_m = dict(bb=b, aa=a, zz=zi, xx=x)
                args_p[which] = vp; args_m[which] = vm
                out[i] = (L(**args_p) - L(**args_m)) / (2 * h)
            return out
        assert _rel(gb[0], fd(b, "bb")) < 1e-7, ("fd b", M, N)
        assert _rel(ga[0], fd(a, "aa")) < 1e-7, ("fd a", M, N)
        assert _rel(gz[0], fd(zi, "zz")) < 1e-7, ("fd zi", M, N)
        assert _rel(gx[0][:8], fd(x, "xx")[:8]) < 1e-7, ("fd x", M, N)


def pin_duality(lib=None):
    """grad_x is the same (b, a) filter run time-reversed on g with zero state
    (Sec. 3.1: the adjoint of the form is a filter running backwards in time)."""
    rng = np.random.default_rng(23)
    for M, N, T in [(2, 2, 300), (6, 4, 77)]:
        b, a = _random_filter(rng, M, N)
        x = rng.standard_normal((1, T)); g = rng.standard_normal((1, T))
        y = oracle.forward(x, b[None], a[None], lib=lib)
        gx = oracle.backward(g, x, y, b[None], a[None], lib=lib)[0]
        rev = oracle.forward(g[:, ::-1], b[None], a[None], lib=lib)[:, ::-1]
        assert _rel(gx, rev) < 1e-12, ("duality", M, N)


def pin_statespace(lib=None):
    """App. B operator under the Sec. 2 mapping gives the same output and gradients."""
    from oracle import statespace
    rng = np.random.default_rng(24)
    for M, N, T in [(1, 1, 40), (2, 2, 100), (5, 2, 64), (4, 0, 33)]:
        b, a = _random_filter(rng, M, N)
        x = rng.standard_normal(T); zi = rng.standard_normal(M); g = rng.standard_normal(T)
        y_ss, gx_ss, gb_ss, ga_ss, gz_ss = statespace.tdf_filter_and_grads(x, b, a, zi, g)
        y = oracle.forward(x[None], b[None], a[None], zi[None], lib=lib)
        gx, gb, ga, gz = oracle.backward(g[None], x[None], y, b[None], a[None], lib=lib)
        for got, ref, nm in [(y[0], y_ss, "y"), (gx[0], gx_ss, "gx"), (gb[0], gb_ss, "gb"),
                             (ga[0], ga_ss, "ga"), (gz[0], gz_ss, "gzi")]:
            assert _rel(got, ref) < 1e-11, ("state space", nm, M, N)


def pin_jvp_single_pole(lib=None):
    """Forward mode, closed form.  One pole, impulse input, x = delta, zero numerator
    tail: y[n] = b0 (-a)^n, so dy/da = -n b0 (-a)^(n-1), dy/db0 = (-a)^n, and the
    initial state's tangent reaches the output as dzi (-a)^n (TDF-II, M = 1)."""
    T, b0, a1 = 40, 0.7, -0.93
    x = np.zeros((1, T)); x[0, 0] = 1.0
    b, a, zi = np.array([[b0, 0.0]]), np.array([[a1]]), np.zeros((1, 1))
    n = np.arange(T, dtype=np.float64)
    p = (-a1) ** n
    dp = np.concatenate([[0.0], n[1:] * (-a1) ** (n[1:] - 1)])   # d/dr of r^n at r = -a1
    one = np.ones((1, 1))
    y, dy = oracle.jvp(x, b, a, zi, da=one, lib=lib)
    assert _rel(y[0], b0 * p) < 1e-14, "jvp primal"
    assert _rel(dy[0], -b0 * dp) < 1e-13, "jvp d/da"
    _, dy = oracle.jvp(x, b, a, zi, db=np.array([[1.0, 0.0]]), lib=lib)
    assert _rel(dy[0], p) < 1e-14, "jvp d/db0"
    _, dy = oracle.jvp(x, b, a, zi, db=np.array([[0.0, 1.0]]), lib=lib)
    assert _rel(dy[0], np.concatenate([[0.0], p[:-1]])) < 1e-14, "jvp d/db1"
    _, dy = oracle.jvp(x, b, a, zi, dzi=2.5 * one, lib=lib)
    assert _rel(dy[0], 2.5 * p) < 1e-14, "jvp d/dzi"
    _, dy = oracle.jvp(x, b, a, zi, dx=x, lib=lib)
    assert _rel(dy[0], b0 * p) < 1e-14, "jvp d/dx"


def pin_jvp_finite_differences(lib=None):
    """Forward mode against FP64 central differences of the forward along one joint
    direction in (x, b, a, zi)."""
    rng = np.random.default_rng(25)
    for M, N, T in [(2, 2, 64), (5, 3, 48), (1, 0, 30), (4, 4, 3)]:
        b, a = _random_filter(rng, M, N, rmax=0.8)
        x = rng.standard_normal(T); zi = rng.standard_normal(M)
        dx, db, da, dz = (rng.standard_normal(v.shape) for v in (x, b, a, zi))
        h = 1e-6
        f = lambda s: oracle.forward((x + s * dx)[None], (b + s * db)[None], (a + s * da)[None],
                                     (zi + s * dz)[None], lib=lib)[0]
        fd = (f(h) - f(-h)) / (2 * h)
        y, dy = oracle.jvp(x[None], b[None], a[None], zi[None], dx[None], db[None], da[None],
                           dz[None], lib=lib)
        assert _rel(y[0], f(0.0)) < 1e-14, ("jvp primal", M, N)
        assert _rel(dy[0], fd) < 1e-7, ("jvp fd", M, N)


def pin_jvp_adjoint(lib=None):
    """Forward and reverse mode are transposes of one linear map:
    <g, J d> = <J^T g, d> with J^T g the backward's (grad_x, grad_b, grad_a, grad_zi)."""
    rng = np.random.default_rng(26)
    for M, N, T in [(2, 2, 200), (6, 4, 77), (3, 0, 5)]:
        b, a = _random_filter(rng, M, N)
        x = rng.standard_normal((1, T)); zi = rng.standard_normal((1, M))
        g = rng.standard_normal((1, T))
        dx, db, da, dz = (rng.standard_normal(v.shape) for v in (x, b[None], a[None], zi))
        y, dy = oracle.jvp(x, b[None], a[None], zi, dx, db, da, dz, lib=lib)
        gx, gb, ga, gz = oracle.backward(g, x, y, b[None], a[None], lib=lib)
        lhs = float((g * dy).sum())
        rhs = float((gx * dx).sum() + (gb * db).sum() + (ga * da).sum() + (gz * dz).sum())
        assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + abs(rhs) + 1.0), ("jvp adjoint", M, N)


def pin_recurrence_dense(lib=None):
    """App. B operator with a dense (non-companion) A: a diagonal A gives per-component
    geometric sums in closed form; a rotation by theta scaled by r gives
    v(n) = r^n R(n theta) v0 for z = 0; and the backward's (grad_A, grad_v0, grad_z)
    equal FP64 central differences of <g, v> (lib unused: numpy operator)."""
    from oracle import statespace as ss
    rng = np.random.default_rng(27)
    lam = np.array([0.9, -0.6, 0.3])
    v0 = rng.standard_normal(3); z = rng.standard_normal((25, 3))
    v = ss.recurrence_forward(np.diag(lam), v0, z)
    for i in range(3):
        ref = [lam[i] ** (n + 1) * v0[i] + sum(lam[i] ** (n - k) * z[k, i] for k in range(n + 1))
               for n in range(25)]
        assert _rel(v[:, i], ref) < 1e-13, "recurrence diagonal"
    r, th = 0.97, 0.4
    Rm = r * np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    w0 = np.array([1.0, -0.5])
    v = ss.recurrence_forward(Rm, w0, np.zeros((30, 2)))
    for n in range(30):
        c, s_ = np.cos((n + 1) * th), np.sin((n + 1) * th)
        ref = r ** (n + 1) * np.array([[c, -s_], [s_, c]]) @ w0
        assert _rel(v[n], ref) < 1e-13, "recurrence rotation"
    for M, T in [(2, 40), (4, 17)]:
        A = 0.5 * rng.standard_normal((M, M)) / np.sqrt(M)
        v0 = rng.standard_normal(M); z = rng.standard_normal((T, M)); g = rng.standard_normal((T, M))
        v = ss.recurrence_forward(A, v0, z)
        gA, gv0, gz = ss.recurrence_backward(A, v0, v, g)
        L = lambda AA, vv, zz: float((g * ss.recurrence_forward(AA, vv, zz)).sum())
        h = 1e-6
        def fd(arr, which):
            out = np.zeros_like(arr)
            for idx in np.ndindex(arr.shape):
                ap, am = arr.copy(), arr.copy(); ap[idx] += h; am[idx] -= h
                kp = dict(AA=A, vv=v0, zz=z); km = dict(AA=A, vv=v0, zz=z)
                kp[which] = ap; km[which] = am
                out[idx] = (L(**kp) - L(**km)) / (2 * h)
            return out
        assert _rel(gA, fd(A, "AA")) < 1e-7, ("recurrence fd A", M)
        assert _rel(gv0, fd(v0, "vv")) < 1e-7, ("recurrence fd v0", M)
        assert _rel(gz, fd(z, "zz")) < 1e-7, ("recurrence fd z", M)


def pin_df1_initial_conditions(lib=None):
    """Direct-form initial conditions (past inputs and outputs): the forward equals
    SciPy's lfiltic + lfilter (library routines); zero past values reduce to the
    zero-state filter; the gradients equal FP64 central differences of <g, y> with
    respect to x, b, a, xpast and ypast."""
    import scipy.signal as ss
    rng = np.random.default_rng(28)
    for M, N, T in [(2, 2, 60), (5, 3, 40), (3, 0, 25), (4, 4, 3)]:
        b, a = _random_filter(rng, M, N, rmax=0.8)
        x = rng.standard_normal(T); xp = rng.standard_normal(N); yp = rng.standard_normal(M)
        af = np.concatenate([[1.0], a])
        y = oracle.forward_df1(x[None], b[None], a[None], xp[None], yp[None], lib=lib)[0]
        ref, _ = ss.lfilter(b, af, x, zi=ss.lfiltic(b, af, yp, xp if N else None))
        assert _rel(y, ref) < 1e-12, ("df1 lfiltic", M, N)
        y0 = oracle.forward_df1(x[None], b[None], a[None], np.zeros((1, N)), np.zeros((1, M)),
                                lib=lib)[0]
        assert _rel(y0, ss.lfilter(b, af, x)) < 1e-12, ("df1 zero past", M, N)
        g = rng.standard_normal(T)
        gx, gb, ga, gxp, gyp = oracle.backward_df1(g[None], x[None], y[None], b[None], a[None],
                                                   xp[None], yp[None], lib=lib)
        L = lambda xx, bb, aa, xq, yq: float(g @ oracle.forward_df1(
            xx[None], bb[None], aa[None], xq[None], yq[None], lib=lib)[0])
        h = 1e-6
        args = dict(xx=x, bb=b, aa=a, xq=xp, yq=yp)
        for nm, got in [("xx", gx[0]), ("bb", gb[0]), ("aa", ga[0]), ("xq", gxp[0]),
                        ("yq", gyp[0])]:
            vec = args[nm]
            fd = np.zeros_like(vec)
            for i in range(vec.size):
                vp, vm = vec.copy(), vec.copy(); vp[i] += h; vm[i] -= h
                fd[i] = (L(**{**args, nm: vp}) - L(**{**args, nm: vm})) / (2 * h)
            if vec.size:
                assert _rel(got, fd) < 1e-7, ("df1 fd", nm, M, N)


def pin_parameter_varying(lib=None):
    """Parameter-varying direct form (oracle.forward_tv / backward_tv): with constant
    coefficients it equals the fixed-coefficient direct form with past outputs
    (forward_df1, itself pinned to SciPy's lfiltic + lfilter), and its per-sample
    coefficient gradients sum to that form's; a first-order recursion
    y[n] = x[n] - a[n] y[n-1] has the closed form sum_k prod_{j=k+1..n} (-a[j]) x[k]
    + prod_{j=0..n} (-a[j]) y[-1]; every gradient equals FP64 central differences."""
    rng = np.random.default_rng(41)
    B, T, N, M = 2, 37, 2, 3
    x = rng.standard_normal((B, T)); yp = rng.standard_normal((B, M)); g = rng.standard_normal((B, T))
    a0 = 0.3 * rng.standard_normal((B, M)); b0 = rng.standard_normal((B, N + 1))
    at = np.repeat(a0[:, None, :], T, axis=1); bt = np.repeat(b0[:, None, :], T, axis=1)
    y = oracle.forward_tv(x, bt, at, yp, lib=lib)
    yr = oracle.forward_df1(x, b0, a0, np.zeros((B, N)), yp, lib=lib)
    assert _rel(y, yr) < 1e-13, "tv constant == df1"
    gx, gb, ga, gyp = oracle.backward_tv(g, x, y, bt, at, yp, lib=lib)
    rx, rb, ra, _, ryp = oracle.backward_df1(g, x, yr, b0, a0, np.zeros((B, N)), yp, lib=lib)
    assert _rel(gx, rx) < 1e-13 and _rel(gb.sum(1), rb) < 1e-12 and _rel(ga.sum(1), ra) < 1e-12, \
        "tv constant gradients == df1"
    assert _rel(gyp, ryp) < 1e-13, "tv constant grad_ypast == df1"
    # first order, varying coefficient
    T1 = 20
    x1 = rng.standard_normal((1, T1)); a1 = rng.uniform(-0.9, 0.9, (1, T1, 1)); y1p = np.array([[0.7]])
    y1 = oracle.forward_tv(x1, np.ones((1, T1, 1)), a1, y1p, lib=lib)[0]
    for n in range(T1):
        ref = sum(np.prod(-a1[0, k + 1:n + 1, 0]) * x1[0, k] for k in range(n + 1)) \
            + np.prod(-a1[0, :n + 1, 0]) * 0.7
        assert abs(y1[n] - ref) < 1e-12 * max(1.0, abs(ref)), "tv first-order closed form"
    # central differences on a small case
    Bs, Ts = 1, 9
    x = rng.standard_normal((Bs, Ts)); yp = rng.standard_normal((Bs, M)); g = rng.standard_normal((Bs, Ts))
    b = rng.standard_normal((Bs, Ts, N + 1)); a = 0.3 * rng.standard_normal((Bs, Ts, M))
    y = oracle.forward_tv(x, b, a, yp, lib=lib)
    gx, gb, ga, gyp = oracle.backward_tv(g, x, y, b, a, yp, lib=lib)
    L = lambda xx, bb, aa, pp: float((g * oracle.forward_tv(xx, bb, aa, pp, lib=lib)).sum())
    h = 1e-6
    args = {"x": x, "b": b, "a": a, "p": yp}
    for name, got in (("x", gx), ("b", gb), ("a", ga), ("p", gyp)):
        fd = np.zeros_like(args[name])
        for idx in np.ndindex(fd.shape):
            hp = {k: v.copy() for k, v in args.items()}; hm = {k: v.copy() for k, v in args.items()}
            hp[name][idx] += h; hm[name][idx] -= h
            fd[idx] = (L(hp["x"], hp["b"], hp["a"], hp["p"]) - L(hm["x"], hm["b"], hm["a"], hm["p"])) / (2 * h)
        assert _rel(got, fd) < 1e-7, ("tv fd", name)


def pin_recurrence_diagonalised(lib=None, ss=None):
    """The diagonalised App. B operator (Diag-EXT): with A's eigendecomposition from
    numpy's eig (a library routine) it equals the dense operator (itself pinned by
    closed forms and central differences above) for random real A with distinct
    eigenvalues, real and complex; a diagonal A gives geometric sums and a scaled
    rotation r R(theta) gives r^n R(n theta) v0 in closed form; its backward
    (grad_A, grad_v0, grad_z) equals FP64 central differences of <g, v>, grad_A taken
    through the eigendecomposition of the perturbed A.  (`ss` may replace the
    oracle module, for planted-mistake checks.)"""
    if ss is None:
        from oracle import statespace as ss
    rng = np.random.default_rng(31)
    eig = lambda A: (lambda w, V: (w, V, np.linalg.inv(V)))(*np.linalg.eig(A))
    for M, T in [(1, 30), (2, 40), (3, 25), (4, 33)]:
        A = 0.6 * rng.standard_normal((M, M)) / np.sqrt(M)
        v0 = rng.standard_normal(M); z = rng.standard_normal((T, M))
        lam, V, Vi = eig(A)
        assert _rel(ss.diag_forward(lam, V, Vi, v0, z), ss.recurrence_forward(A, v0, z)) < 1e-12, \
            ("diag == dense", M)
    lam = np.array([0.9, -0.6, 0.3])
    v0 = rng.standard_normal(3); z = rng.standard_normal((25, 3))
    v = ss.diag_forward(lam, np.eye(3), np.eye(3), v0, z)
    for i in range(3):
        ref = [lam[i] ** (n + 1) * v0[i] + sum(lam[i] ** (n - k) * z[k, i] for k in range(n + 1))
               for n in range(25)]
        assert _rel(v[:, i], ref) < 1e-13, "diag geometric"
    r, th = 0.97, 0.4
    Rm = r * np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    w0 = np.array([1.0, -0.5])
    lam, V, Vi = eig(Rm)
    v = ss.diag_forward(lam, V, Vi, w0, np.zeros((30, 2)))
    for n in range(30):
        c, s_ = np.cos((n + 1) * th), np.sin((n + 1) * th)
        assert _rel(v[n], r ** (n + 1) * np.array([[c, -s_], [s_, c]]) @ w0) < 1e-12, "diag rotation"
    for M, T in [(2, 30), (3, 17), (4, 12)]:
        A = 0.6 * rng.standard_normal((M, M)) / np.sqrt(M)
        v0 = rng.standard_normal(M); z = rng.standard_normal((T, M)); g = rng.standard_normal((T, M))
        lam, V, Vi = eig(A)
        v = ss.diag_forward(lam, V, Vi, v0, z)
        gA, gv0, gz = ss.diag_backward(lam, V, Vi, v0, v, g)
        L = lambda AA, vv, zz: float((g * ss.diag_forward(*eig(AA), vv, zz)).sum())
        h = 1e-6
        def fd(arr, which):
            out = np.zeros_like(arr)
            for idx in np.ndindex(arr.shape):
                ap, am = arr.copy(), arr.copy(); ap[idx] += h; am[idx] -= h
                kp = dict(AA=A, vv=v0, zz=z); km = dict(AA=A, vv=v0, zz=z)
                kp[which] = ap; km[which] = am
                out[idx] = (L(**kp) - L(**km)) / (2 * h)
            return out
        assert _rel(gA, fd(A, "AA")) < 1e-6, ("diag fd A", M)
        assert _rel(gv0, fd(v0, "vv")) < 1e-6, ("diag fd v0", M)
        assert _rel(gz, fd(z, "zz")) < 1e-6, ("diag fd z", M)


ALL_PINS = [pin_single_pole, pin_biquad_allpole, pin_transfer_function, pin_lfilter,
            pin_injection_form, pin_linearity_shift, pin_exact_forward,
            pin_exact_gradients, pin_finite_differences, pin_duality, pin_statespace,
            pin_jvp_single_pole, pin_jvp_finite_differences, pin_jvp_adjoint,
            pin_recurrence_dense, pin_df1_initial_conditions, pin_recurrence_diagonalised,
            pin_parameter_varying]


def run_all(lib=None):
    """Run every pin; returns the list of (name, error message) that failed."""
    failed = []
    for pin in ALL_PINS:
        try:
            pin(lib=lib)
        except Exception as e:  # noqa: BLE001 -- a planted mistake may raise anything
            failed.append((pin.__name__, repr(e)))
    return failed
