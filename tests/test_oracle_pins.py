"""The FP64 oracle against its pins (closed forms, transfer function, SciPy,
exact-rational brute force, finite differences, duality, the App. B operator),
plus mutation checks: a mistake planted in a copy of the oracle must fail a pin."""
import os

import numpy as np
import pytest

import oracle
from oracle import chunked, pyref
from paper_2511_14390_gb300 import inputs

import pins


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda p: p.__name__)
def test_pin(pin, oracle_lib):
    pin()


# Each entry: (description, original snippet, planted mistake).
MUTATIONS = [
    ("forward feedback sign", "- a[k] * yn;", "+ a[k] * yn;"),
    ("forward numerator index", "bcoef(b, N, k + 1) * xn", "bcoef(b, N, k) * xn"),
    ("forward drops state", "const double yn = b[0] * xn + s[0];", "const double yn = b[0] * xn;"),
    ("numerator padding drops b_N", "return k <= N ? b[k] : 0.0;", "return k < N ? b[k] : 0.0;"),
    ("injection drops last zi", "if (zi && n < M) w += zi[n];", "if (zi && n + 1 < M) w += zi[n];"),
    ("adjoint feedback sign", "acc -= a[k - 1] * u[n + k];", "acc += a[k - 1] * u[n + k];"),
    ("grad_x lag ignored", "acc += b[k] * u[n + k];", "acc += b[k] * u[n];"),
    ("grad_b dropped term", "for (int64_t n = k; n < T; ++n) acc += u[n] * x[n - k];",
     "for (int64_t n = k + 1; n < T; ++n) acc += u[n] * x[n - k];"),
    ("grad_b sign", "gb[k] = acc;", "gb[k] = -acc;"),
    ("grad_a sign", "ga[k - 1] = -acc;", "ga[k - 1] = acc;"),
    ("grad_a correlates x", "acc += u[n] * y[n - k];", "acc += u[n] * x[n - k];"),
    ("grad_zi index", "gzi[k] = (k < T) ? u[k] : 0.0;", "gzi[k] = (k + 1 < T) ? u[k + 1] : 0.0;"),
    ("jvp feedback on the primal", "- a[k] * dyn;", "- a[k] * yn;"),
    ("jvp denominator tangent sign", "if (da) d -= da[k] * yn;", "if (da) d += da[k] * yn;"),
    ("jvp numerator tangent index", "if (db) d += bcoef(db, N, k + 1) * xn;",
     "if (db) d += bcoef(db, N, k) * xn;"),
    ("jvp drops the state tangent", "ds[k] = dzi ? dzi[k] : 0.0;", "ds[k] = 0.0;"),
    ("jvp drops db_0", "if (db) dyn += db[0] * xn;", "if (db) dyn += 0.0 * xn;"),
    ("df1 forward drops past outputs",
     "acc -= a[k - 1] * (n - k >= 0 ? y[n - k] : yp[k - n - 1]);",
     "acc -= a[k - 1] * (n - k >= 0 ? y[n - k] : 0.0);"),
    ("df1 grad_a drops past outputs",
     "sum += u[n] * (n - k >= 0 ? y[n - k] : yp[k - n - 1]);",
     "sum += u[n] * (n - k >= 0 ? y[n - k] : 0.0);"),
    ("df1 grad_xpast coefficient index", "if (k - j < T) sum += b[k] * u[k - j];",
     "if (k - j < T) sum += b[k - 1] * u[k - j];"),
    ("df1 grad_ypast sign", "gyp[j - 1] = -sum;", "gyp[j - 1] = sum;"),
    ("tv adjoint takes the coefficient at n", "acc -= a[(n + k) * M + k - 1] * u[n + k];",
     "acc -= a[n * M + k - 1] * u[n + k];"),
    ("tv grad_x takes b at n", "acc += b[(n + k) * (N + 1) + k] * u[n + k];",
     "acc += b[n * (N + 1) + k] * u[n + k];"),
    ("tv grad_a sign", "ga[n * M + k - 1] = -u[n] * yk;", "ga[n * M + k - 1] = u[n] * yk;"),
    ("tv forward past-output index", "acc -= a[n * M + k - 1] * yk;", "acc -= a[n * M + k - 1] * (n - k >= 0 ? yk : 0.0);"),
    ("tv grad_ypast coefficient time", "acc += a[(k - 1 - j) * M + k - 1] * u[k - 1 - j];",
     "acc += a[k - 1] * u[k - 1 - j];"),
]


@pytest.mark.parametrize("desc,orig,mut", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(desc, orig, mut, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "dfilt_oracle.c")).read()
    assert src.count(orig) == 1, f"mutation site not unique: {orig}"
    so = oracle.compile_variant(src.replace(orig, mut), str(tmp_path / "mutant.so"))
    failed = pins.run_all(lib=oracle.load(so))
    assert failed, f"no pin caught the planted mistake: {desc}"


def test_pure_python_matches_c():
    rng = np.random.default_rng(5)
    for M, N, T in [(1, 0, 17), (3, 2, 40), (5, 5, 9)]:
        b = rng.standard_normal(N + 1); a = 0.1 * rng.standard_normal(M)
        x = rng.standard_normal(T); zi = rng.standard_normal(M); g = rng.standard_normal(T)
        y = np.array(pyref.forward(list(x), list(b), list(a), list(zi)))
        yc = oracle.forward(x[None], b[None], a[None], zi[None])[0]
        assert np.allclose(y, yc, rtol=1e-13, atol=1e-13)
        got = pyref.backward(list(g), list(x), list(y), list(b), list(a))
        ref = oracle.backward(g[None], x[None], y[None], b[None], a[None])
        for gp, gc in zip(got, ref):
            assert np.allclose(np.array(gp), gc[0], rtol=1e-12, atol=1e-12)


def test_ragged_equals_per_channel():
    w = inputs.make_ragged(B=12, T_range=(1, 300), M_range=(1, 6), seed=3)
    y = oracle.forward_ragged(w.x, w.offsets, w.Ms, w.Ns, w.b, w.a, w.zi)
    gx, gb, ga, gz = oracle.backward_ragged(w.gy, w.x, y, w.offsets, w.Ms, w.Ns, w.b, w.a)
    for i in range(w.B):
        s, e = w.offsets[i], w.offsets[i + 1]
        M, N = int(w.Ms[i]), int(w.Ns[i])
        bi, ai, zi = w.b[i, : N + 1][None], w.a[i, :M][None], w.zi[i, :M][None]
        yi = oracle.forward(w.x[s:e][None], bi, ai, zi)
        assert np.array_equal(yi[0], y[s:e])
        r = oracle.backward(w.gy[s:e][None], w.x[s:e][None], yi, bi, ai)
        assert np.array_equal(r[0][0], gx[s:e])
        assert np.array_equal(r[1][0], gb[i, : N + 1]) and not gb[i, N + 1:].any()
        assert np.array_equal(r[2][0], ga[i, :M]) and not ga[i, M:].any()
        assert np.array_equal(r[3][0], gz[i, :M])


def test_edge_cases():
    # T = 1, T < M: grad_zi beyond T is zero; zero-length channel in a ragged batch
    b = np.array([[0.5, 0.25, 0.125]]); a = np.array([[0.1, -0.2, 0.05]])
    x = np.array([[2.0]]); zi = np.array([[1.0, 2.0, 3.0]]); g = np.array([[3.0]])
    y = oracle.forward(x, b, a, zi)
    assert y[0, 0] == 0.5 * 2.0 + 1.0
    gx, gb, ga, gz = oracle.backward(g, x, y, b, a)
    assert gx[0, 0] == 0.5 * 3.0 and np.array_equal(gz[0], [3.0, 0.0, 0.0])
    assert np.array_equal(gb[0], [6.0, 0.0, 0.0]) and not ga.any()
    offs = np.array([0, 0, 3], dtype=np.int64)
    Ms = np.array([1, 1], dtype=np.int32); Ns = np.array([0, 0], dtype=np.int32)
    yr = oracle.forward_ragged(np.ones(3), offs, Ms, Ns, np.ones((2, 1)), np.full((2, 1), -0.5))
    assert np.array_equal(yr, [1.0, 1.5, 1.75])


@pytest.mark.parametrize("L", [4, 16, 64])
def test_chunk_algebra_model(L):
    """The FP64 chunked model (Sec. 3.2 operator at chunk granularity) equals the
    sequential oracle, forward and backward, with a ragged tail and zi."""
    rng = np.random.default_rng(L)
    for M, N, T in [(1, 1, 5 * L + 3), (2, 2, 3 * L), (4, 3, 2 * L + 1), (3, 0, L - 1)]:
        if M > L:
            continue
        b, a = pins._random_filter(rng, M, N, rmax=0.9)
        x = rng.standard_normal(T); zi = rng.standard_normal(M); g = rng.standard_normal(T)
        y = oracle.forward(x[None], b[None], a[None], zi[None])[0]
        assert pins._rel(chunked.forward(x, b, a, zi, L), y) < 1e-12
        ref = oracle.backward(g[None], x[None], y[None], b[None], a[None])
        got = chunked.backward(g, x, y, b, a, L)
        for gc, gr in zip(got, ref):
            assert pins._rel(gc, gr[0]) < 1e-11


def test_oracle_threads_deterministic():
    w = inputs.make("biquad_1024x48000", B=16, T=3000)
    y1 = oracle.forward(w.x, w.b, w.a, w.zi, nthreads=1)
    y4 = oracle.forward(w.x, w.b, w.a, w.zi, nthreads=4)
    assert np.array_equal(y1, y4)


# Planted mistakes in the diagonalised state-space operator (oracle/statespace.py):
# each must fail pin_recurrence_diagonalised.
DIAG_MUTATIONS = [
    ("diag input projection", "q = lam * q + Vinv @ z[n]", "q = lam * q + V @ z[n]"),
    ("diag output takes the imaginary part", "out[n] = (V @ q).real", "out[n] = (V @ q).imag"),
    ("diag initial state not projected", "q = Vinv @ np.asarray(v0, dtype=np.float64)",
     "q = np.asarray(v0, dtype=np.complex128)"),
    ("diag adjoint basis not transposed", "diag_forward(lam, Vinv.T, V.T, np.zeros(M), g[::-1])",
     "diag_forward(lam, V, Vinv, np.zeros(M), g[::-1])"),
    ("diag grad_v0 drops lam", "grad_v0 = (Vinv.T @ (lam * (V.T @ grad_z[0]))).real",
     "grad_v0 = (Vinv.T @ (V.T @ grad_z[0])).real"),
    ("diag grad_A pairs v(n+1)", "before = np.vstack([np.asarray(v0, dtype=np.float64)[None, :], v[:-1]])",
     "before = v"),
]


@pytest.mark.parametrize("desc,orig,mut", DIAG_MUTATIONS, ids=[m[0] for m in DIAG_MUTATIONS])
def test_planted_mistake_in_diag_operator_is_caught(desc, orig, mut):
    import types
    from oracle import statespace
    src = open(statespace.__file__).read()
    assert src.count(orig) == 1, f"mutation site not unique: {orig}"
    mod = types.ModuleType("statespace_mutant")
    exec(compile(src.replace(orig, mut), "statespace_mutant.py", "exec"), mod.__dict__)
    with pytest.raises(AssertionError):
        pins.pin_recurrence_diagonalised(ss=mod)
