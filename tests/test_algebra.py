"""CPU checks of the algebra the CUDA paths of the extension rows are built on, each
against the FP64 oracle (no GPU, no CUDA code): the forward-mode derivative as an
input step followed by the all-pole filter; the state-space recurrence as 32-step
chunks combined by a shuffle-style scan with powers of A, then 1024-step segments
combined the same way, in either time direction; the direct-form initial conditions
as a TDF-II state."""
import numpy as np
import pytest
import scipy.signal as ss

import oracle
from oracle import statespace

from pins import _random_filter


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("M,N,T", [(2, 2, 300), (5, 3, 97), (1, 0, 40), (8, 8, 5)])
def test_jvp_is_input_step_then_all_pole_filter(M, N, T):
    """dy = 1/A applied to v = B dx + dB x - dA y, state dzi (the forward mode as the
    library computes it) equals the oracle's step-by-step derivative."""
    rng = np.random.default_rng(40 + M)
    b, a = _random_filter(rng, M, N, rmax=0.9)
    x = rng.standard_normal(T); zi = rng.standard_normal(M)
    dx = rng.standard_normal(T); db = rng.standard_normal(N + 1)
    da = rng.standard_normal(M); dz = rng.standard_normal(M)
    y, dy = oracle.jvp(x[None], b[None], a[None], zi[None], dx[None], db[None], da[None],
                       dz[None])
    v = (np.convolve(b, dx)[:T] + np.convolve(db, x)[:T]
         - np.convolve(np.concatenate([[0.0], da]), y[0])[:T])
    two_step = oracle.forward(v[None], np.ones((1, 1)), a[None], dz[None])[0]
    assert _rel(two_step, dy[0]) < 1e-12


def _chunk_scan(A, v0, z, chunk):
    """Zero-state chunks of `chunk` steps, then a Hillis-Steele scan over the chunks'
    end states with A^(chunk * 2^k) and the entry state injected into chunk 0, then
    every chunk rerun from its entry state (the structure of one segment pass)."""
    T, M = z.shape
    C = (T + chunk - 1) // chunk
    e = np.zeros((C, M))
    for c in range(C):
        s = np.zeros(M)
        for n in range(c * chunk, min(T, (c + 1) * chunk)):
            s = A @ s + z[n]
        e[c] = s
    e[0] += np.linalg.matrix_power(A, chunk) @ v0
    d = 1
    while d < C:
        P = np.linalg.matrix_power(A, chunk * d)
        e = np.vstack([e[:d], e[d:] + (P @ e[:-d].T).T])
        d *= 2
    out = np.zeros((T, M))
    for c in range(C):
        s = v0 if c == 0 else e[c - 1]
        for n in range(c * chunk, min(T, (c + 1) * chunk)):
            s = A @ s + z[n]
            out[n] = s
    return out


@pytest.mark.parametrize("M,T", [(2, 1), (2, 1000), (3, 1025), (4, 3000)])
def test_state_space_chunk_scan(M, T):
    """The chunked scan (32-step chunks inside 1024-step segments) reproduces the App. B
    operator, and run on A^T in reversed time from a zero state its dL/dz."""
    rng = np.random.default_rng(50 + T)
    A = rng.standard_normal((M, M))
    A *= 0.95 / max(abs(np.linalg.eigvals(A)))
    v0 = rng.standard_normal(M); z = rng.standard_normal((T, M)); g = rng.standard_normal((T, M))
    ref = statespace.recurrence_forward(A, v0, z)
    seg = 1024
    out, s = np.zeros_like(ref), v0
    for g0 in range(0, T, seg):                  # segments in order, each from its entry state
        out[g0: g0 + seg] = _chunk_scan(A, s, z[g0: g0 + seg], 32)
        s = out[min(T, g0 + seg) - 1]
    assert _rel(out, ref) < 1e-12
    gz_ref = statespace.recurrence_backward(A, v0, ref, g)[2]
    gz = _chunk_scan(A.T, np.zeros(M), g[::-1], 32)[::-1]
    assert _rel(gz, gz_ref) < 1e-12


@pytest.mark.parametrize("M,N", [(2, 2), (6, 4), (3, 0)])
def test_direct_form_state_formula(M, N):
    """zi[m] = sum_{k>m} b_k x[m-k] - sum_{k>m} a_k y[m-k] equals SciPy's lfiltic, and
    filtering from it equals the oracle's difference equation with the past values."""
    rng = np.random.default_rng(60 + M)
    b, a = _random_filter(rng, M, N)
    xp = rng.standard_normal(N); yp = rng.standard_normal(M); x = rng.standard_normal(50)
    zi = np.array([sum(b[k] * xp[k - m - 1] for k in range(m + 1, N + 1))
                   - sum(a[k - 1] * yp[k - m - 1] for k in range(m + 1, M + 1))
                   for m in range(M)])
    af = np.concatenate([[1.0], a])
    assert _rel(zi, ss.lfiltic(b, af, yp, xp if N else None)) < 1e-13
    y = oracle.forward(x[None], b[None], a[None], zi[None])[0]
    assert _rel(y, oracle.forward_df1(x[None], b[None], a[None], xp[None], yp[None])[0]) < 1e-12
