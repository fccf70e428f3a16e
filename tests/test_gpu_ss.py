"""The App. B recurrence v(n+1) = A v(n) + z(n) with a dense A per channel
(dfilt_ss_forward / dfilt_ss_backward) through the C ABI against the FP64 oracle's
operator and its backward (App. A), element by element: every supported M, lengths
around the 32-step chunks and 1024-step segments, more than 32 segments per channel,
with and without an initial state, near-unit spectral radius, and the paper's M = 2
operator at T = 2^20 on one channel."""
import numpy as np
import pytest
import torch

from oracle import statespace as ss
from paper_2511_14390_gb300 import dfilt

from tol import U32, log_errors

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


def draw(rng, B, T, M, rho):
    """Seeded dense A per channel scaled to spectral radius rho, v0, z, upstream grad."""
    A = rng.standard_normal((B, M, M))
    for i in range(B):
        A[i] *= rho / max(abs(np.linalg.eigvals(A[i])))
    f = lambda *s: rng.standard_normal(s).astype(np.float32)
    return A.astype(np.float32), f(B, M), f(B, T, M), f(B, T, M)


def kappa(A, T):
    """sum_k ||A^k||_2 over k < min(T, 4096): how far one step's rounding can travel."""
    out = []
    for a in np.asarray(A, dtype=np.float64):
        P, s = np.eye(a.shape[0]), 0.0
        for _ in range(min(T, 4096)):
            s += np.linalg.norm(P, 2)
            P = P @ a
        out.append(s)
    return np.array(out)


def run_and_check(name, A, v0, z, gv, tol_scale=32):
    B, T, M = z.shape
    Ad, v0d, zd, gvd = dev(A), dev(v0), dev(z), dev(gv)
    v = dfilt.dfilt_ss_forward(Ad, v0d, zd)
    gA, gv0, gz = dfilt.dfilt_ss_backward(Ad, v0d, v, gvd)
    st = dfilt.dfilt_sync_status()
    assert st == 0, dfilt.STATUS[st]
    v, gA, gv0, gz = (t.cpu().numpy().astype(np.float64) for t in (v, gA, gv0, gz))
    tol = np.maximum(1e-5, tol_scale * U32 * kappa(A, T))
    errs = {k: np.zeros(B) for k in ("v", "gz", "gA", "gv0")}
    for i in range(B):
        v0i = None if v0 is None else v0[i]
        vr = ss.recurrence_forward(A[i], np.zeros(M) if v0i is None else v0i, z[i])
        gAr, gv0r, gzr = ss.recurrence_backward(A[i], np.zeros(M) if v0i is None else v0i, vr, gv[i])
        prev = np.vstack([(np.zeros(M) if v0i is None else v0i)[None], vr[:-1]])
        scale = np.abs(gzr).T @ np.abs(prev)          # natural scale of each dL/dA entry
        errs["v"][i] = np.abs(v[i] - vr).max() / np.abs(vr).max()
        errs["gz"][i] = np.abs(gz[i] - gzr).max() / np.abs(gzr).max()
        errs["gA"][i] = (np.abs(gA[i] - gAr) / scale).max()
        errs["gv0"][i] = np.abs(gv0[i] - gv0r).max() / max(np.abs(gzr).max() * np.abs(A[i]).sum(), 1e-30)
    log_errors(f"ss_{name}", **errs)
    for k, e in errs.items():
        assert (e < tol).all(), (name, k, e, tol)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
@pytest.mark.parametrize("T", [1, 31, 33, 1024, 1025, 5000])
def test_ss_shapes(M, T):
    rng = np.random.default_rng(1000 * M + T)
    A, v0, z, gv = draw(rng, 3, T, M, 0.95)
    run_and_check(f"M{M}_T{T}", A, v0, z, gv)


def test_ss_many_segments_no_initial_state():
    """40000 steps = 40 segments (two rounds of the carry scan); v0 = NULL."""
    rng = np.random.default_rng(7)
    A, _, z, gv = draw(rng, 4, 40000, 2, 0.99)
    run_and_check("many_segments", A, None, z, gv)


def test_ss_near_unit_radius():
    rng = np.random.default_rng(8)
    A, v0, z, gv = draw(rng, 4, 20000, 2, 0.999)
    run_and_check("radius_0999", A, v0, z, gv)


def test_ss_paper_operator_long():
    """The paper's benchmarked operator: M = 2, one sequence of 2^20 steps."""
    rng = np.random.default_rng(9)
    A, v0, z, gv = draw(rng, 1, 1 << 20, 2, 0.95)
    run_and_check("M2_T2^20", A, v0, z, gv)


def test_ss_empty_and_selected_gradients():
    e = torch.empty(0, 5, 2, device=DEV)
    A = torch.eye(2, device=DEV)[None].repeat(0, 1, 1)
    assert dfilt.dfilt_ss_forward(A, None, e).shape == (0, 5, 2)
    rng = np.random.default_rng(10)
    A, v0, z, gv = draw(rng, 2, 3000, 3, 0.9)
    Ad, v0d, zd, gvd = dev(A), dev(v0), dev(z), dev(gv)
    v = dfilt.dfilt_ss_forward(Ad, v0d, zd)
    full = dfilt.dfilt_ss_backward(Ad, v0d, v, gvd)
    part = dfilt.dfilt_ss_backward(Ad, v0d, None, gvd, needs=(False, True))
    assert part[0] is None and torch.equal(part[1], full[1]) and torch.equal(part[2], full[2])
    assert dfilt.dfilt_sync_status() == 0
