"""The diagonalised App. B recurrence (the paper's Diag-EXT: A = V diag(lam) V^-1, the
scan run element by element in the eigenbasis; dfilt_diag_forward / dfilt_diag_backward)
through the C ABI against the FP64 oracle's diagonalised operator and its backward
(App. A), element by element: every supported M, real and complex eigenvalues, lengths
around the 32-step chunks and 1024-step segments, more than 32 segments, with and
without an initial state, spectral radius up to 0.999, the paper's M = 2 operator at
T = 2^16; and against the dense operator's GPU path on the same A.

The oracle runs on the same rounded eigendecomposition (complex64 promoted to FP64), so
the comparison measures the kernels' arithmetic.  Tolerance per channel:
max(1e-5, 32 u32 cond(V) / (1 - rho)): a step's rounding reaches later outputs through
the decaying powers of lam (sum_k rho^k = 1 / (1 - rho)) and the two projections
(cond(V))."""
import numpy as np
import pytest
import torch

from oracle import statespace as ss
from paper_2511_14390_gb300 import dfilt

from tol import U32, log_errors

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def draw(rng, B, T, M, rho):
    """Seeded real A per channel scaled to spectral radius rho, its eigendecomposition
    (numpy's eig; conjugate pairs for complex eigenvalues), v0, z, upstream gradient."""
    A = rng.standard_normal((B, M, M))
    lam = np.zeros((B, M), np.complex64)
    V = np.zeros((B, M, M), np.complex64)
    Vi = np.zeros((B, M, M), np.complex64)
    for i in range(B):
        A[i] *= rho / max(abs(np.linalg.eigvals(A[i])))
        w, vec = np.linalg.eig(A[i])
        lam[i], V[i], Vi[i] = w, vec, np.linalg.inv(vec)
    f = lambda *s: rng.standard_normal(s).astype(np.float32)
    return A.astype(np.float32), lam, V, Vi, f(B, M), f(B, T, M), f(B, T, M)


def dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def run_and_check(name, A, lam, V, Vi, v0, z, gv):
    B, T, M = z.shape
    ld, Vd, Vid, v0d, zd, gvd = dev(lam), dev(V), dev(Vi), dev(v0), dev(z), dev(gv)
    v = dfilt.dfilt_diag_forward(ld, Vd, Vid, v0d, zd)
    gA, gv0, gz = dfilt.dfilt_diag_backward(ld, Vd, Vid, v0d, v, gvd)
    st = dfilt.dfilt_sync_status()
    assert st == 0, dfilt.STATUS[st]
    v, gA, gv0, gz = (t.cpu().numpy().astype(np.float64) for t in (v, gA, gv0, gz))
    errs = {k: np.zeros(B) for k in ("v", "gz", "gA", "gv0")}
    tol = np.zeros(B)
    for i in range(B):
        l64, V64, Vi64 = (t.astype(np.complex128) for t in (lam[i], V[i], Vi[i]))
        v0i = np.zeros(M) if v0 is None else v0[i].astype(np.float64)
        vr = ss.diag_forward(l64, V64, Vi64, v0i, z[i])
        gAr, gv0r, gzr = ss.diag_backward(l64, V64, Vi64, v0i, vr, gv[i])
        prev = np.vstack([v0i[None], vr[:-1]])
        scale = np.abs(gzr).T @ np.abs(prev)          # natural scale of each dL/dA entry
        errs["v"][i] = np.abs(v[i] - vr).max() / np.abs(vr).max()
        errs["gz"][i] = np.abs(gz[i] - gzr).max() / np.abs(gzr).max()
        errs["gA"][i] = (np.abs(gA[i] - gAr) / scale).max()
        errs["gv0"][i] = np.abs(gv0[i] - gv0r).max() / max(np.abs(gzr).max() * np.abs(A[i]).sum(), 1e-30)
        rho = np.abs(l64).max()
        tol[i] = max(1e-5, 32 * U32 * np.linalg.cond(V64) / (1 - rho))
    log_errors(f"diag_{name}", **errs)
    for k, e in errs.items():
        assert (e < tol).all(), (name, k, e, tol)
    return v, gz


@pytest.mark.parametrize("M", [1, 2, 3, 4])
@pytest.mark.parametrize("T", [1, 31, 33, 1024, 1025, 5000])
def test_diag_shapes(M, T):
    rng = np.random.default_rng(2000 * M + T)
    A, lam, V, Vi, v0, z, gv = draw(rng, 3, T, M, 0.95)
    run_and_check(f"M{M}_T{T}", A, lam, V, Vi, v0, z, gv)


def test_diag_many_segments_no_initial_state():
    """40000 steps = 40 segments; v0 = NULL."""
    rng = np.random.default_rng(17)
    A, lam, V, Vi, _, z, gv = draw(rng, 4, 40000, 2, 0.99)
    run_and_check("many_segments", A, lam, V, Vi, None, z, gv)


def test_diag_near_unit_radius():
    rng = np.random.default_rng(18)
    A, lam, V, Vi, v0, z, gv = draw(rng, 4, 20000, 2, 0.999)
    run_and_check("radius_0999", A, lam, V, Vi, v0, z, gv)


def test_diag_paper_operator_long():
    """The paper's benchmarked operator size class: M = 2, 2^16 steps, two channels."""
    rng = np.random.default_rng(19)
    A, lam, V, Vi, v0, z, gv = draw(rng, 2, 1 << 16, 2, 0.95)
    run_and_check("M2_T2^16", A, lam, V, Vi, v0, z, gv)


@pytest.mark.parametrize("M", [2, 4])
def test_diag_matches_dense_operator(M):
    """Diag-EXT and EXT compute the same function of A: the diagonalised path on A's
    eigendecomposition and the dense path on A agree to the FP32 rounding of either."""
    rng = np.random.default_rng(30 + M)
    A, lam, V, Vi, v0, z, gv = draw(rng, 3, 9000, M, 0.9)
    v_d, gz_d = run_and_check(f"vs_dense_M{M}", A, lam, V, Vi, v0, z, gv)
    Ad, v0d, zd, gvd = dev(A), dev(v0), dev(z), dev(gv)
    v_s = dfilt.dfilt_ss_forward(Ad, v0d, zd)
    gA_s, gv0_s, gz_s = dfilt.dfilt_ss_backward(Ad, v0d, v_s, gvd)
    v_s, gz_s = v_s.cpu().numpy(), gz_s.cpu().numpy()
    for i in range(3):
        c = np.linalg.cond(V[i].astype(np.complex128))
        assert np.abs(v_s[i] - v_d[i]).max() / np.abs(v_s[i]).max() < max(1e-5, 64 * U32 * c * 10)
        assert np.abs(gz_s[i] - gz_d[i]).max() / np.abs(gz_s[i]).max() < max(1e-5, 64 * U32 * c * 10)


def test_diag_empty_and_selected_gradients():
    e = torch.empty(0, 5, 2, device=DEV)
    c0 = torch.empty(0, 2, dtype=torch.complex64, device=DEV)
    c00 = torch.empty(0, 2, 2, dtype=torch.complex64, device=DEV)
    assert dfilt.dfilt_diag_forward(c0, c00, c00, None, e).shape == (0, 5, 2)
    rng = np.random.default_rng(20)
    A, lam, V, Vi, v0, z, gv = draw(rng, 2, 3000, 3, 0.9)
    ld, Vd, Vid, v0d, zd, gvd = dev(lam), dev(V), dev(Vi), dev(v0), dev(z), dev(gv)
    v = dfilt.dfilt_diag_forward(ld, Vd, Vid, v0d, zd)
    full = dfilt.dfilt_diag_backward(ld, Vd, Vid, v0d, v, gvd)
    part = dfilt.dfilt_diag_backward(ld, Vd, Vid, v0d, None, gvd, needs=(False, True))
    assert part[0] is None and torch.equal(part[1], full[1]) and torch.equal(part[2], full[2])
    assert dfilt.dfilt_sync_status() == 0
