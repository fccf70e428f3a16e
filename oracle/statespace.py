"""State-space view of the filter (test infrastructure, FP64 numpy).

Two things from the paper, restated in my own code:

* the linear recurrence operator of App. B, ``v(n+1) = A v(n) + z(n)``, whose
  backward pass is the same operator run on (A^T, zero initial state,
  time-reversed upstream gradient), followed by dL/dv(0) = A^T dL/dz(0) and
  dL/dA = sum_n dL/dz(n) v(n)^T  (Eqs. dLdz and dLdvBA, App. A);
* the mapping of Sec. 2 from the direct form to the state-space form: A is the
  companion matrix of the denominator, C = [b_k - a_k b_0]_k, B = e_1, D = b_0;
  the transposed direct form uses A^T and swaps B and C.

The tests use these to cross-check the scalar oracle under that mapping.
"""
from __future__ import annotations

import numpy as np


def recurrence_forward(A, v0, z):
    """App. B operator.  A: (M, M), v0: (M,), z: (T, M) -> v(1..T): (T, M)."""
    A = np.asarray(A, dtype=np.float64)
    v = np.empty_like(np.asarray(z, dtype=np.float64))
    prev = np.asarray(v0, dtype=np.float64)
    for n in range(v.shape[0]):
        prev = A @ prev + z[n]
        v[n] = prev
    return v


def recurrence_backward(A, v0, v, grad_v):
    """Backward of the App. B operator given its output v(1..T) and dL/dv(1..T).

    dL/dz comes from running the same recurrence with A^T and a zero initial
    state on the time-reversed upstream gradient (Eq. dLdz run backwards in time);
    then dL/dv(0) = A^T dL/dz(0) and dL/dA = sum_n dL/dz(n) v(n)^T with
    v(n) = [v0, v(1), ..., v(T-1)] (Eq. dLdvBA).
    Returns (grad_A, grad_v0, grad_z).
    """
    A = np.asarray(A, dtype=np.float64)
    g = np.asarray(grad_v, dtype=np.float64)
    grad_z = recurrence_forward(A.T, np.zeros(A.shape[0]), g[::-1])[::-1]
    grad_v0 = A.T @ grad_z[0]
    prev_states = np.vstack([np.asarray(v0, dtype=np.float64)[None, :], v[:-1]])
    grad_A = grad_z.T @ prev_states
    return grad_A, grad_v0, grad_z


def diag_forward(lam, V, Vinv, v0, z):
    """The App. B operator with A diagonalised, A = V diag(lam) V^-1 (Diag-EXT, Sec. 3.2
    and Sec. 4): in the eigenbasis the state q = V^-1 v evolves element by element,
    q(n+1) = lam * q(n) + V^-1 z(n), q(0) = V^-1 v0, and v(n) = Re(V q(n)) (real for
    a real A whose complex eigenvectors come in conjugate pairs).
    lam: (M,) complex; V, Vinv: (M, M) complex; v0: (M,); z: (T, M) -> v(1..T): (T, M)."""
    lam = np.asarray(lam, dtype=np.complex128)
    V = np.asarray(V, dtype=np.complex128)
    Vinv = np.asarray(Vinv, dtype=np.complex128)
    z = np.asarray(z, dtype=np.float64)
    q = Vinv @ np.asarray(v0, dtype=np.float64)
    out = np.empty(z.shape)
    for n in range(z.shape[0]):
        q = lam * q + Vinv @ z[n]
        out[n] = (V @ q).real
    return out


def diag_backward(lam, V, Vinv, v0, v, grad_v):
    """Backward of the diagonalised operator: App. A's dL/dz is the operator for A^T run
    on the time-reversed upstream gradient from a zero state, and
    A^T = Vinv^T diag(lam) V^T is diagonalised by the transposed pair; then
    dL/dv(0) = A^T dL/dz(0) and dL/dA = sum_n dL/dz(n) v(n)^T with v(n) the state
    before step n.  Returns (grad_A, grad_v0, grad_z), all real."""
    lam = np.asarray(lam, dtype=np.complex128)
    V = np.asarray(V, dtype=np.complex128)
    Vinv = np.asarray(Vinv, dtype=np.complex128)
    g = np.asarray(grad_v, dtype=np.float64)
    M = lam.shape[0]
    grad_z = diag_forward(lam, Vinv.T, V.T, np.zeros(M), g[::-1])[::-1]
    grad_v0 = (Vinv.T @ (lam * (V.T @ grad_z[0]))).real
    before = np.vstack([np.asarray(v0, dtype=np.float64)[None, :], v[:-1]])   # v(0..T-1)
    grad_A = grad_z.T @ before
    return grad_A, grad_v0, grad_z


def companion(a):
    """Companion matrix of 1 + a_1 z^-1 + ... + a_M z^-M (Sec. 2): first row -a,
    ones on the subdiagonal."""
    a = np.asarray(a, dtype=np.float64)
    M = a.shape[0]
    A = np.zeros((M, M))
    A[0, :] = -a
    A[np.arange(1, M), np.arange(0, M - 1)] = 1.0
    return A


def df_to_ss(b, a):
    """Sec. 2 mapping for one channel: returns (A, B, C, D) of the direct form;
    b is zero-padded to order M first (Sec. 2 pads the shorter polynomial)."""
    a = np.asarray(a, dtype=np.float64)
    M = a.shape[0]
    bp = np.zeros(M + 1)
    bp[: len(b)] = np.asarray(b, dtype=np.float64)
    A = companion(a)
    Bv = np.zeros(M)
    Bv[0] = 1.0
    C = bp[1:] - a * bp[0]
    return A, Bv, C, bp[0]


def tdf_filter_and_grads(x, b, a, zi, gy):
    """One channel through the transposed form as a state-space system
    (A^T, input vector C, output vector B = e_1, D = b_0) driven by the App. B
    operator, with all gradients obtained from that operator's backward and the
    chain rule through the Sec. 2 mapping.

    Returns (y, grad_x, grad_b, grad_a, grad_zi) in FP64; grad_b has length N+1.
    """
    x = np.asarray(x, dtype=np.float64)
    gy = np.asarray(gy, dtype=np.float64)
    N = len(b) - 1
    A, e1, C, D = df_to_ss(b, a)
    At = A.T
    M = A.shape[0]
    T = x.shape[0]
    v0 = np.zeros(M) if zi is None else np.asarray(zi, dtype=np.float64)
    z = x[:, None] * C[None, :]                      # z(n) = C x(n)
    v = recurrence_forward(At, v0, z)                # v(1..T)
    states = np.vstack([v0[None, :], v[:-1]])        # v(0..T-1)
    y = states @ e1 + D * x                          # y(n) = e1^T v(n) + D x(n)

    # dL/dv(n) = gy(n) e1 for the states the output reads; v(T) is not read.
    grad_v = np.zeros((T, M))
    grad_v[:-1] = gy[1:, None] * e1[None, :]
    grad_At, grad_v0, grad_z = recurrence_backward(At, v0, v, grad_v)
    grad_v0 = grad_v0 + gy[0] * e1                   # y(0) reads v(0) directly
    grad_x = grad_z @ C + D * gy
    grad_C = grad_z.T @ x                            # z(n) = C x(n)
    grad_D = float(gy @ x)
    # A^T[k, 0] = -a_{k+1};  C_k = b_{k+1} - a_{k+1} b_0;  D = b_0
    grad_a = -grad_At[:, 0] - D * grad_C
    grad_bfull = np.zeros(M + 1)
    grad_bfull[1:] = grad_C
    grad_bfull[0] = grad_D - float(np.asarray(a, dtype=np.float64) @ grad_C)
    return y, grad_x, grad_bfull[: N + 1], grad_a, grad_v0
