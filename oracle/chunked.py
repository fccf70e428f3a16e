"""FP64 model of the chunk algebra (test infrastructure, numpy).

The paper parallelises the state recursion with the associative operator
(A, z) (+) (A', z') = (A'A, A'z + z') of Sec. 3.2.  Applied at chunk
granularity (chunk length L, C = ceil(T/L) chunks, zero-padded tail) the
transposed-direct-form recursion of Sec. 2 becomes, per chunk c,

    Y_c     = T_g X_c + O_L S_c          (zero-state Toeplitz part + free response)
    S_{c+1} = Abar S_c + R_L X_c,  S_0 = zi,   Abar = F^L

where F is the TDF state transition (companion matrix transposed), g the
impulse response of B/A, T_g its lower-triangular L x L Toeplitz matrix,
O_L[i] = e_1^T F^i and R_L[:, j] = F^(L-1-j) Gv (Gv = C of Sec. 2).

The backward (Sec. 3.1, the same recursion reversed in time) is modelled with
the direct-form state of the adjoint: entering chunk c from the right the state
is the next M adjoint values u[(c+1)L .. (c+1)L+M-1] (zero past the end, App. A):

    U_c   = T_h^a G_c + O^u S'_c,   GX_c = T_g^a G_c + O^gx S'_c,   S'_{c-1} = U_c[0:M]

with T^a the upper-triangular (anti-causal) Toeplitz matrices of h = 1/A and g.
This module exists to pin that algebra against the sequential oracle; it is not
what parity is measured against.
"""
from __future__ import annotations

import numpy as np

from .statespace import df_to_ss


def _tdf(b, a):
    A, e1, C, D = df_to_ss(b, a)
    return A.T, C, e1, D     # F, Gv, output vector, D


def impulse(b, a, L):
    """First L samples of the impulse response of B/A (b zero-padded to order M)."""
    F, Gv, e1, D = _tdf(b, a)
    g = np.zeros(L)
    g[0] = D
    s = Gv.copy()
    for n in range(1, L):
        g[n] = s[0]
        s = F @ s
    return g


def forward_tables(b, a, L):
    F, Gv, e1, D = _tdf(b, a)
    M = F.shape[0]
    g = impulse(b, a, L)
    Tg = np.zeros((L, L))
    for i in range(L):
        Tg[i, : i + 1] = g[i::-1]
    OL = np.zeros((L, M))
    r = e1.copy()
    for i in range(L):
        OL[i] = r
        r = r @ F
    RL = np.zeros((M, L))
    v = Gv.copy()
    for j in range(L - 1, -1, -1):
        RL[:, j] = v
        v = F @ v
    Abar = np.linalg.matrix_power(F, L)
    return Tg, OL, RL, Abar


def forward(x, b, a, zi, L):
    """Chunked forward for one channel, FP64."""
    x = np.asarray(x, dtype=np.float64)
    T = x.shape[0]
    M = len(a)
    C = -(-T // L)
    X = np.zeros(C * L)
    X[:T] = x
    X = X.reshape(C, L)
    Tg, OL, RL, Abar = forward_tables(b, a, L)
    S = np.zeros(M) if zi is None else np.asarray(zi, dtype=np.float64).copy()
    Y = np.empty((C, L))
    for c in range(C):
        Y[c] = Tg @ X[c] + OL @ S
        S = Abar @ S + RL @ X[c]
    return Y.reshape(-1)[:T]


def backward_tables(b, a, L):
    M = len(a)
    a = np.asarray(a, dtype=np.float64)
    N = len(b) - 1
    bp = np.zeros(M + 1)
    bp[: N + 1] = np.asarray(b, dtype=np.float64)
    g = impulse(b, a, L)
    h = impulse([1.0], a, L)
    Tga = np.zeros((L, L))
    Tha = np.zeros((L, L))
    for i in range(L):
        Tga[i, i:] = g[: L - i]
        Tha[i, i:] = h[: L - i]
    # free response of the anti-causal all-pole recursion from u[L..L+M-1]
    Ou = np.zeros((L, M))
    for m in range(M):
        u = np.zeros(L + M)
        u[L + m] = 1.0
        for n in range(L - 1, -1, -1):
            u[n] = -a @ u[n + 1: n + 1 + M]
        Ou[:, m] = u[:L]
    Ogx = np.zeros((L, M))
    for m in range(M):
        ext = np.zeros(L + M)
        ext[:L] = Ou[:, m]
        ext[L + m] = 1.0
        for i in range(L):
            Ogx[i, m] = bp @ ext[i: i + M + 1]
    return Tga, Tha, Ou, Ogx


def backward(gy, x, y, b, a, L):
    """Chunked backward for one channel, FP64: (grad_x, grad_b, grad_a, grad_zi)."""
    gy = np.asarray(gy, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    T = gy.shape[0]
    M, N = len(a), len(b) - 1
    C = -(-T // L)
    pad = lambda s: np.concatenate([s, np.zeros(C * L - T)]).reshape(C, L)
    G, X, Y = pad(gy), pad(x), pad(y)
    Tga, Tha, Ou, Ogx = backward_tables(b, a, L)
    S = np.zeros(M)
    GX = np.empty((C, L))
    gb = np.zeros(N + 1)
    ga = np.zeros(M)
    gzi = np.zeros(M)
    for c in range(C - 1, -1, -1):
        U = Tha @ G[c] + Ou @ S
        GX[c] = Tga @ G[c] + Ogx @ S
        ext = np.concatenate([U, S])            # u[cL .. cL+L+M-1]
        for k in range(N + 1):
            gb[k] += ext[k: k + L] @ X[c]       # sum_n u[n+k] x[n]
        for k in range(1, M + 1):
            ga[k - 1] -= ext[k: k + L] @ Y[c]   # -sum_n u[n+k] y[n]
        if c == 0:
            gzi = U[:M].copy()
        S = U[:M].copy()
    gzi[T:] = 0.0
    return GX.reshape(-1)[:T], gb, ga, gzi
