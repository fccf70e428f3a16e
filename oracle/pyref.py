"""Pure-Python restatement of the oracle for tiny cases (test infrastructure).

The arithmetic is generic: pass Python floats for an FP64 run or
``fractions.Fraction`` values for an exact rational run (used by the tests to
build brute-force Jacobians with no rounding at all).

Notation as in the paper's Eq. rtf: ``b = [b_0..b_N]``, ``a = [a_1..a_M]``
(a_0 = 1 implicit), ``zi`` is the transposed-direct-form-II state at n = 0.
"""
from __future__ import annotations


def forward(x, b, a, zi=None):
    """Difference equation of Eq. rtf with the initial state injected into the
    all-pole input (w[n] += zi[n] for n < M); returns y as a list."""
    T, N, M = len(x), len(b) - 1, len(a)
    zero = x[0] * 0 if T else 0
    y = []
    for n in range(T):
        w = zero
        for k in range(N + 1):
            if n - k >= 0:
                w = w + b[k] * x[n - k]
        if zi is not None and n < M:
            w = w + zi[n]
        acc = w
        for k in range(1, M + 1):
            if n - k >= 0:
                acc = acc - a[k - 1] * y[n - k]
        y.append(acc)
    return y


def backward(g, x, y, b, a):
    """Reverse-time adjoint of Sec. 3.1 (scalar form, u[n >= T] = 0 as in App. A).
    Returns (grad_x, grad_b, grad_a, grad_zi) as lists."""
    T, N, M = len(x), len(b) - 1, len(a)
    zero = g[0] * 0 if T else 0
    u = [zero] * T
    for n in range(T - 1, -1, -1):
        acc = g[n]
        for k in range(1, M + 1):
            if n + k < T:
                acc = acc - a[k - 1] * u[n + k]
        u[n] = acc
    gx = []
    for n in range(T):
        acc = zero
        for k in range(N + 1):
            if n + k < T:
                acc = acc + b[k] * u[n + k]
        gx.append(acc)
    gb = []
    for k in range(N + 1):
        acc = zero
        for n in range(k, T):
            acc = acc + u[n] * x[n - k]
        gb.append(acc)
    ga = []
    for k in range(1, M + 1):
        acc = zero
        for n in range(k, T):
            acc = acc + u[n] * y[n - k]
        ga.append(-acc)
    gzi = [u[k] if k < T else zero for k in range(M)]
    return gx, gb, ga, gzi
