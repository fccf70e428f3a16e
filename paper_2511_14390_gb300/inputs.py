"""Seeded synthetic workloads for the direct-form filter path.

This module only draws inputs; it holds none of the filter arithmetic and is the
one module shared by the CUDA path's tests/benchmark and the FP64 oracle's tests.

Recipe (per channel):
  * poles: M//2 conjugate pairs r e^{+-i theta}, r ~ U[r_lo, r_hi], theta ~ U[0, pi];
    odd M adds one real pole with the same radius law and a random sign;
  * a = real(poly(poles))[1:] in FP64, rounded to fp32; the roots of the ROUNDED
    denominator are re-checked in FP64 and the channel is re-drawn when any has
    |z| >= 0.9995 (re-draws are counted);
  * zeros (N > 0): N//2 conjugate pairs with radius U[0, 1.2] and angle U[0, pi], odd N
    adds one real zero; b = poly(zeros) with b_0 = 1, optionally scaled so max|b| = 1;
    all-pole channels (N = 0) have b = [1];
  * x ~ N(0, 1) fp32; zi ~ N(0, 0.1^2) fp32 (or zero); upstream gradient gy ~ N(0, 1).

Seeds: numpy ``default_rng(1000 + config_index)``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# The five workloads (index = seed offset).  Sizes are (B channels, T samples).
CONFIGS = {
    "allpole2_4x4096": dict(idx=0, B=4, T=4096, M=2, N=0, r=(0.5, 0.95), zi=False,
                            bscale=False, grads=("x", "a", "zi")),
    "biquad_1024x48000": dict(idx=1, B=1024, T=48000, M=2, N=2, r=(0.5, 0.99), zi=True,
                              bscale=False, grads=("x", "b", "a", "zi")),
    "allpole16_256x262144": dict(idx=2, B=256, T=262144, M=16, N=0, r=(0.8, 0.995),
                                 zi=False, bscale=False, grads=("x", "a", "zi")),
    "df64_64x1048576": dict(idx=3, B=64, T=1 << 20, M=64, N=64, r=(0.9, 0.999), zi=True,
                            bscale=True, grads=("x", "b", "a", "zi")),
    "ragged4096": dict(idx=4, B=4096, M=(1, 32), T=(1000, 1_000_000), r=(0.5, 0.99),
                       zi=True, bscale=True, grads=("x", "b", "a", "zi")),
}

MAX_ROOT = 0.9995


@dataclass
class Workload:
    """Inputs of one batch.  Fixed shape: x[B,T]; ragged: x packed [sum T_i] with
    offsets[B+1].  b[B, Nmax+1], a[B, Mmax], zi[B, Mmax] (zero-padded rows)."""
    x: np.ndarray
    b: np.ndarray
    a: np.ndarray
    zi: np.ndarray | None
    gy: np.ndarray
    M: int
    N: int
    radius: np.ndarray                     # max pole radius drawn per channel
    offsets: np.ndarray | None = None      # ragged only
    Ms: np.ndarray | None = None           # ragged only
    Ns: np.ndarray | None = None           # ragged only
    redraws: int = 0
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def B(self) -> int:
        return self.b.shape[0]

    @property
    def ragged(self) -> bool:
        return self.offsets is not None

    @property
    def samples(self) -> int:
        return int(self.x.size)


def _poly_real(roots):
    return np.real(np.poly(roots)) if len(roots) else np.ones(1)


def _draw_roots(rng, order, rlo, rhi):
    roots = []
    for _ in range(order // 2):
        r = rng.uniform(rlo, rhi)
        th = rng.uniform(0.0, np.pi)
        roots += [r * np.exp(1j * th), r * np.exp(-1j * th)]
    if order % 2:
        r = rng.uniform(rlo, rhi)
        roots.append(r if rng.uniform() < 0.5 else -r)
    return np.array(roots, dtype=np.complex128)


def draw_denominator(rng, M, rlo, rhi):
    """Returns (a[1..M] fp32, max radius, re-draw count)."""
    redraws = 0
    while True:
        poles = _draw_roots(rng, M, rlo, rhi)
        a64 = _poly_real(poles)
        a32 = a64.astype(np.float32)
        rr = np.abs(np.roots(a32.astype(np.float64))) if M > 0 else np.zeros(0)
        if M == 0 or rr.max() < MAX_ROOT:
            return a32[1:], float(np.abs(poles).max()), redraws
        redraws += 1


def draw_numerator(rng, N, bscale):
    if N == 0:
        return np.ones(1, dtype=np.float32)
    zeros = _draw_roots(rng, N, 0.0, 1.2)
    b = _poly_real(zeros)
    if bscale:
        b = b / np.abs(b).max()
    return b.astype(np.float32)


def make(name: str, *, B: int | None = None, T: int | None = None, seed: int | None = None,
         zi: bool | None = None, M: int | None = None, N: int | None = None) -> Workload:
    """Fixed-shape workload ``name`` from CONFIGS, optionally resized (B, T) or
    re-ordered (M, N) for smaller parity cases."""
    cfg = CONFIGS[name]
    if name == "ragged4096":
        raise ValueError("use make_ragged for the ragged workload")
    B = cfg["B"] if B is None else B
    T = cfg["T"] if T is None else T
    M = cfg["M"] if M is None else M
    N = cfg["N"] if N is None else N
    want_zi = cfg["zi"] if zi is None else zi
    rng = np.random.default_rng(1000 + cfg["idx"] if seed is None else seed)
    a = np.zeros((B, M), dtype=np.float32)
    b = np.zeros((B, N + 1), dtype=np.float32)
    radius = np.zeros(B)
    redraws = 0
    for i in range(B):
        a[i], radius[i], rd = draw_denominator(rng, M, *cfg["r"])
        redraws += rd
        b[i] = draw_numerator(rng, N, cfg["bscale"])
    x = rng.standard_normal((B, T), dtype=np.float32)
    zi_arr = (0.1 * rng.standard_normal((B, M))).astype(np.float32) if want_zi else None
    gy = rng.standard_normal((B, T), dtype=np.float32)
    return Workload(x=x, b=b, a=a, zi=zi_arr, gy=gy, M=M, N=N, radius=radius,
                    redraws=redraws, name=name, meta=dict(cfg))


def make_ragged(name: str = "ragged4096", *, B: int | None = None,
                T_range: tuple[int, int] | None = None, M_range: tuple[int, int] | None = None,
                seed: int | None = None) -> Workload:
    """Ragged workload: orders M_i ~ U{Mlo..Mhi}, N_i ~ U{0..M_i}, lengths
    T_i log-uniform in T_range, packed into one signal with offsets."""
    cfg = CONFIGS[name]
    B = cfg["B"] if B is None else B
    Tlo, Thi = cfg["T"] if T_range is None else T_range
    Mlo, Mhi = cfg["M"] if M_range is None else M_range
    rng = np.random.default_rng(1000 + cfg["idx"] if seed is None else seed)
    Ms = rng.integers(Mlo, Mhi + 1, size=B).astype(np.int32)
    Ns = np.array([rng.integers(0, m + 1) for m in Ms], dtype=np.int32)
    Ts = np.round(np.exp(rng.uniform(np.log(Tlo), np.log(Thi), size=B))).astype(np.int64)
    Mmax, Nmax = int(Ms.max()), int(Ms.max())
    a = np.zeros((B, Mmax), dtype=np.float32)
    b = np.zeros((B, Nmax + 1), dtype=np.float32)
    radius = np.zeros(B)
    redraws = 0
    for i in range(B):
        ai, radius[i], rd = draw_denominator(rng, int(Ms[i]), *cfg["r"])
        a[i, : Ms[i]] = ai
        redraws += rd
        bi = draw_numerator(rng, int(Ns[i]), cfg["bscale"])
        b[i, : Ns[i] + 1] = bi
    offsets = np.zeros(B + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(Ts)
    total = int(offsets[-1])
    x = rng.standard_normal(total, dtype=np.float32)
    zi = np.zeros((B, Mmax), dtype=np.float32)
    if cfg["zi"]:
        for i in range(B):
            zi[i, : Ms[i]] = 0.1 * rng.standard_normal(int(Ms[i]))
    gy = rng.standard_normal(total, dtype=np.float32)
    return Workload(x=x, b=b, a=a, zi=zi, gy=gy, M=Mmax, N=Nmax, radius=radius,
                    offsets=offsets, Ms=Ms, Ns=Ns, redraws=redraws, name=name,
                    meta=dict(cfg))
