"""Seeded workload generator: determinism, stability re-check, shapes."""
import numpy as np

from paper_2511_14390_gb300 import inputs


def test_deterministic_and_shapes():
    w1 = inputs.make("biquad_1024x48000", B=8, T=100)
    w2 = inputs.make("biquad_1024x48000", B=8, T=100)
    assert np.array_equal(w1.x, w2.x) and np.array_equal(w1.a, w2.a)
    assert w1.x.shape == (8, 100) and w1.b.shape == (8, 3) and w1.a.shape == (8, 2)
    assert w1.x.dtype == np.float32 and w1.zi.shape == (8, 2)
    assert inputs.make("allpole2_4x4096").zi is None


def test_rounded_denominators_are_stable():
    for name, B in [("allpole16_256x262144", 8), ("df64_64x1048576", 4)]:
        w = inputs.make(name, B=B, T=8)
        for i in range(B):
            roots = np.roots(np.concatenate([[1.0], w.a[i].astype(np.float64)]))
            assert np.abs(roots).max() < inputs.MAX_ROOT
        if name.startswith("df64"):
            assert np.abs(w.b).max() <= 1.0 + 1e-7


def test_ragged_layout():
    w = inputs.make_ragged(B=32, T_range=(10, 1000))
    assert w.offsets[0] == 0 and w.offsets[-1] == w.x.size
    assert (np.diff(w.offsets) >= 10).all() and (np.diff(w.offsets) <= 1000).all()
    assert ((w.Ns >= 0) & (w.Ns <= w.Ms)).all()
    for i in range(32):
        assert not w.a[i, w.Ms[i]:].any() and not w.b[i, w.Ns[i] + 1:].any()
