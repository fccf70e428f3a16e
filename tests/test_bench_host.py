"""Host-side helpers of bench.py (no GPU): per-pole-radius error bins."""
import numpy as np

import bench


def test_radius_bins():
    per = {"y": np.array([1e-7, 2e-7, 5e-6, 3e-6, 9e-5]), "grad_x": np.arange(5) * 1e-7}
    r = np.array([0.6, 0.85, 0.95, 0.98, 0.995])
    out = bench.radius_bins(per, r)
    assert out["[0.5, 0.9)"]["channels"] == 2
    assert out["[0.5, 0.9)"]["y"]["max"] == 2e-7
    assert abs(out["[0.9, 0.99)"]["y"]["median"] - 4e-6) < 1e-18
    assert out["[0.99, 0.999)"]["grad_x"]["max"] == 4e-7
    assert "other" not in out
    out = bench.radius_bins(per, np.array([0.2, 0.6, 0.6, 0.6, 0.9995]))
    assert out["other"]["channels"] == 2 and out["[0.5, 0.9)"]["channels"] == 3
