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


def test_kernel_name_follows_the_dispatch():
    """Main-kernel names per state bucket: warp-specialised kernels where their layouts
    fit (forward to MB = 16 with two signal stages at 16, backward to MB = 8), the
    first-generation kernels above; double-word scan above order 4."""
    assert bench.kernel_name("forward", 2) == "chunk_fwd_ws_kernel<2, 0, 3>"
    assert bench.kernel_name("forward", 5) == "chunk_fwd_ws_kernel<8, 1, 3>"
    assert bench.kernel_name("forward", 16) == "chunk_fwd_ws_kernel<16, 1, 2>"
    assert bench.kernel_name("forward", 33) == "chunk_fwd_kernel<64, 1>"
    assert bench.kernel_name("backward", 4) == "chunk_bwd_ws_kernel<4, 0>"
    assert bench.kernel_name("backward", 12) == "chunk_bwd_kernel<16, 1, 0>"


def test_profiled_traffic_reads_marker_and_detects_stale_sources(tmp_path, monkeypatch):
    """The committed-summary lookup: the marker's bytes when the recorded SHA-256 of the
    kernel's sources matches, None once a source changed or the workload differs."""
    import hashlib
    src = tmp_path / "k.cu"
    src.write_bytes(b"kernel v1")
    digest = hashlib.sha256(b"kernel v1").hexdigest()
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "my_kernel_wl.md").write_text(
        f"# summary\n<!-- traffic kernel=my_kernel<2,0> workload=wl bytes_per_launch=1.5e+08 "
        f"sources=k.cu sha256={digest} -->\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("my_kernel<2, 0>", "wl") == 1.5e8
    assert bench.profiled_traffic("my_kernel<2, 0>", "other") is None
    src.write_bytes(b"kernel v2")
    assert bench.profiled_traffic("my_kernel<2, 0>", "wl") is None
