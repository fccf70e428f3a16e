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


def test_class_work_and_roofline():
    """Algorithmic work per kernel class (orders >= 3 on the decoupled path, <= 2 on the
    single-kernel one) and the roofline table built from per-class event times."""
    lens = np.array([64 * 10, 64 * 10])
    Ms = np.array([2, 32])
    w = bench.class_work(lens, Ms)
    assert w["fused"]["bytes"] == 20 * 640 + 2 * 4 * 10 * 2
    assert w["u_pass"]["bytes"] == 16 * 640 + 4 * 10 * 32
    assert w["scan"]["ops"] == 2 * 10 * 32 * 32 * bench.DW_MAC_OPS
    cls = {"scan": (3.0, 6), "u_pass": (1.5, 3), "fused": (0.0, 0)}
    dom, table = bench.roofline_from_classes(cls, w, 3, 6000.0, "measured")
    assert dom == "scan" and set(table) == {"scan", "u_pass"}
    assert table["scan"]["bound"] == "alu" and table["u_pass"]["bound"] == "hbm"
    assert abs(table["u_pass"]["achieved"] - w["u_pass"]["bytes"] / 0.5e-3 / 1e9) < 1e-9
    assert abs(table["scan"]["frac"] - table["scan"]["achieved"] / bench.FP32_OPS_PEAK_T) < 1e-12


def test_oracle_sample_is_bounded():
    """The CPU legs time a deterministic, bounded sample of the workload's channels."""
    from paper_2511_14390_gb300 import inputs
    w = inputs.make_ragged(B=64, T_range=(100, 5000), M_range=(1, 4), seed=3)
    kind, idx, n = bench.oracle_sample(w, 20000)
    assert kind == "ragged" and n <= 20000 and len(idx) >= 1
    assert n == int(np.diff(w.offsets)[idx].sum())


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
