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


def test_profiled_tensor_reads_its_own_marker(tmp_path, monkeypatch):
    """A summary may hold several markers: the tensor-pipe lookup takes the `tensor`
    marker of the kernel and workload, beside the traffic one, and goes stale with the
    sources like it."""
    import hashlib
    src = tmp_path / "k.cu"
    src.write_bytes(b"kernel v1")
    digest = hashlib.sha256(b"kernel v1").hexdigest()
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "tc_kernel_wl.md").write_text(
        f"# summary\n<!-- traffic kernel=tc_kernel workload=wl bytes_per_launch=2e+09 "
        f"sources=k.cu sha256={digest} -->\n<!-- tensor kernel=tc_kernel workload=wl "
        f"active_pct=6.86 sources=k.cu sha256={digest} -->\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("tc_kernel", "wl") == 2e9
    assert bench.profiled_tensor("tc_kernel", "wl") == 6.86
    assert bench.profiled_tensor("tc_kernel", "other") is None
    src.write_bytes(b"kernel v2")
    assert bench.profiled_tensor("tc_kernel", "wl") is None


def test_tuner_choice_is_deterministic():
    """The tuner's pick depends only on the measurements: the fastest pair, ties broken
    toward the shorter span and then fewer chains, whatever the order of the candidates."""
    from paper_2511_14390_gb300 import tune
    t = {(4, 8): 2.0, (2, 16): 1.5, (8, 4): 1.5, (1, 8): 3.0, (2, 8): 1.5}
    assert tune.choose(t) == (2, 8)
    shuffled = dict(reversed(list(t.items())))
    assert tune.choose(shuffled) == (2, 8)
    assert tune.shape_key("GB300", 32, 4096, 593554462) == tune.shape_key("GB300", 32, 4500,
                                                                        650000000)
    assert tune.shape_key("GB300", 32, 4096, 593554462) != tune.shape_key("GB300", 16, 4096,
                                                                        593554462)


def test_tuner_cache_roundtrip(tmp_path, monkeypatch):
    """Cached pairs are merged into the file and installed by lookup (through a fake
    library setter: no GPU)."""
    from paper_2511_14390_gb300 import tune
    calls = []
    monkeypatch.setattr(tune.dfilt, "dfilt_tuning_set", lambda mb, s, c: calls.append((mb, s, c)))
    path = str(tmp_path / "cache.json")
    tune.save({"k32": {"span_tiles": 16, "chains_per_sm": 8, "ms": 1.0}}, path)
    tune.save({"k16": {"span_tiles": 2, "chains_per_sm": 16, "ms": 2.0}}, path)
    hits = tune.lookup({32: "k32", 16: "k16", 64: "missing"}, path)
    assert set(hits) == {32, 16} and sorted(calls) == [(16, 2, 16), (32, 16, 8)]
    # the descent installs the best candidate of each bucket in turn
    calls.clear()
    times = iter([3.0, 1.0, 2.0, 5.0])
    table, seen = tune.tune(None, [32, 64], lambda step: next(times), spans=(1, 2),
                            chains={32: (8,), 64: (4,)})
    assert table[32][:2] == (2, 8) and table[64][:2] == (1, 4)
    assert calls[-1] == (64, 1, 4) and (32, 2, 8) in calls
