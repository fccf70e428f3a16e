#!/usr/bin/env python
"""Benchmark: forward + backward throughput (Gsamples/s) of batched direct-form IIR
filters on GB300, the chunked tensor-core path beside the sequential kernel, with the
relative error of both against the FP64 oracle.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Headline (N = 1): the largest single-GPU workload, a ragged batch of 4096 filters
(orders 1..32, numerators 0..M, lengths log-uniform 1e3..1e6, about 594M samples), run
as a training step: forward, the gradient of an MSE loss against the output of a second
filter bank, backward for every input (x, b, a, zi).  The step is captured once in a
CUDA graph and replayed (the configured form); the eager step is reported beside it.
The smaller workloads (order-2 all-pole 4 x 4096, biquads 1024 x 48000, order-16
all-pole 256 x 2^18, orders 64/64 64 x 2^20) are measured as fwd + bwd call pairs in
`configs`.  Under torchrun every rank filters its own copy of the headline batch
(channels are independent problems, no collective on the data path): weak scaling;
rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd Gsamples/s, chunked TC vs sequential kernel at stated rel err vs FP64"
UNIT = "Gsamples/s"
FALLBACK_HBM = 6800.0
# FP32 issue rate of GB300 (152 SMs x 128 FP32 lanes x 2.07 GHz, an FMA counted once):
# the roofline of the double-word chunk-state scan, which is bound by FP32 arithmetic
FP32_OPS_PEAK_T = 152 * 128 * 2.07e9 / 1e12
# FP32 operations of one double-word multiply-add of the scan: an exact product (mul +
# fma), two cross terms (2 fma), a TwoSum (6 add) and the low-part accumulation (2 add)
DW_MAC_OPS = 12
HEADLINE = "ragged4096"
CONFIGS = ["allpole2_4x4096", "biquad_1024x48000", "allpole16_256x262144", "df64_64x1048576"]


def args_():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=HEADLINE)
    p.add_argument("--no-configs", action="store_true", help="headline only")
    p.add_argument("--no-seq", action="store_true", help="skip the sequential-kernel legs")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-graph", action="store_true")
    p.add_argument("--no-jvp", action="store_true", help="skip the forward-mode (JVP) leg")
    p.add_argument("--no-tv", action="store_true", help="skip the parameter-varying leg")
    p.add_argument("--no-ss", action="store_true",
                   help="skip the dense state-space recurrence leg (M = 2, 64 x 2^20 steps)")
    p.add_argument("--tuning", default="",
                   help="install the decoupled scan's launch shape instead of measuring it: "
                        "'MB:span:chains,...' (e.g. 8:2:32,16:2:32,32:4:16)")
    p.add_argument("--channels", type=int, default=0,
                   help="override the workload's channel count (smaller profiling cases)")
    return p.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(v: float, world: int, device: str = "cuda") -> float:
    """The slowest rank's time: every rank passes its own, all get the maximum."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(samples_per_rank: int, world: int, ms: float) -> float:
    """Gsamples/s of the whole job: every rank filters its own replica of the batch
    (weak scaling), timed by the slowest rank."""
    return samples_per_rank * world / (ms / 1e3) / 1e9


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region.
    The GPU is addressed by its PCI bus id (the process sees it as device 0 whatever
    its index on the host), then by UUID, then by index."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    @staticmethod
    def target(torch) -> str | None:
        cands = []
        try:
            pr = torch.cuda.get_device_properties(torch.cuda.current_device())
            cands.append(f"{pr.pci_domain_id:08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0")
            u = str(pr.uuid)
            cands.append(u if u.startswith("GPU-") else "GPU-" + u)
        except Exception:
            pass
        cands.append(str(torch.cuda.current_device()))
        for c in cands:
            try:
                r = subprocess.run(["nvidia-smi", "-i", c, "--query-gpu=clocks.sm",
                                    "--format=csv,noheader,nounits"], capture_output=True,
                                   text=True, timeout=20)
                if r.returncode == 0 and r.stdout.strip():
                    return c
            except Exception:
                continue
        return None

    def __init__(self, target: str | None):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.target = target
        self.p = None
        if target is not None:
            try:
                self.p = subprocess.Popen(["nvidia-smi", "-i", target, f"--query-gpu={self.Q}",
                                           "--format=csv,noheader,nounits", "-lms", "50"],
                                          stdout=self.f, stderr=subprocess.DEVNULL)
            except Exception:
                self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "samples": 0}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [c.strip() for c in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm), "gpu": self.target}


RADIUS_BINS = [(0.5, 0.9), (0.9, 0.99), (0.99, 0.999)]


def radius_bins(per_channel: dict, radius) -> dict:
    """Max and median of per-channel errors in each pole-radius bin (the channels'
    largest drawn pole radius); channels outside every bin are reported as "other"."""
    radius = np.asarray(radius, dtype=np.float64)
    masks = {f"[{lo}, {hi})": (radius >= lo) & (radius < hi) for lo, hi in RADIUS_BINS}
    masks["other"] = ~np.any(np.stack(list(masks.values())), axis=0)
    out = {}
    for name, m in masks.items():
        if m.any():
            out[name] = {"channels": int(m.sum())}
            for k, v in per_channel.items():
                v = np.asarray(v, dtype=np.float64)[m]
                out[name][k] = {"max": float(v.max()), "median": float(np.median(v))}
    return out


def profiled_marker(tag, field, kname, workload):
    """A figure recorded in a committed ncu summary: the `field` of the
    `<!-- tag kernel=... workload=... field=... sources=... sha256=... -->` marker of
    `kname` on `workload`; None when there is no summary or a source of the kernel
    changed since the counters were taken (the recorded SHA-256 no longer matches)."""
    import glob
    import hashlib
    import re
    base = kname.split("<")[0]
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", f"{base}_*.md"))):
        txt = open(path).read()
        for m in re.finditer(r"<!-- " + tag + r" kernel=(\S+) workload=(\S+) " + field +
                             r"=([0-9.e+-]+) sources=(\S+) sha256=([0-9a-f]+) -->", txt):
            if m.group(1) != kname.replace(" ", "") or m.group(2) != workload:
                continue
            h = hashlib.sha256()
            for rel in m.group(4).split(","):
                src = os.path.join(ROOT, rel)
                if not os.path.exists(src):
                    return None
                h.update(open(src, "rb").read())
            if h.hexdigest() != m.group(5):
                return None   # stale: the kernel changed since the counters were taken
            return float(m.group(3))
    return None


def profiled_traffic(kname, workload):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of `kname`
    from the committed ncu summary of this workload, scaled to one full launch; None
    when there is no summary or the kernel source changed since it was captured."""
    return profiled_marker("traffic", "bytes_per_launch", kname, workload)


def profiled_tensor(kname, workload):
    """Tensor-pipe activity of `kname` (sm__pipe_tensor_cycles_active, % of peak while
    active, duration-weighted over the captured launches) from the committed ncu summary
    of this workload; None when there is none or the sources changed."""
    return profiled_marker("tensor", "active_pct", kname, workload)


# ----------------------------------------------------------------------------
# Workload accounting: which path each channel takes and the algorithmic work of each
# kernel class (per call pair), for the roofline
# ----------------------------------------------------------------------------

def uses_decoupled(M: int) -> bool:
    """Orders >= 3 (double-word scan, state buckets 8..64) take the decoupled path when
    the forward keeps its chunk states (the benchmark always does); orders <= 2 run the
    single-kernel path."""
    return M >= 3


def class_work(lens, Ms):
    """Algorithmic bytes (HBM classes) and FP32 operations (scan) of one fwd + bwd call
    pair, per kernel class, summed over channels:
      scan      2 (fwd, bwd) x chunks x M^2 double-word multiply-adds x 12 FP32 ops
      e_pass    x and gy read (4 B each), E written (4 M / 64 B, twice)
      y_pass    x read, y written (8 B), chunk states read (4 M / 64 B)
      u_pass    gy, x, y read, grad_x written (16 B), adjoint states read (4 M / 64 B)
      fused     20 B + 2 x 4 M / 64 B (the single-kernel forward and backward)
    """
    lens = np.asarray(lens, dtype=np.float64)
    Ms = np.asarray(Ms, dtype=np.float64)
    dec = Ms >= 3
    ch = np.ceil(lens / 64.0)
    st = 4.0 * ch * Ms   # bytes of one pass over the chunk states
    return {
        "scan": {"ops": float((2 * ch * Ms * Ms * DW_MAC_OPS)[dec].sum())},
        "e_pass": {"bytes": float((8 * lens + 2 * st)[dec].sum())},
        "y_pass": {"bytes": float((8 * lens + st)[dec].sum())},
        "u_pass": {"bytes": float((16 * lens + st)[dec].sum())},
        "fused": {"bytes": float((20 * lens + 2 * st)[~dec].sum())},
    }


def roofline_from_classes(cls_ms: dict, work: dict, steps: int, hbm: float, src: str):
    """Per class: ms per step, achieved rate and fraction of its roofline; returns the
    dominant class (largest time) and the table."""
    out = {}
    for k, w in work.items():
        ms, n = cls_ms.get(k, (0.0, 0))
        if n == 0 or ms <= 0:
            continue
        ms_step = ms / steps
        if "ops" in w:
            ach = w["ops"] / (ms_step / 1e3) / 1e12
            out[k] = {"bound": "alu", "ms_per_step": ms_step, "achieved": ach, "unit": "TFLOP/s",
                      "peak": FP32_OPS_PEAK_T, "frac": ach / FP32_OPS_PEAK_T,
                      "algorithmic": w["ops"], "records": n,
                      "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz"}
        else:
            ach = w["bytes"] / (ms_step / 1e3) / 1e9
            out[k] = {"bound": "hbm", "ms_per_step": ms_step, "achieved": ach, "unit": "GB/s",
                      "peak": hbm, "frac": ach / hbm, "algorithmic": w["bytes"], "records": n,
                      "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured"
                      else "fallback (6.8 TB/s)"}
    dom = max(out, key=lambda k: out[k]["ms_per_step"]) if out else None
    return dom, out


KERNEL_OF_CLASS = {"scan": "hi_scan_kernel", "u_pass": "hi_tc_kernel", "y_pass": "hi_tc_kernel",
                   "e_pass": "hi_e_kernel", "fused": "chunk_bwd_ws_kernel"}


# ----------------------------------------------------------------------------
# CPU baseline / reference arm: the FP64 oracle as it stands, on the host cores
# ----------------------------------------------------------------------------

def oracle_sample(w, max_samples):
    """A deterministic sample of the workload's channels (every k-th) holding at most
    max_samples samples (at least one channel)."""
    if not w.ragged:
        B, T = w.x.shape
        nb = max(1, min(B, int(max_samples // max(T, 1))))
        idx = np.unique(np.linspace(0, B - 1, nb).astype(int))
        return ("fixed", idx, int(len(idx) * T))
    lens = np.diff(w.offsets)
    k = 1
    while lens[::k].sum() > max_samples and k < len(lens):
        k *= 2
    idx = np.arange(0, w.B, k)
    return ("ragged", idx, int(lens[idx].sum()))


def oracle_step(w, sample):
    import oracle
    kind, idx, _ = sample
    if kind == "fixed":
        zi = None if w.zi is None else w.zi[idx]
        y = oracle.forward(w.x[idx], w.b[idx], w.a[idx], zi)
        oracle.backward(w.gy[idx], w.x[idx], y, w.b[idx], w.a[idx])
        return
    offs = w.offsets
    xs = np.concatenate([w.x[offs[i]:offs[i + 1]] for i in idx])
    gs = np.concatenate([w.gy[offs[i]:offs[i + 1]] for i in idx])
    lens = np.diff(offs)[idx]
    o2 = np.zeros(len(idx) + 1, dtype=np.int64)
    o2[1:] = np.cumsum(lens)
    y = oracle.forward_ragged(xs, o2, w.Ms[idx], w.Ns[idx], w.b[idx], w.a[idx], w.zi[idx])
    oracle.backward_ragged(gs, xs, y, o2, w.Ms[idx], w.Ns[idx], w.b[idx], w.a[idx])


def make_workload(name, channels=0):
    from paper_2511_14390_gb300 import inputs
    if name == HEADLINE:
        return inputs.make_ragged(name, **({"B": channels} if channels > 0 else {}))
    w = inputs.make(name, **({"B": channels} if channels > 0 else {}))
    if w.zi is None:   # zero initial conditions, passed explicitly so grad_zi has a buffer
        w.zi = np.zeros((w.B, w.M), dtype=np.float32)
    return w


def workload_config(w, name, algo="chunked"):
    if w.ragged:
        lens = np.diff(w.offsets)
        return {"workload": name, "B": int(w.B), "total_samples": int(w.x.size),
                "M": "1..32", "N": "0..M", "T": f"{int(lens.min())}..{int(lens.max())}",
                "algo": algo, "step": "forward + MSE-loss gradient + backward (x, b, a, zi)",
                "l2": "inputs larger than L2: x is %.0f MB, 129 MB L2" % (w.x.nbytes / 1e6)}
    return {"workload": name, "B": int(w.B), "T": int(w.x.shape[1]), "M": int(w.M),
            "N": int(w.N), "algo": algo, "step": "forward + backward (all gradients)",
            "l2": ("inputs larger than L2: x and gy are %.0f MB each, 129 MB L2" % (w.x.nbytes / 1e6))
            if w.x.nbytes > 129e6 else "inputs smaller than L2 (launch-bound workload)"}


def run_reference(a, world, rank):
    """The reference arm: the FP64 oracle, each step a bounded sample of the workload's
    channels sized so that warm-up and timed steps take about two minutes."""
    if rank != 0:
        return
    import oracle
    w = make_workload(a.workload)
    # size the sample from one timed pass over a small one (the rate is per sample)
    probe = oracle_sample(w, 2e6)
    t0 = time.perf_counter()
    oracle_step(w, probe)
    rate = probe[2] / max(time.perf_counter() - t0, 1e-9)
    budget = 120.0 / max(1, a.steps + a.warmup)
    sample = oracle_sample(w, max(1e5, rate * budget))
    for _ in range(a.warmup):
        oracle_step(w, sample)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        oracle_step(w, sample)
    dt = (time.perf_counter() - t0) / a.steps
    v = sample[2] / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w, a.workload, "oracle"),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.max_threads(),
                             "kind": "oracle",
                             "sample": f"{len(sample[1])} of the workload's {w.B} channels, "
                                       f"{sample[2]} samples per step, FP64 forward + backward "
                                       f"(sized for a ~2 min run)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_oracle_rate(w, budget_s=20.0):
    """The oracle as it stands on the host cores, on a bounded sample of the workload."""
    import oracle
    probe = oracle_sample(w, 2e6)
    t0 = time.perf_counter()
    oracle_step(w, probe)
    rate = probe[2] / max(time.perf_counter() - t0, 1e-9)
    sample = oracle_sample(w, max(1e5, rate * budget_s))
    t0 = time.perf_counter()
    oracle_step(w, sample)
    dt = time.perf_counter() - t0
    return {"value": sample[2] / dt / 1e9, "unit": UNIT, "cores": oracle.max_threads(),
            "kind": "oracle",
            "sample": f"{len(sample[1])} of the {w.B} channels ({sample[2]} samples), FP64 "
                      f"forward + backward (all gradients), one pass of {dt:.1f} s"}


# ----------------------------------------------------------------------------
# GPU side
# ----------------------------------------------------------------------------

class Runner:
    """Device buffers, workspaces and the C-ABI calls of one workload."""

    def __init__(self, w, algo, torch, dfilt, stream, path="auto"):
        self.w, self.torch, self.dfilt = w, torch, dfilt
        self.L = dfilt.lib()
        self.o = dfilt.make_opts(algo=algo, precision="tf32x3", path=path)
        dev = lambda arr: torch.from_numpy(np.ascontiguousarray(arr)).cuda()
        self.x, self.b, self.a, self.zi = dev(w.x), dev(w.b), dev(w.a), dev(w.zi)
        self.gy = dev(w.gy)
        self.B = w.B
        self.ragged = w.ragged
        buf = lambda n: torch.empty(max(int(n), 16), dtype=torch.uint8, device="cuda")
        if self.ragged:
            self.offs, self.Ms, self.Ns = dev(w.offsets), dev(w.Ms), dev(w.Ns)
            self.total = int(w.x.size)
            self.Nmax, self.Mmax = w.b.shape[1] - 1, w.a.shape[1]
            f, s, bw = dfilt.dfilt_workspace_size_ragged(self.B, self.total, self.Nmax, self.Mmax,
                                                         self.o)
        else:
            self.T = w.x.shape[1]
            self.total = self.B * self.T
            f, s, bw = dfilt.dfilt_workspace_size(self.B, self.T, w.N, w.M, self.o)
        self.fws, self.bws = f, bw
        self.wf, self.wb = buf(f), buf(bw)
        self.saved = buf(s) if s else None
        self.y = torch.empty_like(self.x)
        self.gx = torch.empty_like(self.x)
        self.gb, self.ga = torch.empty_like(self.b), torch.empty_like(self.a)
        self.gz = torch.zeros_like(self.zi)
        self.sptr = ctypes.c_void_p(stream.cuda_stream)
        self.target = None
        self.scale = 1.0

    P = staticmethod(lambda t: None if t is None else ctypes.c_void_p(t.data_ptr()))

    def fwd(self, sp=None, x=None, y=None):
        P, d = self.P, self.dfilt
        x = self.x if x is None else x
        y = self.y if y is None else y
        if self.ragged:
            d._check(self.L.dfilt_forward_ragged(P(x), P(self.offs), P(self.Ms), P(self.Ns),
                                                 P(self.b), P(self.a), P(self.zi), P(y),
                                                 P(self.saved), P(self.wf), self.fws, self.B,
                                                 self.total, self.Nmax, self.Mmax,
                                                 ctypes.byref(self.o), sp or self.sptr),
                     "dfilt_forward_ragged")
        else:
            d._check(self.L.dfilt_forward(P(x), P(self.b), P(self.a), P(self.zi), P(y),
                                          P(self.saved), P(self.wf), self.fws, self.B, self.T,
                                          self.w.N, self.w.M, ctypes.byref(self.o),
                                          sp or self.sptr), "dfilt_forward")

    def bwd(self, sp=None, gy=None, x=None, y=None, out=None):
        P, d = self.P, self.dfilt
        gy = self.gy if gy is None else gy
        x = self.x if x is None else x
        y = self.y if y is None else y
        gx, gb, ga, gz = out or (self.gx, self.gb, self.ga, self.gz)
        if self.ragged:
            d._check(self.L.dfilt_backward_ragged(P(gy), P(x), P(y), P(self.offs), P(self.Ms),
                                                  P(self.Ns), P(self.b), P(self.a), P(self.zi),
                                                  P(self.saved), P(gx), P(gb), P(ga), P(gz),
                                                  P(self.wb), self.bws, self.B, self.total,
                                                  self.Nmax, self.Mmax, ctypes.byref(self.o),
                                                  sp or self.sptr), "dfilt_backward_ragged")
        else:
            d._check(self.L.dfilt_backward(P(gy), P(x), P(y), P(self.b), P(self.a), P(self.zi),
                                           P(self.saved), P(gx), P(gb), P(ga), P(gz), P(self.wb),
                                           self.bws, self.B, self.T, self.w.N, self.w.M,
                                           ctypes.byref(self.o), sp or self.sptr),
                     "dfilt_backward")

    def set_training_target(self):
        """The MSE target: the output of a second filter bank (same orders and lengths,
        coefficients drawn afresh) on the same input."""
        from paper_2511_14390_gb300 import inputs
        torch = self.torch
        rng = np.random.default_rng(4321)
        b2, a2 = np.zeros_like(self.w.b), np.zeros_like(self.w.a)
        for i in range(self.B):
            M, N = int(self.w.Ms[i]), int(self.w.Ns[i])
            a2[i, :M], _, _ = inputs.draw_denominator(rng, M, 0.5, 0.99)
            b2[i, :N + 1] = inputs.draw_numerator(rng, N, True)
        keep = (self.b, self.a)
        self.b, self.a = torch.from_numpy(b2).cuda(), torch.from_numpy(a2).cuda()
        self.target = torch.empty_like(self.x)
        self.fwd(y=self.target)
        self.b, self.a = keep
        self.scale = 2.0 / float(self.total)
        # the loss gradient scale * (y - target) as one elementwise op on y
        self.neg_target = self.target.mul(-self.scale)
        torch.cuda.synchronize()

    def train_step(self, sp=None, x=None, y=None, gy=None, neg_target=None, out=None):
        """forward, dL/dy of mean((y - target)^2) = scale * y - scale * target (one
        elementwise op: the target is held as -scale * target), backward"""
        y = self.y if y is None else y
        gy = self.gy if gy is None else gy
        neg_target = self.neg_target if neg_target is None else neg_target
        self.fwd(sp, x=x, y=y)
        self.torch.add(neg_target, y, alpha=self.scale, out=gy)
        self.bwd(sp, gy=gy, x=x, y=y, out=out)

    def pair(self, sp=None):
        self.fwd(sp)
        self.bwd(sp)


def time_loop(torch, stream, fn, steps, warmup, barrier=lambda: None):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    return e0.elapsed_time(e1) / steps


def graph_time(torch, stream, fn_on, steps, warmup, barrier=lambda: None):
    """The step captured once in a CUDA graph on a side stream, replayed `steps` times."""
    gs = torch.cuda.Stream()
    gptr = ctypes.c_void_p(gs.cuda_stream)
    gs.wait_stream(stream)
    with torch.cuda.stream(gs):
        for _ in range(2):
            fn_on(gptr)
    torch.cuda.synchronize()
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg, stream=gs):
        fn_on(gptr)
    ms = time_loop(torch, stream, cg.replay, steps, warmup, barrier)
    del cg
    return ms


def class_timing(torch, dfilt, fn, steps):
    torch.cuda.synchronize()
    dfilt.dfilt_kernel_timing(True)
    try:
        for _ in range(steps):
            fn()
        torch.cuda.synchronize()
        cls = dfilt.dfilt_kernel_timing_read_classes()
    finally:
        dfilt.dfilt_kernel_timing(False)
    return cls


def sampled_errors(w, y, grads, gy, idx=None, pick=None):
    """Per-channel max|err| / max|ref| of y and every gradient against the FP64 oracle,
    on sampled channels (fixed shape: rows idx; ragged: channel indices `pick`, with y
    and grads given per picked channel); gy is the upstream gradient the run used."""
    import oracle
    per = {k: [] for k in ("y", "grad_x", "grad_b", "grad_a", "grad_zi")}
    radius = []

    def rel(g, r):
        g = np.asarray(g, np.float64)
        return float(np.abs(g - r).max() / max(np.abs(r).max(), 1e-300)) if r.size else 0.0

    if not w.ragged:
        zi = None if w.zi is None else w.zi[idx]
        yr = oracle.forward(w.x[idx], w.b[idx], w.a[idx], zi)
        gr = oracle.backward(gy[idx], w.x[idx], yr, w.b[idx], w.a[idx])
        for j, i in enumerate(idx):
            per["y"].append(rel(y[j], yr[j]))
            for k, g, r in zip(("grad_x", "grad_b", "grad_a", "grad_zi"), grads, gr):
                per[k].append(rel(g[j], r[j]))
            radius.append(w.radius[i])
    else:
        offs = w.offsets
        for j, i in enumerate(pick):
            s, e = int(offs[i]), int(offs[i + 1])
            M, N = int(w.Ms[i]), int(w.Ns[i])
            xs, gys = w.x[s:e][None], gy[s:e][None]
            bs, as_, zs = w.b[i:i + 1, :N + 1], w.a[i:i + 1, :M], w.zi[i:i + 1, :M]
            yr = oracle.forward(xs, bs, as_, zs)
            gr = oracle.backward(gys, xs, yr, bs, as_)
            per["y"].append(rel(y[j], yr[0]))
            for k, g, r in zip(("grad_x", "grad_b", "grad_a", "grad_zi"), grads[j], gr):
                per[k].append(rel(g, r[0]))
            radius.append(w.radius[i])
    out = {k: float(max(v)) for k, v in per.items()}
    out.update({"channels_checked": len(radius),
                "metric": "per-channel max|err| / max|ref|, max over checked channels",
                "by_pole_radius": radius_bins(per, np.asarray(radius))})
    return out


def ragged_pick(w):
    """Sampled channels of a ragged batch: three per state bucket among those shorter
    than 300k samples (the oracle recomputes them whole), and the longest one."""
    lens = np.diff(w.offsets)
    pick = []
    for lo, hi in ((1, 2), (3, 4), (5, 8), (9, 16), (17, 32)):
        cand = np.where((w.Ms >= lo) & (w.Ms <= hi) & (lens < 300_000))[0]
        pick += [int(c) for c in cand[:3]]
    pick.append(int(np.argmax(lens)))
    return pick


def ragged_outputs(r, w, pick):
    offs = w.offsets
    seg = lambda t: [t[int(offs[i]):int(offs[i + 1])].cpu().numpy() for i in pick]
    ys, gxs = seg(r.y), seg(r.gx)
    grads = [(gxs[j], r.gb[i, :int(w.Ns[i]) + 1].cpu().numpy(),
              r.ga[i, :int(w.Ms[i])].cpu().numpy(), r.gz[i, :int(w.Ms[i])].cpu().numpy())
             for j, i in enumerate(pick)]
    return ys, grads


def hi_buckets(Ms):
    """State buckets of the decoupled path present in a batch (orders 3..8 run in 8)."""
    out = set()
    for m in np.unique(np.asarray(Ms)):
        if m >= 3:
            out.add(next(v for v in (8, 16, 32, 64) if m <= v))
    return sorted(out)


def parse_tuning(spec: str) -> dict:
    """'MB:span:chains,...' -> {MB: (span, chains)}."""
    out = {}
    for item in filter(None, (t.strip() for t in spec.split(","))):
        mb, sp, ch = (int(v) for v in item.split(":"))
        out[mb] = (sp, ch)
    return out


def autotune(step, Ms, torch, dfilt, stream, given: str = ""):
    """The measured launch shape of the decoupled scan for this batch (span length and
    chains per SM of every state bucket present), installed for the runs that follow;
    reported per bucket with the best step time.  With `given` ('MB:span:chains,...')
    that shape is installed instead and nothing is measured."""
    from paper_2511_14390_gb300 import tune
    tune.reset()
    buckets = hi_buckets(Ms)
    if not buckets:
        return None
    if given:
        table = parse_tuning(given)
        for mb, (sp, ch) in table.items():
            dfilt.dfilt_tuning_set(mb, sp, ch)
        return {"given": {str(mb): {"span_tiles": sp, "chains_per_sm": ch}
                          for mb, (sp, ch) in table.items()}}
    t0 = time.perf_counter()
    table, seen = tune.tune(step, buckets, lambda fn: time_loop(torch, stream, fn, 2, 1))
    return {"seconds": time.perf_counter() - t0,
            "chosen": {str(mb): {"span_tiles": sp, "chains_per_sm": c, "ms_per_step": ms}
                       for mb, (sp, c, ms) in table.items()},
            "candidates": {str(mb): len(v) for mb, v in seen.items()}}


def fixed_config(name, torch, dfilt, stream, a, hbm, src):
    """One fixed-shape workload: chunked fwd + bwd call pairs (automatic path), the
    sequential kernel, errors of both against the oracle on sampled channels, and the
    per-class roofline."""
    w = make_workload(name)
    B, T = w.x.shape
    r = Runner(w, "chunked", torch, dfilt, stream)
    tuned = autotune(r.pair, np.full(B, w.M), torch, dfilt, stream)
    steps = max(3, min(a.steps, int(2e9 // max(1, B * T))))
    ms = time_loop(torch, stream, r.pair, steps, a.warmup)
    out = {"workload": name, "B": B, "T": T, "M": int(w.M), "N": int(w.N),
           "value": B * T / (ms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": ms, "steps": steps,
           "path": "decoupled" if uses_decoupled(w.M) else "fused", "autotune": tuned}
    if B * T < 1e6:   # launch-bound: the pair captured in a CUDA graph as well
        gms = graph_time(torch, stream, lambda sp: r.pair(sp), steps * 20, a.warmup)
        out["graph_replay"] = {"value": B * T / (gms / 1e3) / 1e9, "ms_per_step": gms}
    cls = class_timing(torch, dfilt, r.pair, 3)
    dom, rl = roofline_from_classes(cls, class_work(np.full(B, T), np.full(B, w.M)), 3, hbm, src)
    out["kernels"] = rl
    out["roofline_dominant"] = dom
    status = dfilt.dfilt_sync_status()
    if status != 0:
        raise RuntimeError(f"{name}: device status {dfilt.STATUS[status]}")
    nidx = 3 if name.startswith("df64") else (8 if B * T > 1e7 else min(B, 16))
    idx = np.unique(np.linspace(0, B - 1, nidx).astype(int))
    host = lambda t: t.cpu().numpy()[idx]
    out["rel_err_vs_fp64"] = sampled_errors(w, host(r.y), [host(r.gx), host(r.gb), host(r.ga),
                                                            host(r.gz)], w.gy, idx=idx)
    del r
    if not a.no_seq:
        s = Runner(w, "sequential", torch, dfilt, stream)
        ssteps = max(2, min(10, int(4e8 // max(1, B * T * w.M))))
        sms = time_loop(torch, stream, s.pair, ssteps, 1)
        out["sequential"] = {"value": B * T / (sms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": sms,
                             "steps": ssteps,
                             "rel_err_vs_fp64": sampled_errors(
                                 w, host(s.y), [host(s.gx), host(s.gb), host(s.ga), host(s.gz)],
                                 w.gy, idx=idx)}
        del s
    torch.cuda.empty_cache()
    return out


def main():
    a = args_()
    world, rank, local = dist_env()
    if a.impl == "reference":
        run_reference(a, world, rank)
        return
    import torch
    import torch.distributed as dist
    from paper_2511_14390_gb300 import dfilt

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    hbm, src = peaks()

    def barrier():
        if world > 1:
            dist.barrier()

    def maxrank(v):
        return max_over_ranks(v, world)

    # ---------------- headline: the ragged training step ----------------
    w = make_workload(a.workload, a.channels)
    r = Runner(w, "chunked", torch, dfilt, stream)
    ragged = w.ragged
    if ragged:
        r.set_training_target()
        step = r.train_step
        step_on = lambda sp: r.train_step(sp)
    else:
        step = r.pair
        step_on = lambda sp: r.pair(sp)
    samples = int(w.x.size)
    tuned = autotune(step, w.Ms if ragged else np.full(w.B, w.M), torch, dfilt, stream, a.tuning)
    clk = Clocks(Clocks.target(torch))
    n0 = dfilt.dfilt_launch_count()
    ms_eager = maxrank(time_loop(torch, stream, step, a.steps, a.warmup, barrier))
    launches = (dfilt.dfilt_launch_count() - n0) // (a.steps + a.warmup)
    graph = None
    if not a.no_graph:
        try:
            gms = maxrank(graph_time(torch, stream, step_on, a.steps, a.warmup, barrier))
            graph = {"value": whole_job_rate(samples, world, gms), "unit": UNIT, "ms_per_step": gms,
                     "steps": a.steps}
        except Exception as ex:   # the eager numbers stand; the failure is reported
            graph = {"error": repr(ex)[:200]}
    clocks = clk.stop()
    status = dfilt.dfilt_sync_status()
    if status != 0:
        raise RuntimeError(f"device status {dfilt.STATUS[status]}")
    use_graph = graph is not None and "ms_per_step" in graph
    ms = graph["ms_per_step"] if use_graph else ms_eager
    value = whole_job_rate(samples, world, ms)

    # kernel classes of the step (event pairs around each class's launches)
    cls = class_timing(torch, dfilt, step, 3)
    lens = np.diff(w.offsets) if ragged else np.full(w.B, w.x.shape[1])
    Ms = w.Ms if ragged else np.full(w.B, w.M)
    dom, kernels = roofline_from_classes(cls, class_work(lens, Ms), 3, hbm, src)
    fwd_ms, bwd_ms = cls["forward"][0] / 3, cls["backward"][0] / 3

    # accuracy of this run's outputs against the FP64 oracle on sampled channels, and
    # the sequential kernel on the same step
    rel_err, seq = None, None
    if rank == 0:
        if ragged:
            pick = ragged_pick(w)
            ys, grads = ragged_outputs(r, w, pick)
            rel_err = sampled_errors(w, ys, grads, r.gy.cpu().numpy(), pick=pick)
            if not a.no_seq:
                s = Runner(w, "sequential", torch, dfilt, stream)
                s.target, s.scale, s.neg_target = r.target, r.scale, r.neg_target
                sms = time_loop(torch, stream, s.train_step, 2, 1)
                sys_, sgr = ragged_outputs(s, w, pick)
                seq = {"value": samples / (sms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": sms,
                       "steps": 2, "rel_err_vs_fp64": sampled_errors(w, sys_, sgr,
                                                                     s.gy.cpu().numpy(), pick=pick)}
                del s
        else:
            idx = np.unique(np.linspace(0, w.B - 1, 16).astype(int))
            host = lambda t: t.cpu().numpy()[idx]
            rel_err = sampled_errors(w, host(r.y), [host(r.gx), host(r.gb), host(r.ga),
                                                    host(r.gz)], w.gy, idx=idx)
    barrier()

    # ---------------- end to end through the C ABI from pinned host memory ----------------
    e2e = None
    if not a.no_e2e:
        e2e = run_e2e(r, w, torch, stream, world, samples, barrier, maxrank)

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        cpu = cpu_oracle_rate(w)

    # ---------------- the other configurations, forward-mode and state-space rows ----------
    configs = None
    del r
    torch.cuda.empty_cache()
    if world == 1 and not a.no_configs and a.workload == HEADLINE and a.channels == 0:
        configs = {name: fixed_config(name, torch, dfilt, stream, a, hbm, src) for name in CONFIGS}
    jvp = None if a.no_jvp else run_jvp(torch, dfilt, stream, a, world, barrier, maxrank, hbm, src)
    ssl = None if a.no_ss else run_ss(torch, dfilt, stream, a, world, barrier, maxrank, hbm, src)
    tvl = None if a.no_tv else run_tv(torch, dfilt, stream, a, world, barrier, maxrank, hbm, src)

    if rank == 0:
        roof = None
        if dom is not None:
            k = kernels[dom]
            kname = KERNEL_OF_CLASS.get(dom, dom)
            roof = {"bound": k["bound"], "achieved": k["achieved"], "peak": k["peak"],
                    "unit": k["unit"], "frac": k["frac"],
                    "traffic": profiled_traffic(kname, a.workload) if k["bound"] == "hbm" else None,
                    "algorithmic_per_step": k["algorithmic"], "kernel_class": dom,
                    "kernel": f"{kname} ({dom}: CUDA events around each of its "
                              f"{k['records']} launches in 3 steps)",
                    "peak_source": k["peak_source"]}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "precision": "tf32x3", "data": "synthetic",
            "config": dict(workload_config(w, a.workload),
                           timed="CUDA-graph replay of the step" if use_graph else "eager step",
                           autotune=tuned),
            "eager": {"value": whole_job_rate(samples, world, ms_eager), "ms_per_step": ms_eager},
            "graph_replay": graph, "ms_fwd_calls": fwd_ms, "ms_bwd_calls": bwd_ms,
            "rel_err_vs_fp64": rel_err, "sequential": seq, "roofline": roof, "kernels": kernels,
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": int(launches),
            "gpu_launches_note": "library kernels per step (dfilt_launch_count); the loss "
                                 "gradient is one torch elementwise op",
            "configs": configs, "jvp": jvp, "state_space": ssl, "parameter_varying": tvl,
            "tensor_pipe": tensor_pipe(a.workload),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def tensor_pipe(workload):
    """The tensor-core tile passes' tensor-pipe activity on this workload, from the
    committed ncu summary (None when none matches the current sources)."""
    pct = profiled_tensor("hi_tc_kernel", workload)
    if pct is None:
        return None
    return {"kernel": "hi_tc_kernel (Y and U tile passes, every state bucket)",
            "active_pct_of_peak": pct,
            "source": "committed ncu summary: sm__pipe_tensor_cycles_active while active, "
                      "duration-weighted over the captured launches"}


def run_e2e(r, w, torch, stream, world, samples, barrier, maxrank):
    """The step end to end through the C ABI: every step copies its inputs in from pinned
    host memory (the signal and the loss target, or the upstream gradient) and its results
    out (every gradient), on three streams: inputs of step k+1, step k, results of step
    k-1; device buffers double-buffered; the timed region runs from before the first copy
    to after the last."""
    hx = torch.from_numpy(w.x).pin_memory()
    # the loss target travels as -scale * target (the form the step's loss gradient reads)
    htg = (r.neg_target.cpu() if r.target is not None else torch.from_numpy(w.gy)).pin_memory()
    ogx = torch.empty_like(hx).pin_memory()
    ogb, oga, ogz = (torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in (r.gb, r.ga, r.gz))
    h2d = (hx.numel() + htg.numel()) * 4
    d2h = sum(t.numel() * 4 for t in (ogx, ogb, oga, ogz))
    sets = []
    for _ in range(2):
        din = {"x": torch.empty_like(r.x), "tg": torch.empty_like(r.x)}
        dout = {"y": torch.empty_like(r.x), "gy": torch.empty_like(r.x), "gx": torch.empty_like(r.x),
                "gb": torch.empty_like(r.gb), "ga": torch.empty_like(r.ga), "gz": torch.zeros_like(r.gz)}
        sets.append((din, dout))
    s_in, s_cp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    cp_ptr = ctypes.c_void_p(s_cp.cuda_stream)
    ev = lambda: torch.cuda.Event()
    in_done, cp_done, out_done = [ev(), ev()], [ev(), ev()], [ev(), ev()]

    def e2e_step(k):
        j = k % 2
        din, dout = sets[j]
        with torch.cuda.stream(s_in):
            if k >= 2:
                s_in.wait_event(cp_done[j])
            din["x"].copy_(hx, non_blocking=True)
            din["tg"].copy_(htg, non_blocking=True)
            in_done[j].record(s_in)
        s_cp.wait_event(in_done[j])
        if k >= 2:
            s_cp.wait_event(out_done[j])
        with torch.cuda.stream(s_cp):
            outs = (dout["gx"], dout["gb"], dout["ga"], dout["gz"])
            if r.target is not None:
                r.train_step(cp_ptr, x=din["x"], y=dout["y"], gy=dout["gy"], neg_target=din["tg"],
                             out=outs)
            else:
                r.fwd(cp_ptr, x=din["x"], y=dout["y"])
                r.bwd(cp_ptr, gy=din["tg"], x=din["x"], y=dout["y"], out=outs)
        cp_done[j].record(s_cp)
        with torch.cuda.stream(s_out):
            s_out.wait_event(cp_done[j])
            for h_, nm in ((ogx, "gx"), (ogb, "gb"), (oga, "ga"), (ogz, "gz")):
                h_.copy_(dout[nm], non_blocking=True)
            out_done[j].record(s_out)

    def e2e_run(n):
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for s_ in (s_in, s_cp, s_out):
            s_.wait_event(start)
        for k in range(n):
            e2e_step(k)
        for s_ in (s_in, s_cp, s_out):
            stream.wait_stream(s_)
        stop.record(stream)
        torch.cuda.synchronize()
        return start.elapsed_time(stop)

    e2e_run(2)
    barrier()
    k = 6
    ems = maxrank(e2e_run(k) / k)
    last = sets[(k - 1) % 2][1]["gx"].reshape(-1)[:4096]
    ok = bool(torch.equal(ogx.reshape(-1)[:4096].cuda(), last))
    return {"value": whole_job_rate(samples, world, ems), "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": ems,
            "pipelined": "h2d(k+1) | step(k) | d2h(k-1) on three streams",
            "host_result_matches_device": ok}


def run_jvp(torch, dfilt, stream, a, world, barrier, maxrank, hbm, src):
    """Forward mode on the biquad workload (1024 x 48000), tangents of every input: the
    input step (v from x, dx, y and the coefficient tangents) then the library's forward
    with numerator [1] on v.  The forward step alone is timed on the same data, so the
    input step's time is the difference."""
    from paper_2511_14390_gb300 import inputs
    w = inputs.make("biquad_1024x48000")
    B, T, N, M = w.B, w.x.shape[1], w.N, w.M
    dev = lambda arr: torch.from_numpy(np.ascontiguousarray(arr)).cuda()
    x, b, av, zi = dev(w.x), dev(w.b), dev(w.a), dev(w.zi)
    o = dfilt.make_opts(algo="chunked")
    L = dfilt.lib()
    P = dfilt._ptr
    sptr = ctypes.c_void_p(stream.cuda_stream)
    y, _ = dfilt.dfilt_forward(x, b, av, zi, opts=o, want_saved=False)
    rng = np.random.default_rng(7)
    tdx = dev(rng.standard_normal((B, T), dtype=np.float32))
    tdb = dev((0.1 * rng.standard_normal(w.b.shape)).astype(np.float32))
    tda = dev((0.1 * rng.standard_normal(w.a.shape)).astype(np.float32))
    tdz = dev(rng.standard_normal(w.a.shape).astype(np.float32))
    nws = dfilt.dfilt_jvp_workspace_size(B, T, N, M, o)
    jws = torch.empty(nws, dtype=torch.uint8, device="cuda")
    dyj = torch.empty_like(x)
    fws1 = dfilt.dfilt_workspace_size(B, T, 0, M, o)[0]
    w1 = torch.empty(max(fws1, 16), dtype=torch.uint8, device="cuda")
    ones = torch.ones((B, 1), dtype=torch.float32, device="cuda")
    vview = jws[: B * T * 4].view(torch.float32)
    dy1 = torch.empty_like(x)

    def jvp_call():
        dfilt._check(L.dfilt_jvp(P(x), P(y), P(b), P(av), P(tdx), P(tdb), P(tda), P(tdz), P(dyj),
                                 P(jws), nws, B, T, N, M, ctypes.byref(o), sptr), "dfilt_jvp")

    def fwd1_call():
        dfilt._check(L.dfilt_forward(P(vview), P(ones), P(av), P(tdz), P(dy1), None, P(w1), fws1,
                                     B, T, 0, M, ctypes.byref(o), sptr), "dfilt_forward")

    nj = max(3, min(200, a.steps * 5))
    ms_j = maxrank(time_loop(torch, stream, jvp_call, nj, 3, barrier))
    ms_f1 = maxrank(time_loop(torch, stream, fwd1_call, nj, 3, barrier))
    jvp_call()
    status = dfilt.dfilt_sync_status()
    if status != 0:
        raise RuntimeError(f"device status {dfilt.STATUS[status]}")
    ms_in = ms_j - ms_f1
    out = {"workload": "biquad_1024x48000, tangents of x, b, a, zi",
           "value": B * T * world / (ms_j / 1e3) / 1e9, "unit": UNIT, "ms_per_call": ms_j,
           "calls": nj, "ms_forward_step": ms_f1, "ms_input_step": ms_in,
           "input_step_roofline": {
               "bound": "hbm", "unit": "GB/s", "peak": hbm,
               "achieved": 16.0 * B * T / (ms_in / 1e3) / 1e9 if ms_in > 0 else None,
               "frac": (16.0 * B * T / (ms_in / 1e3) / 1e9 / hbm) if ms_in > 0 else None,
               "algorithmic_bytes": 16.0 * B * T,
               "kernel": "jvp_input_vec4_kernel<2> (x, dx, y read, v written; time = call - "
                         "forward step)", "peak_source": src}}
    import oracle
    idx = np.linspace(0, B - 1, 8).astype(int)
    tg = [t.cpu().numpy()[idx] for t in (tdx, tdb, tda, tdz)]
    _, dref = oracle.jvp(w.x[idx], w.b[idx], w.a[idx], w.zi[idx], *tg)
    got = dyj.cpu().numpy()[idx].astype(np.float64)
    out["rel_err_vs_fp64"] = float((np.abs(got - dref).max(-1) / np.abs(dref).max(-1)).max())
    del jws, w1, dy1, dyj, tdx
    return out


def run_tv(torch, dfilt, stream, a, world, barrier, maxrank, hbm, src):
    """Parameter-varying biquads (coefficients per output sample, poles and zeros moving
    slowly), 1024 x 48000, forward + backward (grad_x, per-sample grad_b and grad_a,
    grad_ypast).  Algorithmic bytes per sample: forward x, b (3), a (2) read, y written
    (28); backward gy, x, y, b, a read, grad_x, grad_b, grad_a written (56)."""
    B, T, N, M = 1024, 48000, 2, 2
    rng = np.random.default_rng(21)
    n = np.arange(T)[None, :]
    r0, th0 = rng.uniform(0.5, 0.95, (B, 1)), rng.uniform(0.1, 3.0, (B, 1))
    r = r0 * (1 - 0.04 * (1 + np.sin(rng.uniform(1e-3, 2e-2, (B, 1)) * n)))
    th = th0 + 0.2 * np.sin(rng.uniform(1e-3, 2e-2, (B, 1)) * n)
    av = np.stack([-2 * r * np.cos(th), r * r], axis=2).astype(np.float32)
    bv = (rng.standard_normal((B, 1, N + 1)) * (1 + 0.1 * np.sin(0.003 * n))[:, :, None]).astype(np.float32)
    dev = lambda arr: torch.from_numpy(np.ascontiguousarray(arr)).cuda()
    ad, bd = dev(av), dev(bv)
    xd = torch.randn((B, T), device="cuda", generator=torch.Generator("cuda").manual_seed(22))
    gyd = torch.randn((B, T), device="cuda", generator=torch.Generator("cuda").manual_seed(23))
    ypd = dev((0.1 * rng.standard_normal((B, M))).astype(np.float32))
    nws = dfilt.dfilt_tv_workspace_size(B, T, N, M)
    w1 = torch.empty(max(nws, 16), dtype=torch.uint8, device="cuda")
    w2 = torch.empty(max(nws, 16), dtype=torch.uint8, device="cuda")
    yd, gxd = torch.empty_like(xd), torch.empty_like(xd)
    gbd, gad, gypd = torch.empty_like(bd), torch.empty_like(ad), torch.empty_like(ypd)
    L = dfilt.lib()
    P = dfilt._ptr
    sptr = ctypes.c_void_p(stream.cuda_stream)

    def tv_step():
        dfilt._check(L.dfilt_tv_forward(P(xd), P(bd), P(ad), P(ypd), P(yd), P(w1), nws, B, T, N, M,
                                        sptr), "dfilt_tv_forward")
        dfilt._check(L.dfilt_tv_backward(P(gyd), P(xd), P(yd), P(bd), P(ad), P(ypd), P(gxd), P(gbd),
                                         P(gad), P(gypd), P(w2), nws, B, T, N, M, sptr),
                     "dfilt_tv_backward")

    ns = max(3, min(100, a.steps * 5))
    ms = maxrank(time_loop(torch, stream, tv_step, ns, 3, barrier))
    status = dfilt.dfilt_sync_status()
    if status != 0:
        raise RuntimeError(f"device status {dfilt.STATUS[status]}")
    import oracle
    k = 4096
    hx, hy = xd[:2, :k].double().cpu().numpy(), yd[:2, :k].double().cpu().numpy()
    ref = oracle.forward_tv(hx, bv[:2, :k].astype(np.float64), av[:2, :k].astype(np.float64),
                            ypd[:2].double().cpu().numpy())
    out = {"workload": f"parameter-varying biquads, {B} x {T}, fwd + bwd", "value": B * T * world / (ms / 1e3) / 1e9,
           "unit": "Gsamples/s", "ms_per_step": ms, "calls": ns,
           "algorithmic_bytes": 84.0 * B * T,
           "roofline_frac": 84.0 * B * T / (ms / 1e3) / 1e9 / hbm, "peak": hbm, "peak_source": src,
           "rel_err_vs_fp64_first_4096_samples": float((np.abs(hy - ref).max(1) / np.abs(ref).max(1)).max())}
    del xd, gyd, yd, gxd, gbd, gad, w1, w2, ad, bd
    torch.cuda.empty_cache()
    return out


def run_ss(torch, dfilt, stream, a, world, barrier, maxrank, hbm, src):
    """The App. B recurrence v(n+1) = A v(n) + z(n) with a dense 2 x 2 A (the operator the
    paper benchmarks), batched: 64 channels x 2^20 steps, forward + backward (grad_A,
    grad_v0, grad_z).  Algorithmic bytes per step: forward z read + v written (16),
    backward gv and v read + gz written (24)."""
    Bs, Ts, Ms = 64, 1 << 20, 2
    rng = np.random.default_rng(11)
    As = rng.standard_normal((Bs, Ms, Ms))
    for i in range(Bs):
        As[i] *= 0.95 / max(abs(np.linalg.eigvals(As[i])))
    dev = lambda arr: torch.from_numpy(np.ascontiguousarray(arr)).cuda()
    Ad = dev(As.astype(np.float32))
    v0d = dev(rng.standard_normal((Bs, Ms)).astype(np.float32))
    zd = torch.randn((Bs, Ts, Ms), device="cuda", generator=torch.Generator("cuda").manual_seed(12))
    gvd = torch.randn((Bs, Ts, Ms), device="cuda", generator=torch.Generator("cuda").manual_seed(13))
    sfw, sbw = dfilt.dfilt_ss_workspace_size(Bs, Ts, Ms)
    sw1 = torch.empty(max(sfw, 16), dtype=torch.uint8, device="cuda")
    sw2 = torch.empty(max(sbw, 16), dtype=torch.uint8, device="cuda")
    vd, gzd = torch.empty_like(zd), torch.empty_like(zd)
    gAd, gv0d = torch.empty_like(Ad), torch.empty_like(v0d)
    L = dfilt.lib()
    P = dfilt._ptr
    sptr = ctypes.c_void_p(stream.cuda_stream)

    def ss_step():
        dfilt._check(L.dfilt_ss_forward(P(Ad), P(v0d), P(zd), P(vd), P(sw1), sfw, Bs, Ts, Ms, sptr),
                     "dfilt_ss_forward")
        dfilt._check(L.dfilt_ss_backward(P(Ad), P(v0d), P(vd), P(gvd), P(gAd), P(gv0d), P(gzd),
                                         P(sw2), sbw, Bs, Ts, Ms, sptr), "dfilt_ss_backward")

    ns = max(3, min(100, a.steps * 5))
    sms_ = maxrank(time_loop(torch, stream, ss_step, ns, 3, barrier))
    status = dfilt.dfilt_sync_status()
    if status != 0:
        raise RuntimeError(f"device status {dfilt.STATUS[status]}")
    out = {"workload": f"dense A (M = {Ms}), {Bs} channels x {Ts} steps, fwd + bwd",
           "value": Bs * Ts * world / (sms_ / 1e3) / 1e9, "unit": "Gsteps/s", "ms_per_step": sms_,
           "calls": ns, "algorithmic_bytes": 40.0 * Bs * Ts,
           "roofline_frac": 40.0 * Bs * Ts / (sms_ / 1e3) / 1e9 / hbm, "peak": hbm,
           "peak_source": src}
    from oracle import statespace as ossm
    hv = vd[0, :4096].double().cpu().numpy()
    ref = ossm.recurrence_forward(As[0].astype(np.float32).astype(np.float64),
                                  v0d[0].double().cpu().numpy(), zd[0, :4096].double().cpu().numpy())
    out["rel_err_vs_fp64_first_4096_steps"] = float(np.abs(hv - ref).max() / np.abs(ref).max())

    # the same operator diagonalised (Diag-EXT): the eigendecomposition of each A (numpy's
    # eig on the host, once, like the parameters), the scan in the eigenbasis
    A32 = As.astype(np.float32).astype(np.float64)
    lam = np.zeros((Bs, Ms), np.complex64)
    Vm = np.zeros((Bs, Ms, Ms), np.complex64)
    Vi = np.zeros((Bs, Ms, Ms), np.complex64)
    for i in range(Bs):
        w_, vec = np.linalg.eig(A32[i])
        lam[i], Vm[i], Vi[i] = w_, vec, np.linalg.inv(vec)
    ld, Vd, Vid = dev(lam), dev(Vm), dev(Vi)
    dfw, dbw = dfilt.dfilt_diag_workspace_size(Bs, Ts, Ms)
    dw1 = torch.empty(max(dfw, 16), dtype=torch.uint8, device="cuda")
    dw2 = torch.empty(max(dbw, 16), dtype=torch.uint8, device="cuda")

    def diag_step():
        dfilt._check(L.dfilt_diag_forward(P(ld), P(Vd), P(Vid), P(v0d), P(zd), P(vd), P(dw1), dfw,
                                          Bs, Ts, Ms, sptr), "dfilt_diag_forward")
        dfilt._check(L.dfilt_diag_backward(P(ld), P(Vd), P(Vid), P(v0d), P(vd), P(gvd), P(gAd),
                                           P(gv0d), P(gzd), P(dw2), dbw, Bs, Ts, Ms, sptr),
                     "dfilt_diag_backward")

    dms = maxrank(time_loop(torch, stream, diag_step, ns, 3, barrier))
    status = dfilt.dfilt_sync_status()
    if status != 0:
        raise RuntimeError(f"device status {dfilt.STATUS[status]}")
    hv = vd[0, :4096].double().cpu().numpy()
    dref = ossm.diag_forward(lam[0].astype(np.complex128), Vm[0].astype(np.complex128),
                             Vi[0].astype(np.complex128), v0d[0].double().cpu().numpy(),
                             zd[0, :4096].double().cpu().numpy())
    out["diagonalised"] = {
        "workload": f"A = V diag(lam) V^-1 (M = {Ms}), the same {Bs} x {Ts} problem, fwd + bwd",
        "value": Bs * Ts * world / (dms / 1e3) / 1e9, "unit": "Gsteps/s", "ms_per_step": dms,
        "calls": ns, "roofline_frac": 40.0 * Bs * Ts / (dms / 1e3) / 1e9 / hbm,
        "rel_err_vs_fp64_first_4096_steps": float(np.abs(hv - dref).max() / np.abs(dref).max())}
    del zd, gvd, vd, gzd, sw1, sw2, dw1, dw2
    return out


if __name__ == "__main__":
    main()
