#!/usr/bin/env python
"""Benchmark: forward + backward throughput (Gsamples/s) of batched direct-form IIR
filters on GB300, chunked tensor-core path vs the sequential kernel, at a stated
relative error against the FP64 oracle.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = coefficient setup + forward + backward (all gradients) over one batch of
the workload (default: 1024 biquad channels x 48000 samples).  Under torchrun every
rank filters its own copy of the batch (channels are independent problems, no
collective on the data path): weak scaling.  Rank 0 prints one JSON line.
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


def args_():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="biquad_1024x48000")
    p.add_argument("--algo", default="chunked", choices=["chunked", "sequential"])
    p.add_argument("--no-seq", action="store_true", help="skip the sequential-kernel leg")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-jvp", action="store_true", help="skip the forward-mode (JVP) leg")
    p.add_argument("--no-ss", action="store_true",
                   help="skip the dense state-space recurrence leg (M = 2, 64 x 2^20 steps)")
    p.add_argument("--graph", action="store_true",
                   help="also time the step captured in a CUDA graph (launch-bound workloads)")
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
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
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
                "samples": len(sm)}


def gpu_uuid(torch):
    try:
        u = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(torch.cuda.current_device())


# ----------------------------------------------------------------------------
# CPU baseline: the FP64 oracle as it stands, on the host cores
# ----------------------------------------------------------------------------

def cpu_oracle_rate(w, budget_s=3.0):
    import oracle
    total, t0, reps = 0, time.perf_counter(), 0
    while True:
        y = oracle.forward(w.x, w.b, w.a, w.zi)
        oracle.backward(w.gy, w.x, y, w.b, w.a)
        total += w.x.size
        reps += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": total / dt / 1e9, "unit": UNIT, "cores": oracle.max_threads(),
            "kind": "oracle",
            "sample": f"the whole workload ({w.B} x {w.x.shape[1]}), FP64 forward + backward "
                      f"(all gradients), repeated {reps}x over {dt:.1f} s"}


def run_reference(a, world, rank):
    from paper_2511_14390_gb300 import inputs
    import oracle
    if rank != 0:
        return
    w = inputs.make(a.workload)
    # each step filters a bounded sample of the workload's channels, sized from one
    # timed whole-workload pass so that warm-up + timed steps take about two minutes
    t0 = time.perf_counter()
    oracle.backward(w.gy, w.x, oracle.forward(w.x, w.b, w.a, w.zi), w.b, w.a)
    t_full = time.perf_counter() - t0
    nb = int(w.B * min(1.0, 120.0 / max(1, a.steps + a.warmup) / max(t_full, 1e-9)))
    nb = max(1, min(w.B, nb))
    xs, gs, bs, as_ = w.x[:nb], w.gy[:nb], w.b[:nb], w.a[:nb]
    zs = None if w.zi is None else w.zi[:nb]
    step = lambda: oracle.backward(gs, xs, oracle.forward(xs, bs, as_, zs), bs, as_)
    for _ in range(a.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        step()
    dt = (time.perf_counter() - t0) / a.steps
    v = xs.size / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w, a.workload, "oracle"),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.max_threads(),
                             "kind": "oracle",
                             "sample": f"{nb} of the workload's {w.B} channels x {w.x.shape[1]} "
                                       f"samples per step (sized for a ~2 min run)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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


def kernel_name(direction, M):
    """Main kernel of the chunked path for a state bucket (the warp-specialised kernels
    serve the buckets whose layouts fit; see the dispatch in csrc/chunk_*.cu)."""
    mb = next(v for v in (2, 4, 8, 16, 32, 64) if M <= v)
    f64 = 1 if M > 2 else 0
    if direction == "forward":
        if mb >= 32:
            return f"chunk_fwd_kernel<{mb}, {f64}>"
        stages = 2 if mb == 16 else 3   # signal stages that fit shared memory
        return f"chunk_fwd_ws_kernel<{mb}, {f64}, {stages}>"
    return f"chunk_bwd_ws_kernel<{mb}, {f64}>" if mb <= 8 else f"chunk_bwd_kernel<{mb}, {f64}, 0>"


def profiled_traffic(kname, workload):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of `kname`
    from the committed ncu summary of this workload, scaled to one full launch; None
    when there is no summary or the kernel source changed since it was captured."""
    import glob
    import hashlib
    import re
    base = kname.split("<")[0]
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", f"{base}_*.md"))):
        txt = open(path).read()
        m = re.search(r"<!-- traffic kernel=(\S+) workload=(\S+) bytes_per_launch=([0-9.e+]+) "
                      r"sources=(\S+) sha256=([0-9a-f]+) -->", txt)
        if not m or m.group(1) != kname.replace(" ", "") or m.group(2) != workload:
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


def workload_config(w, name, algo):
    return {"workload": name, "B": int(w.B), "T": int(w.x.shape[1]), "M": int(w.M),
            "N": int(w.N), "algo": algo,
            "l2": "inputs larger than L2: x and gy are %.0f MB each, 129 MB L2" % (w.x.nbytes / 1e6)}


# ----------------------------------------------------------------------------
# GPU legs
# ----------------------------------------------------------------------------

def main():
    a = args_()
    world, rank, local = dist_env()
    if a.impl == "reference":
        run_reference(a, world, rank)
        return
    import torch
    import torch.distributed as dist
    from paper_2511_14390_gb300 import dfilt, inputs

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = inputs.make(a.workload, **({"B": a.channels} if a.channels > 0 else {}))
    B, T = w.x.shape
    N, M = w.N, w.M
    if w.zi is None:   # zero initial conditions, passed explicitly so grad_zi has a buffer
        w.zi = np.zeros((B, M), dtype=np.float32)
    dev = lambda arr: torch.from_numpy(np.ascontiguousarray(arr)).cuda()
    x, b, av, zi, gy = dev(w.x), dev(w.b), dev(w.a), dev(w.zi), dev(w.gy)
    L = dfilt.lib()
    stream = torch.cuda.current_stream()
    sptr = ctypes.c_void_p(stream.cuda_stream)

    def setup(algo):
        o = dfilt.make_opts(algo=algo, precision="tf32x3")
        fws, sv, bws = dfilt.dfilt_workspace_size(B, T, N, M, o)
        buf = lambda n: torch.empty(max(n, 16), dtype=torch.uint8, device="cuda")
        st = {"o": o, "fws": fws, "bws": bws, "y": torch.empty_like(x),
              "saved": buf(sv) if sv else None, "wf": buf(fws), "wb": buf(bws),
              "gx": torch.empty_like(x), "gb": torch.empty_like(b), "ga": torch.empty_like(av),
              "gz": torch.empty_like(zi)}
        return st

    P = dfilt._ptr

    def fwd(st, sp=None):
        dfilt._check(L.dfilt_forward(P(x), P(b), P(av), P(zi), P(st["y"]), P(st["saved"]),
                                     P(st["wf"]), st["fws"], B, T, N, M, ctypes.byref(st["o"]),
                                     sp or sptr), "dfilt_forward")

    def bwd(st, sp=None):
        yarg = None if st["saved"] is not None else st["y"]
        dfilt._check(L.dfilt_backward(P(gy), P(x), P(yarg), P(b), P(av), P(zi), P(st["saved"]),
                                      P(st["gx"]), P(st["gb"]), P(st["ga"]), P(st["gz"]),
                                      P(st["wb"]), st["bws"], B, T, N, M, ctypes.byref(st["o"]),
                                      sp or sptr), "dfilt_backward")

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(st, steps, warmup, kernel_timing=False):
        for _ in range(warmup):
            fwd(st)
            bwd(st)
        torch.cuda.synchronize()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
        barrier()
        torch.cuda.synchronize()
        if kernel_timing:   # event pairs around each call's main kernel, on this stream
            dfilt.dfilt_kernel_timing(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(steps):
            ev[k][0].record(stream)
            fwd(st)
            ev[k][1].record(stream)
            bwd(st)
            ev[k][2].record(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        kern = None
        if kernel_timing:
            (fm, fn), (bm, bn) = dfilt.dfilt_kernel_timing_read()
            dfilt.dfilt_kernel_timing(False)
            kern = (fm / max(fn, 1), bm / max(bn, 1), fn, bn)
        tot = e0.elapsed_time(e1)
        tf = [e[0].elapsed_time(e[1]) for e in ev]
        tb = [e[1].elapsed_time(e[2]) for e in ev]
        return tot / steps, statistics.mean(tf), statistics.mean(tb), kern

    def maxrank(v):
        return max_over_ranks(v, world)

    algo = a.algo
    st = setup(algo)
    clk = Clocks(gpu_uuid(torch))
    ms, ms_f, ms_b, kern = timed(st, a.steps, a.warmup, kernel_timing=True)
    clocks = clk.stop()
    ms = maxrank(ms)
    samples_all = B * T * world

    # the same step captured once in a CUDA graph and replayed (removes launch gaps)
    graph = None
    if a.graph:
        gs = torch.cuda.Stream()
        gptr = ctypes.c_void_p(gs.cuda_stream)
        gs.wait_stream(stream)
        with torch.cuda.stream(gs):
            for _ in range(3):
                fwd(st, gptr)
                bwd(st, gptr)
        torch.cuda.synchronize()
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg, stream=gs):
            fwd(st, gptr)
            bwd(st, gptr)
        for _ in range(a.warmup):
            cg.replay()
        torch.cuda.synchronize()
        barrier()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(a.steps):
            cg.replay()
        g1.record(stream)
        torch.cuda.synchronize()
        barrier()
        gms = maxrank(g0.elapsed_time(g1) / a.steps)
        graph = {"value": samples_all / (gms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": gms,
                 "steps": a.steps}
        del cg
    value = whole_job_rate(B * T, world, ms)
    status = dfilt.dfilt_sync_status()
    if status != 0:
        raise RuntimeError(f"device status {dfilt.STATUS[status]}")

    # accuracy of this run's outputs against the FP64 oracle on sampled channels
    rel_err = None
    if rank == 0:
        import oracle
        idx = np.unique(np.linspace(0, B - 1, 32).astype(int))
        sub = inputs.Workload(x=w.x[idx], b=w.b[idx], a=w.a[idx], zi=w.zi[idx], gy=w.gy[idx],
                              M=M, N=N, radius=w.radius[idx])
        yr = oracle.forward(sub.x, sub.b, sub.a, sub.zi)
        gr = oracle.backward(sub.gy, sub.x, yr, sub.b, sub.a)
        rel = lambda g, r: (np.abs(g.cpu().numpy()[idx].astype(np.float64) - r).max(-1)
                            / np.abs(r).max(-1))
        per = {"y": rel(st["y"], yr), "grad_x": rel(st["gx"], gr[0]),
               "grad_b": rel(st["gb"], gr[1]), "grad_a": rel(st["ga"], gr[2]),
               "grad_zi": rel(st["gz"], gr[3])}
        rel_err = {k: float(v.max()) for k, v in per.items()}
        rel_err.update({"channels_checked": len(idx),
                        "metric": "per-channel max|err| / max|ref|, max over checked channels",
                        "by_pole_radius": radius_bins(per, w.radius[idx])})

    # sequential-kernel leg (the baseline the chunked form is compared with)
    seq = None
    if not a.no_seq and algo == "chunked":
        sst = setup("sequential")
        sms, sf, sb, _ = timed(sst, max(3, min(50, a.steps // 4)), 3)
        sms = maxrank(sms)
        seq = {"value": samples_all / (sms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": sms,
               "ms_fwd": sf, "ms_bwd": sb}
        del sst

    # Forward mode (Jacobian-vector product) on the same workload, tangents of every
    # input: the call runs the input step (v from x, dx, y and the coefficient tangents)
    # and then the library's forward with numerator [1] on v.  The forward step alone is
    # timed on the same data, so the input step's time is the difference.
    jvp = None
    if not a.no_jvp and algo == "chunked":
        o = st["o"]
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
            dfilt._check(L.dfilt_jvp(P(x), P(st["y"]), P(b), P(av), P(tdx), P(tdb), P(tda),
                                     P(tdz), P(dyj), P(jws), nws, B, T, N, M, ctypes.byref(o),
                                     sptr), "dfilt_jvp")

        def fwd1_call():
            dfilt._check(L.dfilt_forward(P(vview), P(ones), P(av), P(tdz), P(dy1), None, P(w1),
                                         fws1, B, T, 0, M, ctypes.byref(o), sptr), "dfilt_forward")

        def time_calls(fn, n):
            for _ in range(max(3, a.warmup)):
                fn()
            torch.cuda.synchronize()
            barrier()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for _ in range(n):
                fn()
            t1.record(stream)
            torch.cuda.synchronize()
            barrier()
            return maxrank(t0.elapsed_time(t1) / n)

        nj = max(3, min(200, a.steps))
        ms_j = time_calls(jvp_call, nj)
        ms_f1 = time_calls(fwd1_call, nj)
        jvp_call()          # dyj of the tangents, for the accuracy check below
        status = dfilt.dfilt_sync_status()
        if status != 0:
            raise RuntimeError(f"device status {dfilt.STATUS[status]}")
        hbm_j, src_j = peaks()
        ms_in = ms_j - ms_f1
        jvp = {"value": samples_all / (ms_j / 1e3) / 1e9, "unit": UNIT, "ms_per_call": ms_j,
               "calls": nj, "ms_forward_step": ms_f1, "ms_input_step": ms_in,
               "input_step_roofline": {
                   "bound": "hbm", "unit": "GB/s", "peak": hbm_j,
                   "achieved": 16.0 * B * T / (ms_in / 1e3) / 1e9 if ms_in > 0 else None,
                   "frac": (16.0 * B * T / (ms_in / 1e3) / 1e9 / hbm_j) if ms_in > 0 else None,
                   "algorithmic_bytes": 16.0 * B * T,
                   "kernel": (f"jvp_input_vec4_kernel<{max(N, M)}>" if max(N, M) <= 4
                              and T % 4 == 0 else "jvp_input_kernel")
                             + " (x, dx, y read, v written; time = call - forward step)",
                   "peak_source": src_j},
               "call_roofline_frac": 16.0 * B * T / (ms_j / 1e3) / 1e9 / hbm_j,
               "gpu_launches_per_call": 3}
        if rank == 0:
            import oracle
            idx = np.linspace(0, B - 1, 8).astype(int)
            tg = [t.cpu().numpy()[idx] for t in (tdx, tdb, tda, tdz)]
            _, dref = oracle.jvp(w.x[idx], w.b[idx], w.a[idx], w.zi[idx], *tg)
            got = dyj.cpu().numpy()[idx].astype(np.float64)
            jvp["rel_err_vs_fp64"] = float((np.abs(got - dref).max(-1)
                                            / np.abs(dref).max(-1)).max())
            if world == 1 and not a.no_cpu:
                sub = max(1, min(B, 64))
                t0, reps = time.perf_counter(), 0
                tgs = [t.cpu().numpy()[:sub] for t in (tdx, tdb, tda, tdz)]
                while time.perf_counter() - t0 < 2.0 or reps == 0:
                    oracle.jvp(w.x[:sub], w.b[:sub], w.a[:sub], w.zi[:sub], *tgs)
                    reps += 1
                dt = time.perf_counter() - t0
                jvp["cpu_baseline"] = {"value": sub * T * reps / dt / 1e9, "unit": UNIT,
                                       "cores": oracle.max_threads(), "kind": "oracle",
                                       "sample": f"{sub} of the {B} channels, FP64 JVP, "
                                                 f"repeated {reps}x over {dt:.1f} s"}
        del jws, w1, dy1, dyj, tdx

    # The App. B recurrence v(n+1) = A v(n) + z(n) with a dense 2 x 2 A (the operator the
    # paper benchmarks), batched: 64 channels x 2^20 steps, forward + backward (grad_A,
    # grad_v0, grad_z).  Algorithmic bytes per step: forward z read + v written (16),
    # backward gv and v read + gz written (24).
    ssl = None
    if not a.no_ss:
        Bs, Ts, Ms = 64, 1 << 20, 2
        rng = np.random.default_rng(11)
        As = rng.standard_normal((Bs, Ms, Ms))
        for i in range(Bs):
            As[i] *= 0.95 / max(abs(np.linalg.eigvals(As[i])))
        Ad = dev(As.astype(np.float32))
        v0d = dev(rng.standard_normal((Bs, Ms)).astype(np.float32))
        zd = torch.randn((Bs, Ts, Ms), device="cuda", generator=torch.Generator("cuda").manual_seed(12))
        gvd = torch.randn((Bs, Ts, Ms), device="cuda", generator=torch.Generator("cuda").manual_seed(13))
        sfw, sbw = dfilt.dfilt_ss_workspace_size(Bs, Ts, Ms)
        sw1 = torch.empty(max(sfw, 16), dtype=torch.uint8, device="cuda")
        sw2 = torch.empty(max(sbw, 16), dtype=torch.uint8, device="cuda")
        vd, gzd = torch.empty_like(zd), torch.empty_like(zd)
        gAd, gv0d = torch.empty_like(Ad), torch.empty_like(v0d)

        def ss_step():
            dfilt._check(L.dfilt_ss_forward(P(Ad), P(v0d), P(zd), P(vd), P(sw1), sfw, Bs, Ts, Ms,
                                            sptr), "dfilt_ss_forward")
            dfilt._check(L.dfilt_ss_backward(P(Ad), P(v0d), P(vd), P(gvd), P(gAd), P(gv0d),
                                             P(gzd), P(sw2), sbw, Bs, Ts, Ms, sptr),
                         "dfilt_ss_backward")

        for _ in range(max(3, a.warmup)):
            ss_step()
        torch.cuda.synchronize()
        barrier()
        ns = max(3, min(100, a.steps))
        s0, s1, s2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        s0.record(stream)
        for _ in range(ns):
            ss_step()
        s1.record(stream)
        torch.cuda.synchronize()
        barrier()
        sms_ = maxrank(s0.elapsed_time(s1) / ns)
        status = dfilt.dfilt_sync_status()
        if status != 0:
            raise RuntimeError(f"device status {dfilt.STATUS[status]}")
        hbm_s, src_s = peaks()
        steps_all = Bs * Ts * world
        ssl = {"workload": f"dense A (M = {Ms}), {Bs} channels x {Ts} steps, fwd + bwd",
               "value": steps_all / (sms_ / 1e3) / 1e9, "unit": "Gsteps/s", "ms_per_step": sms_,
               "calls": ns, "algorithmic_bytes": 40.0 * Bs * Ts,
               "roofline_frac": 40.0 * Bs * Ts / (sms_ / 1e3) / 1e9 / hbm_s,
               "peak": hbm_s, "peak_source": src_s,
               # forward: powers, pass 1, carry, pass 2; backward: the same four on A^T
               # plus the dL/dA partials and their final sum
               "gpu_launches_per_step": 10}
        if rank == 0:
            from oracle import statespace as ossm
            hv = vd[0, :4096].double().cpu().numpy()
            ref = ossm.recurrence_forward(As[0].astype(np.float32).astype(np.float64),
                                          v0d[0].double().cpu().numpy(),
                                          zd[0, :4096].double().cpu().numpy())
            ssl["rel_err_vs_fp64_first_4096_steps"] = float(np.abs(hv - ref).max()
                                                           / np.abs(ref).max())
            if world == 1 and not a.no_cpu:
                zc, gc = zd[0].double().cpu().numpy(), gvd[0].double().cpu().numpy()
                A0 = As[0].astype(np.float32).astype(np.float64)
                t0, reps, nst = time.perf_counter(), 0, 1 << 16
                while time.perf_counter() - t0 < 2.0 or reps == 0:
                    vv = ossm.recurrence_forward(A0, np.zeros(2), zc[:nst])
                    ossm.recurrence_backward(A0, np.zeros(2), vv, gc[:nst])
                    reps += 1
                dt = time.perf_counter() - t0
                ssl["cpu_baseline"] = {"value": nst * reps / dt / 1e9, "unit": "Gsteps/s",
                                       "cores": 1, "kind": "oracle",
                                       "sample": f"{nst} steps of one channel, FP64 numpy "
                                                 f"operator fwd + bwd, repeated {reps}x "
                                                 f"over {dt:.1f} s"}
        del zd, gvd, vd, gzd, sw1, sw2

    # End to end through the public API from pinned host buffers, pipelined across steps
    # the way a streaming caller would run it: step k's inputs are copied host -> device
    # on one stream while step k-1 computes and step k-2's results are copied back on a
    # third (device inputs and outputs double-buffered; every step's copies lie inside
    # the timed region, which runs from before the first copy to after the last one).
    e2e = None
    if not a.no_e2e:
        hx = torch.from_numpy(w.x).pin_memory()
        hgy = torch.from_numpy(w.gy).pin_memory()
        hb, ha, hz = (torch.from_numpy(t).pin_memory() for t in (w.b, w.a, w.zi))
        oy = torch.empty_like(hx).pin_memory()
        ogx = torch.empty_like(hx).pin_memory()
        ogb, oga, ogz = (torch.empty_like(t).pin_memory() for t in (hb, ha, hz))
        h2d = sum(t.numel() * 4 for t in (hx, hgy, hb, ha, hz))
        d2h = sum(t.numel() * 4 for t in (oy, ogx, ogb, oga, ogz))
        sets = []
        for j in range(2):
            din = {"x": x if j == 0 else torch.empty_like(x), "gy": gy if j == 0 else torch.empty_like(gy),
                   "b": torch.empty_like(b), "a": torch.empty_like(av), "zi": torch.empty_like(zi)}
            dout = {"y": torch.empty_like(x), "gx": torch.empty_like(x), "gb": torch.empty_like(b),
                    "ga": torch.empty_like(av), "gz": torch.empty_like(zi)}
            sets.append((din, dout))
        s_in, s_cp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        cp_ptr = ctypes.c_void_p(s_cp.cuda_stream)
        ev = lambda: torch.cuda.Event()
        in_done, cp_done, out_done = [ev(), ev()], [ev(), ev()], [ev(), ev()]
        est = st   # workspaces and the saved buffer: used by the compute stream only

        def e2e_step(k):
            j = k % 2
            din, dout = sets[j]
            with torch.cuda.stream(s_in):            # inputs of step k
                if k >= 2:
                    s_in.wait_event(cp_done[j])      # step k-2 has finished reading set j
                for nm, h_ in (("x", hx), ("gy", hgy), ("b", hb), ("a", ha), ("zi", hz)):
                    din[nm].copy_(h_, non_blocking=True)
                in_done[j].record(s_in)
            s_cp.wait_event(in_done[j])
            if k >= 2:
                s_cp.wait_event(out_done[j])         # step k-2's results copied out of set j
            dfilt._check(L.dfilt_forward(P(din["x"]), P(din["b"]), P(din["a"]), P(din["zi"]),
                                         P(dout["y"]), P(est["saved"]), P(est["wf"]), est["fws"],
                                         B, T, N, M, ctypes.byref(est["o"]), cp_ptr), "dfilt_forward")
            yarg = None if est["saved"] is not None else dout["y"]
            dfilt._check(L.dfilt_backward(P(din["gy"]), P(din["x"]), P(yarg), P(din["b"]),
                                          P(din["a"]), P(din["zi"]), P(est["saved"]), P(dout["gx"]),
                                          P(dout["gb"]), P(dout["ga"]), P(dout["gz"]), P(est["wb"]),
                                          est["bws"], B, T, N, M, ctypes.byref(est["o"]), cp_ptr),
                         "dfilt_backward")
            cp_done[j].record(s_cp)
            with torch.cuda.stream(s_out):           # results of step k
                s_out.wait_event(cp_done[j])
                for h_, nm in ((oy, "y"), (ogx, "gx"), (ogb, "gb"), (oga, "ga"), (ogz, "gz")):
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

        e2e_run(3)
        barrier()
        k = max(3, min(50, a.steps // 4))
        ems = maxrank(e2e_run(k) / k)
        # the last step's results are on the host: check them against the device path
        ok = bool(torch.equal(ogx[:2].cuda(), sets[(k - 1) % 2][1]["gx"][:2]))
        e2e = {"value": samples_all / (ems / 1e3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": ems,
               "pipelined": "h2d(k+1) | compute(k) | d2h(k-1) on three streams",
               "host_result_matches_device": ok}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        cpu = cpu_oracle_rate(w)

    if rank == 0:
        hbm, src = peaks()
        # algorithmic bytes per sample: forward reads x, writes y; backward reads gy and
        # x, writes grad_x (y is recomputed from M floats of chunk state per 64 samples)
        # (the sequential kernel re-reads y in the backward)
        if algo == "chunked":
            bytes_f = (8.0 + (4.0 * M / 64.0)) * B * T
            bytes_b = (12.0 + (4.0 * M / 64.0)) * B * T
        else:
            bytes_f, bytes_b = 8.0 * B * T, 16.0 * B * T
        kf, kb, kfn, kbn = kern
        dom_b, dom_ms, dom = ((bytes_b, kb, "backward") if kb >= kf else (bytes_f, kf, "forward"))
        achieved = dom_b / (dom_ms / 1e3) / 1e9
        kname = kernel_name(dom, M) if algo == "chunked" else ("seq_fwd_kernel" if dom == "forward" else "seq_bwd_kernel")
        traffic = profiled_traffic(kname, a.workload)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "precision": "tf32x3" if algo == "chunked" else "fp32",
            "data": "synthetic", "config": workload_config(w, a.workload, algo),
            "ms_fwd": ms_f, "ms_bwd": ms_b, "ms_fwd_kernel": kf, "ms_bwd_kernel": kb,
            "rel_err_vs_fp64": rel_err, "sequential": seq,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic,
                         "algorithmic_bytes": dom_b,
                         "kernel": f"{kname} ({dom} main kernel, CUDA events around each of "
                                   f"its {kfn if dom == 'forward' else kbn} launches)",
                         "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured"
                         else "fallback (6.8 TB/s)"},
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "graph_replay": graph,
            "jvp": jvp, "state_space": ssl,
            # per step: forward = setup + main kernel, backward = main kernel (its work
            # counter is cleared by a memset)
            "gpu_launches": 3 * a.steps if algo == "chunked" else 2 * a.steps,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
