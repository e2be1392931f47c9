"""Benchmark of the GB300 look-ahead decentralized particle filter step.

Workload: the growth/conditionally-linear-Gaussian model (x of dim 2 with the
growth map, z of dim 8, y = x.^2/20 + C z + noise) with N = 65536 outer
particles, M = 128 inner particles each and L = 16 look-ahead draws, FP32,
T = 200 synthetic observations. One "step" is one full LA-DPF step (the fused
inner-step/look-ahead kernel, the outer reduction and the outer resampling).

Metric: particle-updates/s = N * M * steps / time, the inputs (all y_t)
resident in device memory. The state (2 x 302 MB) is larger than the 129 MB
L2, so no L2 flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs an independent filter (weak scaling,
replicas; no collective on the data path); the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "growth_clg10"
METRIC = "particle-updates/s (N*M per step)"
UNIT = "particle-updates/s"
KERNEL_SOURCES = ["paper_1203_2394_gb300/csrc/dpf_step_warp.cuh", "paper_1203_2394_gb300/csrc/dpf_step.cuh",
                  "paper_1203_2394_gb300/csrc/dpf_common.cuh", "paper_1203_2394_gb300/csrc/dpf_variant.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "step_warp_kernel_growth_clg10_traffic.json")


def b_alg(d1, d2, M, s):
    """Algorithmic bytes per particle update: read and write z and lq once, plus the
    per-outer-particle x (read + write), weight, ancestor and selection."""
    return 2 * (d2 + 1) * s + (2 * d1 * s + 12) / M


def kernel_hash():
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, p), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def measured_tflops():
    """The measured dense BF16 burst rate (TFLOP/s) of this machine's GPUs."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p))["bf16_tflops"]), "measured"
    return 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def stop(self, window=None):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines, span = self.lines, "timed region"
        if window is not None:
            inside = [x for x in lines if window[0] <= x[0] <= window[1] + 0.2]
            if not inside:
                # a timed region shorter than the sampling period: the samples just before
                # and just after it (the GPU is loaded by the warm-up and the timed steps)
                before = [x for x in lines if x[0] < window[0]][-1:]
                after = [x for x in lines if x[0] > window[1]][:1]
                inside, span = before + after, "adjacent to a timed region shorter than 200 ms"
            lines = inside
        for ts, ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm), "span": span}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, ws: int, device=None) -> float:
    """Largest value over the ranks (the job's time is its slowest rank's)."""
    if ws <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_oracle_median(spec, N, M, L, runs=3, **kw):
    """cpu_oracle_rate run `runs` times: (median rate, threads, sample, all rates)."""
    rates, threads, sample = [], None, None
    for _ in range(runs):
        r, threads, sample = cpu_oracle_rate(spec, N, M, L, **kw)
        rates.append(r)
    return statistics.median(rates), threads, sample, rates


def cpu_oracle_rate(spec, N, M, L, budget_s=15.0, n_sample=65536, max_steps=16, seed=0, threads=None):
    """The FP64 C oracle, as it stands, on a bounded sample of the workload: the
    first steps (at most max_steps, stopping after budget_s seconds) of a filter with
    n_sample outer particles (same M, L and model), all host cores. Returns
    (particle-updates/s, threads, sample description)."""
    from oracle import oracle
    from paper_1203_2394_gb300 import workloads
    threads = threads or os.cpu_count() or 1
    n_sample = min(n_sample, N)
    _, ys = workloads.simulate(spec, max_steps, 0)
    o = oracle.Oracle(oracle.OracleModel.from_spec(spec), n_sample, M, L, seed, nthreads=threads)
    x, z, lq = o.init()
    t0 = time.perf_counter()
    steps = 0
    while steps < max_steps:
        r = o.step(steps + 1, ys[steps], x, z, lq)
        x, z, lq = r["x"], r["z"], r["lq"]
        steps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    sample = (f"{steps} full LA-DPF steps of a {n_sample}-outer-particle filter (M={M}, L={L}, same "
              f"model), {threads} OpenMP threads, {dt:.1f} s wall")
    return n_sample * M * steps / dt, threads, sample


def run_reference(args):
    """The reference arm: the FP64 C oracle, as it stands, on the host cores. Each
    step is one full LA-DPF step of a bounded sample of the workload (1024 outer
    particles with the workload's M, L and model); the run stops after 150 s."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle
    from paper_1203_2394_gb300 import workloads
    spec = workloads.make_model(WORKLOAD, 0)
    sz = spec.sizes
    n_sample, M, L = 1024, sz["M"], sz["L"]
    threads = os.cpu_count() or 1
    _, ys = workloads.simulate(spec, args.warmup + args.steps + 1, 0)
    o = oracle.Oracle(oracle.OracleModel.from_spec(spec), n_sample, M, L, 0, nthreads=threads)
    x, z, lq = o.init()
    for t in range(1, args.warmup + 1):
        r = o.step(t, ys[t - 1], x, z, lq)
        x, z, lq = r["x"], r["z"], r["lq"]
    t0 = time.perf_counter()
    done = 0
    for t in range(args.warmup + 1, args.warmup + args.steps + 1):
        r = o.step(t, ys[t - 1], x, z, lq)
        x, z, lq = r["x"], r["z"], r["lq"]
        done += 1
        if time.perf_counter() - t0 > 150:
            break
    dt = time.perf_counter() - t0
    value = n_sample * M * done / dt
    sample = (f"{done} timed LA-DPF steps of a {n_sample}-outer-particle filter (M={M}, L={L}, same "
              f"model) after {args.warmup} warm-up steps, {threads} OpenMP threads, {dt:.1f} s")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": done, "warmup": args.warmup, "ms_per_step": dt / done * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: growth-map x (d1=2), linear-Gaussian z (d2=8), dy=2, "
                               f"N={sz['N']}, M={M}, L={L}",
                   "reference": f"FP64 C oracle on a {n_sample}-outer-particle sample per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "cpu": cpu_model(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run(args):
    import numpy as np
    import torch

    from paper_1203_2394_gb300 import dpf, workloads

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    spec = workloads.make_model(WORKLOAD, 0)
    sz = spec.sizes
    N, M, L, T = sz["N"], sz["M"], sz["L"], sz["T"]
    if args.outer:  # a smaller case of the same kernel (profiling); stated in the config
        N = int(args.outer)
    K, W = args.steps, args.warmup
    _, ys = workloads.simulate(spec, max(T, K + W + 1), 0)
    stream = torch.cuda.Stream(device=dev)
    model = dpf.Model.from_spec(spec, dpf.DPF_F32)
    f = dpf.Filter(model, spec.d1, spec.d2, N, M, L, seed=rank, stream=stream)
    y_dev = torch.tensor(ys.astype(np.float32), device=dev)
    assert N * M * (K + W) > 0
    means = torch.zeros((K + W, spec.d), dtype=torch.float64, device=dev)
    logz = torch.zeros(K + W, dtype=torch.float64, device=dev)
    ystep = y_dev.stride(0) * 4

    # ---- device-resident timing ----
    # the clock sampler starts first, so that the warm-up steps, not an idle pause,
    # directly precede the timed ones
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    with torch.cuda.stream(stream):
        for k in range(W):
            f.step_device(y_dev.data_ptr() + k * ystep, means[k].data_ptr(), logz[k].data_ptr())
        f.sync()
        f.profile(True)
        f.profile_read()  # reset
        barrier(ws)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        w0 = time.monotonic()
        e0.record(stream)
        for k in range(W, W + K):
            f.step_device(y_dev.data_ptr() + k * ystep, means[k].data_ptr(), logz[k].data_ptr())
        e1.record(stream)
        torch.cuda.synchronize(dev)
        w1 = time.monotonic()
        f.sync()
        ms = e0.elapsed_time(e1)
        kern_ms, kern_n = f.profile_read()
        f.profile(False)
        clk = clocks.stop(window=(w0, w1))
    barrier(ws)
    ms_max = max_over_ranks(ms, ws, dev)
    value = ws * N * M * K / (ms_max / 1e3)

    # ---- end to end through the public API with host buffers ----
    f2 = dpf.Filter(model, spec.d1, spec.d2, N, M, L, seed=rank + 1000, stream=stream)
    y_pinned = torch.tensor(ys.astype(np.float32)).pin_memory()
    ynp = y_pinned.numpy()
    for k in range(W):
        f2.step(ynp[k])
    barrier(ws)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for k in range(W, W + K):
        f2.step(ynp[k])
    t_e2e = time.perf_counter() - t0
    t_e2e = max_over_ranks(t_e2e, ws, dev)
    e2e_value = ws * N * M * K / t_e2e
    f2.close()

    if rank != 0:
        f.close()
        return 0
    peak, peak_kind = measured_peaks()
    per = b_alg(spec.d1, spec.d2, M, 4)
    kern_avg_s = kern_ms / 1e3 / max(1, kern_n)
    achieved = per * N * M / kern_avg_s / 1e9
    traffic = None
    if os.path.exists(TRAFFIC_FILE):
        tj = json.load(open(TRAFFIC_FILE))
        if tj.get("kernel_hash") == kernel_hash():
            traffic = tj.get("dram_bytes_per_launch")
    cpu = None
    if ws == 1 and not args.no_cpu:
        r, threads, sample, rs = cpu_oracle_median(spec, N, M, L, budget_s=10.0, max_steps=12)
        r1, _, sample1, rs1 = cpu_oracle_median(spec, N, M, L, budget_s=3.0, n_sample=1024, max_steps=4,
                                                threads=1)
        cpu = {"value": r, "unit": UNIT, "cores": threads, "cpu": cpu_model(), "kind": "oracle",
               "sample": sample + "; median of 3 runs", "runs": rs,
               "single_thread": {"value": r1, "unit": UNIT, "sample": sample1 + "; median of 3 runs",
                                 "runs": rs1}}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
        "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: growth-map x (d1=2), linear-Gaussian z (d2=8), dy=2, "
                               f"N={N}, M={M}, L={L}, FP32",
                   "N": N, "M": M, "L": L, "d1": spec.d1, "d2": spec.d2, "dy": spec.dy,
                   "l2": f"state (2 x {N * M * (spec.d2 + 1) * 4 / 1e6:.0f} MB) larger than L2; no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "step_warp_kernel", "kernel_ms": kern_avg_s * 1e3,
                     "bytes_per_update": per, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"},
        # e2e: y_t in (dy floats); out, the statistics and the error word (4 + d + 1
        # doubles) that the outer stage writes to the context's pinned host mirror
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": spec.dy * 4,
                "d2h_bytes_per_step": (5 + spec.d) * 8},
        "lookahead_evaluations_per_s": value * L,  # the N M L look-ahead pairs of every step
        "gpu_launches": 2 * K,  # the step kernel and the outer stage, each step
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    f.close()
    if ws == 1 and not args.no_legs:
        line.update(secondary_legs())
    print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def secondary_legs():
    """Short runs of the other configurations, reported beside the headline (one GPU):
    the 512-filter batched workload (10 graph-captured steps), the learned proposals at
    N = 262144, M = 64 (10 steps each form, with RMSE and inner ESS), four filters of
    the high-dimensional workload as one batch (10 graph-captured steps), and the
    outer-amortised proposal at the high-dimensional size against the plain filter (10
    steps each form, with RMSE and inner ESS). Each carries its own clocks."""
    import torch
    out = {}
    legs = [("batched", run_batched, dict(filters=512, steps=10, warmup=3)),
            ("learned", run_learned, dict(steps=10, warmup=3)),
            ("highdim", run_highdim, dict(filters=4, steps=10, warmup=3)),
            ("highdim_learned", run_highdim_learned, dict(steps=10, warmup=3))]
    for name, fn, kw in legs:
        t0 = time.perf_counter()
        try:
            out[name] = fn(argparse.Namespace(**kw))
        except Exception as e:  # a leg that fails is reported, the headline stands
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["leg_wall_s"] = time.perf_counter() - t0
        torch.cuda.empty_cache()
    return out


def run_batched(args):
    """The many-filter workload: 512 independent linear-Gaussian filters (d = 16, dy = 4,
    split d1 in {1, 2, 4, 8}, N ~ U[1024, 65536], M in {16, 32, 64, 128, 256}, L = 8, FP32),
    T = args.steps steps in one graph-captured run after autotuning; then the batched
    launch against the same filters stepped one at a time on a subset."""
    import numpy as np
    import torch

    from paper_1203_2394_gb300 import dpf, workloads

    torch.cuda.set_device(0)
    rng = np.random.default_rng(0)
    F = args.filters
    d1s = [int(v) for v in rng.choice([1, 2, 4, 8], F)]
    Ns = [int(v) for v in rng.integers(1024, 65537, F)]
    Ms = [int(v) for v in rng.choice([16, 32, 64, 128, 256], F)]
    L, T = 8, args.steps
    free, _ = torch.cuda.mem_get_info()
    need = sum(n * m * (16 - d + 1) * 4 * 2 for n, m, d in zip(Ns, Ms, d1s)) * 1.15
    scale = 1.0
    if need > 0.9 * free:  # run a proportional share of the filters (stated in the output)
        scale = 0.9 * free / need
        F = max(1, int(F * scale))
        d1s, Ns, Ms = d1s[:F], Ns[:F], Ms[:F]
    specs = [workloads.make_model("lg16", 1000 + f, d1=d1s[f]) for f in range(F)]
    models = [dpf.Model.from_spec(sp, dpf.DPF_F32) for sp in specs]
    # enough observations for the timed run and for the subset comparison below (12 steps)
    ys = np.stack([workloads.simulate(sp, max(T + args.warmup, 12), 5 + f)[1] for f, sp in enumerate(specs)],
                  axis=1).astype(np.float32)
    yd = torch.tensor(ys, device="cuda")
    stream = torch.cuda.Stream()
    b = dpf.Batch(models, d1s, Ns, Ms, L, list(range(F)), stream=stream)
    b.run_device(yd.data_ptr(), args.warmup, graph=True)
    t0 = time.perf_counter()
    report = b.autotune(reps=2)  # on the live state after the warm-up steps
    tune_s = time.perf_counter() - t0
    upd = sum(n * m for n, m in zip(Ns, Ms))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    w0 = time.monotonic()
    e0.record(stream)
    b.run_device(yd[args.warmup:].data_ptr(), T, graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    w1 = time.monotonic()
    clk = clocks.stop(window=(w0, w1))
    ms = e0.elapsed_time(e1)
    value = upd * T / (ms / 1e3)
    b.close()
    del b
    torch.cuda.empty_cache()
    # the batched launch against the same filters stepped one at a time (subset)
    S = min(32, F)
    sub = list(range(S))
    bs = dpf.Batch([models[f] for f in sub], [d1s[f] for f in sub], [Ns[f] for f in sub],
                   [Ms[f] for f in sub], L, sub, stream=stream)
    singles = [dpf.Filter(models[f], d1s[f], 16 - d1s[f], Ns[f], Ms[f], L, f, stream=stream) for f in sub]
    ysub = yd[:, :S].contiguous()
    steps_sub, w_sub = 10, 2

    def time_batch(bt):
        bt.run_device(ysub.data_ptr(), w_sub, graph=True)
        bt.autotune(reps=2)
        torch.cuda.synchronize()
        e0.record(stream)
        bt.run_device(ysub[w_sub:].data_ptr(), steps_sub, graph=True)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    ms_b = time_batch(bs)
    for k in range(w_sub):
        for q, f in enumerate(sub):
            singles[q].step_device(ysub[k, q].data_ptr())
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(w_sub, w_sub + steps_sub):
        for q, f in enumerate(sub):
            singles[q].step_device(ysub[k, q].data_ptr())
    e1.record(stream)
    torch.cuda.synchronize()
    ms_s = e0.elapsed_time(e1)
    for s_ in singles:
        s_.close()
    bs.close()
    # the same shapes when every filter is a decomposition of one system: the model
    # constants are then shared by a class and reach the kernel as a launch parameter
    same = [dpf.Model.from_spec(workloads.make_model("lg16", 0, d1=d1s[f]), dpf.DPF_F32) for f in sub]
    bo = dpf.Batch(same, [d1s[f] for f in sub], [Ns[f] for f in sub], [Ms[f] for f in sub], L, sub,
                   stream=stream)
    ms_o = time_batch(bo)
    bo.close()
    upd_sub = sum(Ns[f] * Ms[f] for f in sub) * steps_sub
    # roofline of the whole step (every launch of the graph): the filters' algorithmic
    # bytes against the step time
    bytes_step = sum(b_alg(d1s[f], 16 - d1s[f], Ms[f], 4) * Ns[f] * Ms[f] for f in range(F))
    peak, peak_kind = measured_peaks()
    achieved = bytes_step / (ms / T / 1e3) / 1e9
    classes = report.get("classes", []) if isinstance(report, dict) else []
    n_classes = len(classes)
    # step launches a step: one a class, or one a filter of a class the autotuner split
    n_step_launches = sum(c["filters"] if c.get("split") else 1 for c in classes)
    n_variants = len(set(d1s))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": T,
        "warmup": args.warmup, "ms_per_step": ms / T, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batched: {F} linear-Gaussian filters (d=16, dy=4, d1 in {{1,2,4,8}}, "
                               f"N~U[1024,65536], M in {{16..256}}, L={L}), one graph per run",
                   "filters": F, "share_of_512": F / 512, "particles_per_step": upd,
                   "l2": "state far larger than L2; no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "whole batched step (graph)",
                     "bytes_per_step": bytes_step,
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                     else "fallback 6.8 TB/s"},
        "gpu_launches": T * (n_step_launches + n_variants + 1) if n_classes else None,
        "autotune": report, "autotune_s": tune_s,
        "vs_one_by_one": {"filters": S, "steps": steps_sub, "batched_updates_per_s": upd_sub / (ms_b / 1e3),
                          "one_by_one_updates_per_s": upd_sub / (ms_s / 1e3), "speedup": ms_s / ms_b,
                          "one_system_batched_updates_per_s": upd_sub / (ms_o / 1e3)},
        "clocks": clk,
    }
    return line


def run_highdim(args):
    """The high-dimensional workload: growth_clg64 (x of dim 8 with the growth map, z of
    dim 56 with a dense A_zz, dy = 8), F filters of N = 32768, M = 256, L = 16, FP32,
    every filter's state resident, stepped as one batch (each filter's own tensor-core step
    launch on the batch's stream, the outer stages of all filters in two launches), the
    timed steps one captured graph. Then the tensor-core propagation against the CUDA-core
    one on one member stepped alone."""
    import numpy as np
    import torch

    from paper_1203_2394_gb300 import dpf, workloads

    torch.cuda.set_device(0)
    spec = workloads.make_model("growth_clg64", 0)
    sz = spec.sizes
    N, M, L = sz["N"], sz["M"], sz["L"]
    K, W = args.steps, args.warmup
    F = args.filters if args.filters else 64
    free, _ = torch.cuda.mem_get_info()
    per_filter = 2 * N * M * (spec.d2 + 1) * 4 + N * (16 * 64 + 2 * L * 40)
    share = 1.0
    if F * per_filter > 0.9 * free:  # a proportional share of the filters (stated in the output)
        F2 = max(1, int(0.9 * free // per_filter))
        share = F2 / F
        F = F2
    stream = torch.cuda.Stream()
    model = dpf.Model.from_spec(spec, dpf.DPF_F32)
    b = dpf.Batch([model] * F, [spec.d1] * F, [N] * F, [M] * F, L, list(range(F)), stream=stream)
    # W + K steps of the batch, then 8 more observations for member 0 stepped alone
    ys = np.stack([workloads.simulate(spec, W + K + 8, 5 + f)[1] for f in range(F)], axis=1)
    yd = torch.tensor(ys.astype(np.float32), device="cuda")  # (T, F, dy)
    b.run_device(yd.data_ptr(), W, graph=True)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    w0 = time.monotonic()
    e0.record(stream)
    b.run_device(yd[W:].data_ptr(), K, graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    w1 = time.monotonic()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop(window=(w0, w1))
    value = F * N * M * K / (ms / 1e3)
    # the step kernel alone, and the tensor cores against the CUDA cores, on member 0
    # stepped on its own after the batched run (same state, next steps)
    cmp = {}
    f0 = b.filter(0)
    row = W + K  # the member's next observations, one a step
    with torch.cuda.stream(stream):
        for tc in (True, False):
            f0.set_tensor_cores(tc)
            f0.step_device(yd[row, 0].data_ptr())  # settle the launch shape
            row += 1
            f0.sync()
            f0.profile(True)
            f0.profile_read()
            for r in range(3):
                f0.step_device(yd[row, 0].data_ptr())
                row += 1
            f0.sync()
            a, n = f0.profile_read()
            f0.profile(False)
            cmp["tensor_cores" if tc else "cuda_cores"] = a / max(1, n)
        f0.set_tensor_cores(True)
    b.close()
    peak, peak_kind = measured_peaks()
    per = b_alg(spec.d1, spec.d2, M, 4)
    kern_s = cmp["tensor_cores"] / 1e3  # the step kernel, CUDA events around each launch
    achieved = per * N * M / kern_s / 1e9
    mma_flop = 3 * 2 * N * M * 64 * spec.d2  # 3xTF32, A_zz padded to 64 rows
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": W,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"growth_clg64: growth-map x (d1=8), linear-Gaussian z (d2=56, dense A_zz), "
                               f"dy=8, {F} filters of N={N}, M={M}, L={L}, FP32, one batch, one graph per run",
                   "filters": F, "share_of_64": F / 64 if share == 1.0 else share,
                   "l2": "state far larger than L2; no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "step_kernel_wide (tensor-core)",
                     "kernel_ms": kern_s * 1e3, "bytes_per_update": per,
                     "kernel_timing": "member 0 stepped alone right after the timed batch, CUDA events "
                                      "around each of 3 launches, fresh observations",
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"},
        "tensor": {"mma_tflops": mma_flop / kern_s / 1e12, "mma_flop_per_launch": mma_flop},
        "propagation_kernel_ms": cmp,
        # each step: a step launch a filter, the outer-sums and the resampling launches
        "gpu_launches": K * (F + 2),
        "clocks": clk,
    }
    return line


def run_highdim_learned(args):
    """The learned proposal at the high-dimensional size: growth_clg64 (d1 = 8, d2 = 56,
    dy = 8), N = 32768, L = 16, FP32. The outer-amortised form (one network row per
    group: MLP 3 x 256 ReLU, an affine head of 2 d2 = 112 outputs, BF16 weights, FP32
    accumulation) is trained on the GPU on 1,048,576 rows the plain filter records
    (4 steps x 1024 groups x M = 256), centred at each particle's own prior mean (and, for
    comparison, at the group's mean prior mean); then the filter with it and the plain filter are
    timed over the same steps at M = 256 and M = 128 (the learned form without the
    per-group fallback, and at M = 256 also with it), and their accuracy (RMSE of the
    filtered mean against the simulated states, inner ESS) is measured on an untimed run."""
    import numpy as np
    import torch

    from paper_1203_2394_gb300 import dpf, workloads

    torch.cuda.set_device(0)
    spec = workloads.make_model("growth_clg64", 0)
    sz = spec.sizes
    N, M, L = sz["N"], sz["M"], sz["L"]
    d1, d2, dy = spec.d1, spec.d2, spec.dy
    K, W = args.steps, args.warmup
    model = dpf.Model.from_spec(spec, dpf.DPF_F32)
    if getattr(args, "profile_run", False):
        # one plain step, then two learned steps (prepare, four network products, update,
        # the look-ahead step and the outer stage each)
        pr = dpf.Proposal(d1, d2, dy, hidden=256, amortised_Qz=spec.Q[d1:, d1:])
        W0 = workloads.init_mlp_weights(2 * d1 + dy + 2 * d2, 256, 2 * d2, seed=0)
        W0["W4"] *= 0.1
        pr.set_weights(W0)
        pr.set_centre(True)
        f = dpf.Filter(model, d1, d2, N, M, L, seed=3)
        f.set_proposal(pr)
        f.set_fallback(0.0)
        _, ys = workloads.simulate(spec, 3, 0)
        for t in range(3):
            f.step(ys[t].astype(np.float32))
        torch.cuda.synchronize()
        f.close()
        pr.close()
        return {"workload": "highdim_learned profile run", "steps": 3, "N": N, "M": M, "L": L}
    stream = torch.cuda.Stream()
    # ---- training rows and training ----
    t0 = time.perf_counter()
    n_rec, t_rec = 1024, 4
    _, ys_tr = workloads.simulate(spec, t_rec + 2, 100)
    rec = dpf.Filter(model, d1, d2, n_rec, M, L, seed=1, stream=stream)
    rec.set_debug(True)
    rows = []
    for t in range(t_rec + 1):
        rec.step(ys_tr[t].astype(np.float32))
        if t >= 1:
            rows.append(rec.record_amortised())
    rec.close()
    G = torch.cat([r[0] for r in rows]); Zm = torch.cat([r[1] for r in rows]); wm = torch.cat([r[2] for r in rows])
    del rows
    din, dout = 2 * d1 + dy + 2 * d2, 2 * d2
    A0 = workloads.init_mlp_weights(din, 256, dout, seed=0)
    A0["W4"][:] = 0.0
    A0["b4"][:] = 0.0  # start at the identity map (the prior)
    props, losses = {}, {}
    for centre in ("particle", "group"):
        pr = dpf.Proposal(d1, d2, dy, hidden=256, stream=stream, amortised_Qz=spec.Q[d1:, d1:])
        pr.set_centre(centre == "particle")
        pr.set_weights(A0)
        Zc = Zm
        if centre == "particle":  # the rows' centre block: the particle's own prior mean
            Zc = Zm.clone()
            Zc[:, 2 * d2:] = Zm[:, d2:2 * d2]
        losses[centre] = [float(v) for v in pr.train(G, Zc, wm, batch=2048, epochs=3, lr=1e-3, seed=2)]
        props[centre] = pr
        del Zc
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    n_rows = int(G.shape[0])
    prop = props["particle"]
    del G, Zm, wm
    torch.cuda.empty_cache()
    # ---- timing ----
    _, ys = workloads.simulate(spec, W + K + 1, 0)
    yd = torch.tensor(ys.astype(np.float32), device="cuda")

    def timed(m_inner, use_prop, frac=0.0):
        f = dpf.Filter(model, d1, d2, N, m_inner, L, seed=3, stream=stream)
        if use_prop:
            f.set_proposal(use_prop)
            f.set_fallback(frac)
        with torch.cuda.stream(stream):
            for k in range(W):
                f.step_device(yd[k].data_ptr())
            f.sync()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(W, W + K):
                f.step_device(yd[k].data_ptr())
            e1.record(stream)
            torch.cuda.synchronize()
            f.sync()
        f.close()
        return e0.elapsed_time(e1) / K

    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    w0 = time.monotonic()
    ms = {("learned", M, 0.0): timed(M, prop)}
    w1 = time.monotonic()
    clk = clocks.stop(window=(w0, w1))
    ms[("plain", M, None)] = timed(M, None)
    ms[("learned", M // 2, 0.0)] = timed(M // 2, prop)
    ms[("plain", M // 2, None)] = timed(M // 2, None)
    ms[("learned", M, 0.25)] = timed(M, prop, 0.25)
    ms[("learned_group_centre", M, 0.0)] = timed(M, props["group"])
    # ---- accuracy on an untimed run ----
    T = 50
    s_true, ya = workloads.simulate(spec, T, 200)

    def accuracy(m_inner, use_prop, frac):
        f = dpf.Filter(model, d1, d2, N, m_inner, L, seed=5, stream=stream)
        if use_prop:
            f.set_proposal(use_prop)
            f.set_fallback(frac)
        err, ess, fb = [], [], []
        for t in range(T):
            m, _ = f.step(ya[t].astype(np.float32))
            err.append(m - s_true[t + 1])
            if t >= 1:
                lq = torch.tensor(f.read("lq"), device="cuda", dtype=torch.float64)
                Wt = torch.exp(lq - lq.max(dim=1, keepdim=True).values)
                ess.append(float((Wt.sum(1) ** 2 / (Wt * Wt).sum(1)).mean()) / m_inner)
                if use_prop:
                    fb.append(float(np.mean(f.read("fallback"))))
        f.close()
        return {"rmse_vs_truth": float(np.sqrt(np.mean(np.square(err)))), "inner_ess": float(np.mean(ess)),
                "fallback_share": float(np.mean(fb)) if fb else None}

    acc = {}
    for kind, m_inner, frac in ms:
        use = {"learned": prop, "learned_group_centre": props["group"]}.get(kind)
        acc[(kind, m_inner, frac)] = accuracy(m_inner, use, frac)
    for pr in props.values():
        pr.close()

    def form_name(kind, m_inner, frac):
        return f"{kind}_M{m_inner}" + (f"_fallback{frac}" if frac else "")
    forms = {form_name(kind, m_inner, frac): {"M": m_inner, "fallback_threshold": frac, "ms_per_step": v,
                                              "value": N * m_inner / (v / 1e3), **acc[(kind, m_inner, frac)]}
             for (kind, m_inner, frac), v in ms.items()}
    v_l = forms[f"learned_M{M}"]["ms_per_step"]
    mlp_flop = 2 * (din * 256 + 2 * 256 * 256 + 256 * dout)  # per group
    line = {
        "metric": METRIC, "value": N * M / (v_l / 1e3), "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": W,
        "ms_per_step": v_l, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 filter, bf16 MLP", "data": "synthetic",
        "config": {"workload": f"learned proposal at the high-dimensional size: growth_clg64 (d1={d1}, d2={d2}, "
                               f"dy={dy}), N={N}, M={M}, L={L}, FP32; outer-amortised MLP 3x256 ReLU, affine "
                               "head, BF16 weights, FP32 accumulate; one filter",
                   "centre": "learned forms: the particle's own prior mean; learned_group_centre: the group's "
                             "mean prior mean",
                   "training_rows": n_rows, "training_epochs": 3, "training_batch": 2048,
                   "training_s_both": train_s, "training_losses": losses,
                   "l2": "state far larger than L2; no flush"},
        "forms": forms,
        "accuracy_steps": T,
        "network_flop_per_group": mlp_flop,
        # the headline form (no fallback) each step: the prepare pass, four network
        # products, the update pass, the look-ahead step and the outer stage
        "gpu_launches": 8 * K,
        "clocks": clk,
    }
    return line


def run_compare(args):
    """The paper's comparison (Section 4.1): the LA-DPF (N = 65536, M = 128, L = 16) against
    the DPF without look-ahead of the same sizes and the bootstrap particle filter with
    N (M + 1) = 8,454,144 particles (the paper sizes the PF so), on the growth workload in
    FP32: time per step (device observations, CUDA events over the timed steps) and RMSE of
    the filtered mean against the true state, per block."""
    import numpy as np
    import torch

    from paper_1203_2394_gb300 import dpf, workloads

    torch.cuda.set_device(0)
    spec = workloads.make_model(WORKLOAD, 0)
    sz = spec.sizes
    N, M, L = sz["N"], sz["M"], sz["L"]
    K, W = args.steps, args.warmup
    T = W + K
    s_true, ys = workloads.simulate(spec, T, 0)
    model = dpf.Model.from_spec(spec, dpf.DPF_F32)
    yd = torch.tensor(ys.astype(np.float32), device="cuda")
    stream = torch.cuda.current_stream()

    def timed(f, name):
        means = torch.zeros((T, spec.d), dtype=torch.float64, device="cuda")
        for k in range(W):
            f.step_device(yd[k].data_ptr(), means[k].data_ptr())
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(W, T):
            f.step_device(yd[k].data_ptr(), means[k].data_ptr())
        e1.record(stream)
        torch.cuda.synchronize()
        f.sync()
        m = means.cpu().numpy()
        err = m[W:] - s_true[W + 1:T + 1]  # the estimates of the timed steps against the truth
        d1 = spec.d1
        return {"ms_per_step": e0.elapsed_time(e1) / K,
                "rmse_x": float(np.sqrt(np.mean(err[:, :d1] ** 2))),
                "rmse_z": float(np.sqrt(np.mean(err[:, d1:] ** 2)))}

    la = dpf.Filter(model, spec.d1, spec.d2, N, M, L, seed=0)
    r_la = timed(la, "ladpf")
    la.close()
    sd = dpf.StandardDPF(model, spec.d1, spec.d2, N, M, seed=0)
    r_sd = timed(sd, "dpf")
    sd.close()
    r_sd["particle_updates_per_s"] = N * M / (r_sd["ms_per_step"] / 1e3)
    Np = N * (M + 1)
    pfl = dpf.ParticleFilter(model, spec.d1, spec.d2, Np, seed=0)
    r_pf = timed(pfl, "pf")
    pfl.close()
    r_la["particle_updates_per_s"] = N * M / (r_la["ms_per_step"] / 1e3)
    r_pf["particles"] = Np
    r_pf["particle_updates_per_s"] = Np / (r_pf["ms_per_step"] / 1e3)
    line = {
        "metric": METRIC, "value": r_la["particle_updates_per_s"], "unit": UNIT, "n_gpus": 1, "steps": K,
        "warmup": W, "ms_per_step": r_la["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"comparison on {WORKLOAD}: LA-DPF N={N}, M={M}, L={L} against the DPF "
                               f"without look-ahead (same N, M) and the bootstrap PF with N(M+1)={Np} "
                               f"particles, FP32; RMSE over the {K} timed steps"},
        "ladpf": r_la, "dpf": r_sd, "pf": r_pf,
    }
    print(json.dumps(line))
    return 0


def run_table2(args):
    """The Gaussian approximation of the mixture prior against its Monte Carlo evaluation
    (Section 4.2, Table 2), as the paper runs it: the DPF without look-ahead with N = 100,
    M = 19 and 100 runs, in FP32, on the paper's model 1 (Table 1) over 250 steps, and on
    lg4 (x depends on z linearly) over 50 steps. Reports the RMSE of the filtered mean against
    the true state per block (x, z), averaged over the runs, and the time of a run."""
    import numpy as np
    import torch

    from paper_1203_2394_gb300 import dpf, workloads

    torch.cuda.set_device(0)
    N, M, R = 100, 19, 100
    spec = workloads.make_model("lg4", 0)
    cases = [("model1", dpf.PaperModel(1), 1, 1, 250,
              lambda r, T: workloads.simulate_paper(1, T, 1000 + r)),
             ("lg4", dpf.Model.from_spec(spec, dpf.DPF_F32), spec.d1, spec.d2, 50,
              lambda r, T: workloads.simulate(spec, T, 1000 + r))]
    out, wall = {}, {}
    for name, model, d1, d2, T, sim in cases:
        res = {False: [], True: []}
        t0 = time.perf_counter()
        for r in range(R):
            s_true, ys = sim(r, T)
            for gauss in (False, True):
                f = dpf.StandardDPF(model, d1, d2, N, M, seed=r)
                f.set_gaussian_approx(gauss)
                means = np.array([f.step(ys[t].astype(np.float32))[0] for t in range(T)])
                f.close()
                err = means - s_true[1:]
                res[gauss].append((np.sqrt(np.mean(err[:, :d1] ** 2)), np.sqrt(np.mean(err[:, d1:] ** 2))))
        wall[name] = time.perf_counter() - t0
        mc, ga = np.array(res[False]), np.array(res[True])
        out[name] = {"steps": T, "ms_per_step": wall[name] / (2 * R * T) * 1e3,
                     "gaussian": {"rmse_x": float(ga[:, 0].mean()), "rmse_z": float(ga[:, 1].mean())},
                     "monte_carlo": {"rmse_x": float(mc[:, 0].mean()), "rmse_z": float(mc[:, 1].mean())}}
    line = {
        "metric": "RMSE against the true state (mean over runs)", "value": out["model1"]["gaussian"]["rmse_x"],
        "unit": "state units", "n_gpus": 1, "steps": 250, "warmup": 0, "ms_per_step": out["model1"]["ms_per_step"],
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"Gaussian against Monte Carlo evaluation of the mixture prior: DPF without "
                               f"look-ahead, N={N}, M={M}, {R} runs, FP32, on the paper's model 1 (250 steps) and "
                               f"on lg4 (50 steps); value: model 1, Gaussian, RMSE of x"},
        **out,
        "paper_table2_model1": {"gaussian": {"rmse_x": 1.3197, "rmse_z": 1.1705},
                                "monte_carlo": {"rmse_x": 1.3216, "rmse_z": 1.1640}},
    }
    print(json.dumps(line))
    return 0


def run_paper(args):
    """The paper's comparison (Section 4.1) on its own benchmark models (Table 1): for
    model 1 and model 2, the LA-DPF (N = 65536, M = 128, L = 16), the DPF without look-ahead
    (same N, M) and the bootstrap particle filter with N (M + 1) = 8,454,144 particles, FP32, over R runs of 250 steps (the paper's
    horizon) on seeded trajectories: the RMSE of the filtered mean against the true state per
    block (x, z), averaged over the runs, and the time per step (device observations, CUDA
    events over the steps after the first 10)."""
    import numpy as np
    import torch

    from paper_1203_2394_gb300 import dpf, workloads

    torch.cuda.set_device(0)
    N, M, L, T, W0 = 65536, 128, 16, 250, 10
    R = max(1, min(args.runs, 8))
    stream = torch.cuda.current_stream()

    def run(f, yd, s_true, d, d1):
        means = torch.zeros((T, d), dtype=torch.float64, device="cuda")
        for k in range(W0):
            f.step_device(yd[k].data_ptr(), means[k].data_ptr())
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(W0, T):
            f.step_device(yd[k].data_ptr(), means[k].data_ptr())
        e1.record(stream)
        torch.cuda.synchronize()
        f.sync()
        err = means.cpu().numpy() - s_true[1:]
        return (e0.elapsed_time(e1) / (T - W0), float(np.sqrt(np.mean(err[:, :d1] ** 2))),
                float(np.sqrt(np.mean(err[:, d1:] ** 2))))

    out = {}
    for kind in (1, 2):
        pm = dpf.PaperModel(kind)
        res = {"ladpf": [], "dpf": [], "pf": []}
        for r in range(R):
            s_true, ys = workloads.simulate_paper(kind, T, 100 + r)
            yd = torch.tensor(ys.astype(np.float32), device="cuda")
            f = dpf.Filter(pm, pm.d1, pm.d2, N, M, L, seed=r)
            res["ladpf"].append(run(f, yd, s_true, pm.d, pm.d1))
            f.close()
            f = dpf.StandardDPF(pm, pm.d1, pm.d2, N, M, seed=r)
            res["dpf"].append(run(f, yd, s_true, pm.d, pm.d1))
            f.close()
            f = dpf.ParticleFilter(pm, pm.d1, pm.d2, N * (M + 1), seed=r)
            res["pf"].append(run(f, yd, s_true, pm.d, pm.d1))
            f.close()
        out[f"model{kind}"] = {
            k: {"ms_per_step": float(np.mean([v[0] for v in res[k]])),
                "rmse_x": float(np.mean([v[1] for v in res[k]])),
                "rmse_z": float(np.mean([v[2] for v in res[k]]))} for k in res}
        out[f"model{kind}"]["pf"]["particles"] = N * (M + 1)
    ms = out["model1"]["ladpf"]["ms_per_step"]
    line = {
        "metric": METRIC, "value": N * M / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": T - W0,
        "warmup": W0, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"the paper's models 1 and 2 (Table 1): LA-DPF N={N}, M={M}, L={L} against the "
                               f"DPF without look-ahead (same N, M) and the bootstrap PF with N(M+1)={N * (M + 1)} particles, FP32, {R} runs of {T} steps; "
                               f"value: model 1's LA-DPF"},
        **out,
    }
    print(json.dumps(line))
    return 0


def run_bandit(args):
    """Automatic state decomposition on the paper's model 1 (Section 4.3): two actions, the
    table's order (x outer, z inner) and the other way (perm = (1, 0)), each an LA-DPF in FP32
    stepped on the same observations, at two sizes (N, M, L) = (100, 10, 8) and (1000, 32, 16).
    Every step each action earns alpha / (alpha + eps^2), eps = y_t - yhat_t with yhat_t =
    h(f(m_{t-1}, t-1)) from its own filtered mean; Hedge takes both rewards, Exp3 (gamma = 0.2,
    eta = 0.5) only its chosen action's. The output at step t is the chosen action's filtered
    mean (Hedge: its most probable action). Reports the RMSE against the true state of each
    fixed action and of both bandits, and the final probabilities, averaged over R runs of T
    steps."""
    import numpy as np
    import torch

    from paper_1203_2394_gb300 import dpf, workloads

    torch.cuda.set_device(0)
    T, R = 1000, max(1, min(args.runs, 8))
    ETA, GAMMA = 0.5, 0.2
    alpha = float(args.alpha)

    def f_mean(m, s):  # the table's transition mean at step s
        x, z = m
        return np.array([x + z / (1 + z * z), x + 0.5 * z + 25 * z / (1 + z * z) + 8 * np.cos(1.2 * s)])

    def h(m):
        return np.arctan(m[0]) + m[1] ** 2 / 20

    def one_size(N, M, L):
        res = {k: [] for k in ("action1", "action2", "hedge", "exp3")}
        probs = {"hedge": [], "exp3": []}
        chosen1 = []
        for r in range(R):
            s_true, ys = workloads.simulate_paper(1, T, 500 + r)
            fs = [dpf.Filter(dpf.PaperModel(1, perm=p), 1, 1, N, M, L, seed=r) for p in (None, (1, 0))]
            hedge = dpf.Bandit(dpf.DPF_HEDGE, 2, ETA, 0.0, seed=r)
            exp3 = dpf.Bandit(dpf.DPF_EXP3, 2, ETA, GAMMA, seed=r)
            prev = [np.zeros(2), np.zeros(2)]  # s_0 ~ N(0, I): the prior mean
            err = {k: [] for k in res}
            n1 = 0
            for t in range(1, T + 1):
                y = ys[t - 1].astype(np.float32)
                rew = np.array([dpf.bandit_reward(y, [h(f_mean(prev[a], t - 1))], alpha) for a in range(2)])
                a3 = exp3.choose()
                ah = int(np.argmax(hedge.probs()))
                means = [f.step(y)[0] for f in fs]
                hedge.update(rew)
                exp3.update(rew[a3:a3 + 1])  # Exp3 is told the tried action's reward only
                n1 += a3 == 0
                for k, mu in (("action1", means[0]), ("action2", means[1]), ("hedge", means[ah]),
                              ("exp3", means[a3])):
                    err[k].append(mu - s_true[t])
                prev = means
            for f in fs:
                f.close()
            for k in res:
                res[k].append(np.sqrt(np.mean(np.array(err[k]) ** 2, axis=0)))
            probs["hedge"].append(hedge.probs().tolist())
            probs["exp3"].append(exp3.probs().tolist())
            chosen1.append(n1 / T)
            hedge.close()
            exp3.close()
        out = {k: {"rmse_x": float(np.mean([v[0] for v in res[k]])), "rmse_z": float(np.mean([v[1] for v in res[k]]))}
               for k in res}
        out["final_probs"] = {k: np.mean(v, axis=0).tolist() for k, v in probs.items()}
        out["exp3_share_action1"] = float(np.mean(chosen1))
        return out

    t0 = time.perf_counter()
    small = one_size(100, 10, 8)
    large = one_size(1000, 32, 16)
    wall = time.perf_counter() - t0
    line = {
        "metric": "RMSE against the true state (mean over runs)", "value": small["exp3"]["rmse_z"],
        "unit": "state units", "n_gpus": 1, "steps": T, "warmup": 0, "ms_per_step": wall / (2 * R * T) * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"automatic decomposition of the paper's model 1: two LA-DPFs (x outer / z outer), "
                               f"FP32, Hedge and Exp3 (eta={ETA}, gamma={GAMMA}, alpha={alpha}), {R} runs of {T} "
                               f"steps, at N, M, L = 100, 10, 8 and 1000, 32, 16; value: Exp3's RMSE of z at the "
                               f"small size"},
        "n100_m10_l8": small, "n1000_m32_l16": large,
    }
    print(json.dumps(line))
    return 0


def run_learned(args):
    """The learned-proposal workload: the lg4 model in FP32 with N = 262144 outer and
    M = 64 inner particles. A proposal (MLP 3 x 256 ReLU, 4-component mixture head, BF16
    weights, FP32 accumulation) is trained on the GPU on 10^6 rows the plain filter
    records, and so is the outer-amortised form (one network row per group); then the
    filter with the mixture (L = 1), the plain filter (L = 8) and the filter with the
    amortised form (L = 8) are timed over the same steps, and their accuracy (RMSE of the
    filtered mean against the Kalman filter, inner ESS) is measured on a separate
    untimed run."""
    import numpy as np
    import torch

    from paper_1203_2394_gb300 import dpf, workloads

    torch.cuda.set_device(0)
    spec = workloads.make_model("lg4", 0)
    model = dpf.Model.from_spec(spec, dpf.DPF_F32)
    N, M = 262144, 64
    K, W = args.steps, args.warmup
    stream = torch.cuda.Stream()
    # ---- training rows and training ----
    t0 = time.perf_counter()
    # 8 steps x 2048 outer x 64 inner = 1,048,576 rows of the plain filter (L = 8)
    _, ys_tr = workloads.simulate(spec, 10, 100)
    rec = dpf.Filter(model, 2, 2, 2048, M, 8, seed=1, stream=stream)
    rec.set_debug(True)
    rows, arows = [], []
    for t in range(9):
        rec.step(ys_tr[t].astype(np.float32))
        if t >= 1:
            rows.append(rec.record())
            arows.append(rec.record_amortised())
    rec.close()
    F = torch.cat([r[0] for r in rows]); Z = torch.cat([r[1] for r in rows]); w = torch.cat([r[2] for r in rows])
    del rows
    prop = dpf.Proposal(2, 2, 2, hidden=256, components=4, stream=stream)
    W0 = workloads.init_mlp_weights(8, 256, 20, seed=0)
    W0["b4"][12:] = np.log(np.sqrt(0.1))
    prop.set_weights(W0)
    losses = prop.train(F, Z, w, batch=1024, epochs=3, lr=1e-3, seed=2)
    train_s = time.perf_counter() - t0
    del F, Z, w
    # the outer-amortised form: rows of the same recorder, one network row per group
    G = torch.cat([r[0] for r in arows]); Zm = torch.cat([r[1] for r in arows]); wm = torch.cat([r[2] for r in arows])
    del arows
    Qz = spec.Q[2:, 2:]
    aprop = dpf.Proposal(2, 2, 2, hidden=256, stream=stream, amortised_Qz=Qz)
    A0 = workloads.init_mlp_weights(10, 256, 4, seed=0)
    A0["W4"][:] = 0.0
    A0["b4"][:] = 0.0
    aprop.set_weights(A0)
    alosses = aprop.train(G, Zm, wm, batch=1024, epochs=3, lr=1e-3, seed=2)
    del G, Zm, wm
    # ---- timing ----
    _, ys = workloads.simulate(spec, W + K + 1, 0)
    yd = torch.tensor(ys.astype(np.float32), device="cuda")

    def timed(L, use_prop, n_outer=N, m_inner=M):
        f = dpf.Filter(model, 2, 2, n_outer, m_inner, L, seed=3, stream=stream)
        if use_prop:
            f.set_proposal(use_prop)
        with torch.cuda.stream(stream):
            for k in range(W):
                f.step_device(yd[k].data_ptr())
            f.sync()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(W, W + K):
                f.step_device(yd[k].data_ptr())
            e1.record(stream)
            torch.cuda.synchronize()
            f.sync()
        f.close()
        return e0.elapsed_time(e1)

    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    w0 = time.monotonic()
    ms_l = timed(1, prop)
    w1 = time.monotonic()
    clk = clocks.stop(window=(w0, w1))
    ms_p = timed(8, None)
    ms_a = timed(8, aprop)
    ms_p4 = timed(8, None, N, 4 * M)  # the plain filter with four times the inner particles
    # ---- accuracy on an untimed run ----
    T = 25
    _, ya = workloads.simulate(spec, T, 200)
    import numpy.linalg as la_

    def kalman_means(ys_):
        m, P = spec.m0.copy(), spec.P0.copy()
        out = []
        for y in ys_:
            m = spec.A @ m
            P = spec.A @ P @ spec.A.T + spec.Q
            S = spec.H @ P @ spec.H.T + spec.R
            Kg = P @ spec.H.T @ la_.inv(S)
            m = m + Kg @ (y - spec.H @ m)
            P = P - Kg @ S @ Kg.T
            out.append(m.copy())
        return np.array(out)
    km = kalman_means(ya)

    def accuracy(L, use_prop, n_outer=N, m_inner=M):
        f = dpf.Filter(model, 2, 2, n_outer, m_inner, L, seed=5, stream=stream)
        if use_prop:
            f.set_proposal(use_prop)
        err, ess = [], []
        for t in range(T):
            m, _ = f.step(ya[t].astype(np.float32))
            err.append(m - km[t])
            if t >= 1:
                lq = f.read("lq").astype(np.float64)
                Wt = np.exp(lq - lq.max(axis=1, keepdims=True))
                ess.append(float(np.mean(Wt.sum(1) ** 2 / (Wt * Wt).sum(1)) / m_inner))
        f.close()
        return float(np.sqrt(np.mean(np.square(err)))), float(np.mean(ess))

    rmse_l, ess_l = accuracy(1, prop)
    rmse_p, ess_p = accuracy(8, None)
    rmse_a, ess_a = accuracy(8, aprop)
    rmse_p4, ess_p4 = accuracy(8, None, N, 4 * M)
    value = N * M * K / (ms_l / 1e3)
    mlp_flop = 2 * (8 * 256 + 2 * 256 * 256 + 256 * 20)  # per inner particle
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": W,
        "ms_per_step": ms_l / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 filter, bf16 MLP", "data": "synthetic",
        "config": {"workload": f"learned proposal: lg4 model (d=4, x 2 / z 2), FP32, N={N}, M={M}, L=1; "
                               "MLP 3x256 ReLU, 4-component mixture head, BF16 weights, FP32 accumulate",
                   "training_rows": 8 * 2048 * M, "training_epochs": 3, "training_s": train_s,
                   "training_losses": list(losses),
                   "l2": "state larger than L2; no flush"},
        "tensor": {"mlp_tflops": mlp_flop * N * M * K / (ms_l / 1e3) / 1e12,
                   "mlp_flop_per_update": mlp_flop},
        "plain": {"L": 8, "value": N * M * K / (ms_p / 1e3), "ms_per_step": ms_p / K},
        "plain_4M": {"L": 8, "M": 4 * M, "ms_per_step": ms_p4 / K, "rmse_vs_kalman": rmse_p4,
                     "inner_ess": ess_p4, "value": N * 4 * M * K / (ms_p4 / 1e3)},
        "amortised": {"L": 8, "value": N * M * K / (ms_a / 1e3), "ms_per_step": ms_a / K,
                      "training_losses": list(alosses), "network_rows_per_step": N},
        "accuracy": {"steps": T, "rmse_vs_kalman_learned": rmse_l, "rmse_vs_kalman_plain": rmse_p,
                     "rmse_vs_kalman_amortised": rmse_a, "inner_ess_learned": ess_l,
                     "inner_ess_plain": ess_p, "inner_ess_amortised": ess_a},
        # the learned pass, the fallback lists, the fallback groups' step, the look-ahead
        # step and the outer stage, each step
        "gpu_launches": 5 * K,
        "clocks": clk,
    }
    tf_peak, tf_kind = measured_tflops()
    line["roofline"] = {"bound": "tensor", "achieved": line["tensor"]["mlp_tflops"], "peak": tf_peak,
                        "unit": "TFLOP/s", "frac": line["tensor"]["mlp_tflops"] / tf_peak, "traffic": None,
                        "kernel": "whole step with the mixture proposal (learned_kernel dominates)",
                        "flop_per_update": mlp_flop,
                        "peak_source": f"{tf_kind} (MEASURED_PEAKS.json bf16_tflops)"}
    prop.close()
    aprop.close()
    return line
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--workload", default="growth_clg10", choices=["growth_clg10", "batched", "highdim", "highdim_learned", "learned", "compare", "table2", "paper",
                             "bandit"],
                    help="the headline single-filter workload, the many-filter one, the d2 = 56 one, "
                         "the learned-proposal one, or the LA-DPF against the bootstrap PF")
    ap.add_argument("--runs", type=int, default=3, help="runs per model of the paper and bandit workloads (at most 8)")
    ap.add_argument("--alpha", type=float, default=0.001, help="the bandit reward's alpha (the paper's 0.001)")
    ap.add_argument("--filters", type=int, default=None,
                    help="filters of the batched (default 512) or high-dimensional (default 64) workload")
    ap.add_argument("--outer", type=int, default=None,
                    help="outer particles of the headline workload (default its 65536; for profiling a "
                         "smaller case of the same kernel)")
    ap.add_argument("--profile-run", action="store_true",
                    help="highdim_learned: only three steps of the learned filter (untrained network, no "
                         "fallback), no timing: the launches a profiler captures")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the short batched, learned and high-dimensional legs of the default run")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        if args.filters is None:
            args.filters = 512
        print(json.dumps(run_batched(args)))
        return 0
    if args.workload == "highdim":
        print(json.dumps(run_highdim(args)))
        return 0
    if args.workload == "learned":
        print(json.dumps(run_learned(args)))
        return 0
    if args.workload == "highdim_learned":
        print(json.dumps(run_highdim_learned(args)))
        return 0
    if args.workload == "compare":
        return run_compare(args)
    if args.workload == "table2":
        return run_table2(args)
    if args.workload == "paper":
        return run_paper(args)
    if args.workload == "bandit":
        return run_bandit(args)
    return run(args)


if __name__ == "__main__":
    sys.exit(main())
