"""Benchmark of the additive-kernel NFFT fast summation on GB300.

Workload (one GPU): n = 1,000,000 points, p = 8 standardized Gaussian features
min-max scaled to [-0.24, 0.24], windows {0,1,2},{3,4,5},{6,7} (d = 3, 3, 2),
Gaussian kernel, ell = sigma_f = sigma_eps = ln 2, N = 32 / 32 / 64, cutoff
s = 5, FP32, 32 right-hand sides [y, 31 Rademacher probes].

One step = new hyperparameters (Fourier coefficients of the kernel and its
ell-derivative, recomputed on the device) + one application of K_hat to the
32 right-hand sides (spread, DFT, multiply, inverse DFT, interpolate, window
sum). The point set is fixed during hyperparameter training, so the plan
(binning and sorting of the points) is built once, before the timed region.

Metric: additive-kernel MVMs/s (one MVM = K_hat applied to one vector, all
windows). `e2e` times the same step through the C ABI with the right-hand
sides in pinned host memory and the result copied back every step.

--impl reference times the FP64 CPU oracle (Fourier-truncated sum) on the
host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2504_00480_gb300 import inputs  # noqa: E402

METRIC = ("additive-kernel MVMs/s (n=1M, 32 RHS) vs plain FP64 path; HBM GB/s")
UNIT = "MVM/s"
N_POINTS = 1_000_000
R = 32
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def workload_config(n=N_POINTS):
    return {"workload": f"additive Gaussian kernel, n={n}, p=8, windows d=(3,3,2), "
                        f"N=(32,32,64), s=5, sigma_os=2, 32 RHS, FP32",
            "n": n, "rhs": R, "windows": [[0, 1, 2], [3, 4, 5], [6, 7]], "N": [32, 32, 64],
            "cutoff": 5, "kernel": "gauss", "l2": "inputs larger than L2; L2 flushed between steps"}


# ---------------------------------------------------------------------------
# clocks sampled with nvidia-smi during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", delete=False, suffix=".csv")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.f is None:
            return None
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.f.name)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, flags in rows for k, fl in enumerate(flags)
                          if fl.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def measured_traffic(kernel, n, R):
    """DRAM bytes (read + write) of one launch of `kernel` from the committed
    ncu summary in profiles/traffic.json, or None when the summary does not
    match this workload or the kernel source changed after the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        entry = json.load(open(path))[kernel]
    except (OSError, KeyError, ValueError):
        return None
    if entry.get("n") != n or entry.get("rhs") != R:
        return None
    src = os.path.join(ROOT, "paper_2504_00480_gb300", "csrc", entry["source_file"])
    try:
        import hashlib
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    return entry["bytes"] if digest == entry.get("source_sha256") else None


# ---------------------------------------------------------------------------
# reference arm / CPU baseline: the FP64 oracle on host cores
# ---------------------------------------------------------------------------
def oracle_mvms_per_s(w, target_s=15.0):
    """Time the oracle's truncated sum (Sec. 3.1 eq. (3.3), one RHS) on a prefix
    sample of the workload and scale to MVMs/s at the full n (its cost is
    linear in n at fixed N)."""
    import oracle
    n_full = w.n

    def run(m):
        t = time.perf_counter()
        oracle.truncated_matvec(w.X[:m], w.windows, w.kernel, w.ell, w.sigma_f, w.sigma_eps,
                                w.V[:m, :1], w.N)
        return time.perf_counter() - t

    m0 = 20_000
    t0 = run(m0)
    m = int(min(n_full, max(m0, m0 * target_s / max(t0, 1e-3))))
    t = run(m) if m > m0 else t0
    m = m if m > m0 else m0
    rate = (m / n_full) / t
    return rate, {"points": m, "seconds": t, "rhs": 1}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = inputs.nlml_grad(R=2)
    times = []
    info = None
    for it in range(args.warmup + args.steps):
        rate, info = oracle_mvms_per_s(w, target_s=args.ref_seconds)
        if it >= args.warmup:
            times.append(rate)
    v = statistics.median(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * R / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(),
            "cpu_baseline": {"kind": "oracle", "value": v, "unit": UNIT,
                             "cores": os.cpu_count(),
                             "sample": f"oracle truncated sum on the first {info['points']} "
                                       f"points, 1 RHS, {info['seconds']:.1f} s, scaled "
                                       f"linearly to n={N_POINTS}"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2504_00480_gb300 import agp, build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    agp.load_library()

    w = inputs.nlml_grad(R=R)
    X = torch.tensor(w.X, dtype=torch.float32, device=dev)
    V = torch.tensor(w.V, dtype=torch.float32, device=dev)
    Out = torch.empty_like(V)
    plan = agp.Plan(X, w.windows, w.N, w.cutoff, w.kernel, w.ell, w.sigma_f, w.sigma_eps)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    ells = [w.ell * (1.0 + 1e-3 * k) for k in range(args.warmup + args.steps + 1)]

    def step(k):
        plan.set_hyper(ells[k], w.sigma_f, w.sigma_eps)
        agp.agp_matvec(plan.handle, V, Out, True)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()

    # device-timed region
    plan.profile(True)
    plan.profile_read(reset=True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))                  # L2 flush, outside the timed events
            evs[k][0].record(stream)
            step(args.warmup + k)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    prof = plan.profile_read(reset=True)
    plan.profile(False)
    ms = sum(a.elapsed_time(b) for a, b in evs)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t)
    ms_step = ms / args.steps
    value = world * R * args.steps / (ms / 1e3)
    launches_per_step = sum(p["launches"] for p in prof.values()) / args.steps

    # Roofline of the dominant kernel: the d=3 launch of spreading or
    # interpolation (one launch covers both d=3 windows). Algorithmic work of
    # one launch: one FMA per tap, point and RHS = 2 flop x n x R x sum of
    # (2s)^3 over the d=3 windows; its average duration comes from the
    # library's CUDA events around each launch on the launching stream.
    dom = max(("spread", "interp"), key=lambda s: prof[s]["ms_by_dim"][3])
    launch_ms = prof[dom]["ms_by_dim"][3] / max(1, prof[dom]["timed_by_dim"][3])
    taps3 = sum((2 * w.cutoff) ** len(win) for win in w.windows if len(win) == 3)
    flops_launch = 2.0 * w.n * R * taps3
    achieved = flops_launch / (launch_ms / 1e3) / 1e12
    clocks = clk.summary()
    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * 2070e6 / 1e12   # FP32 FMA at max SM clock
    traffic = measured_traffic(f"k_{dom}", w.n, R)

    # end-to-end through the C ABI with host buffers
    Vh = torch.tensor(w.V, dtype=torch.float32).pin_memory()
    Oh = torch.empty_like(Vh).pin_memory()
    for k in range(2):
        V.copy_(Vh, non_blocking=True)
        step(k)
        Oh.copy_(Out, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    e0.record(stream)
    for k in range(args.steps):
        V.copy_(Vh, non_blocking=True)
        step(args.warmup + k)
        Oh.copy_(Out, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([e2e_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t)
    e2e = world * R * args.steps / (e2e_ms / 1e3)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, info = oracle_mvms_per_s(w, target_s=args.ref_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"oracle truncated sum on the first {info['points']} points, 1 RHS, "
                         f"{info['seconds']:.1f} s, scaled linearly to n={N_POINTS}"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic", "config": workload_config(w.n),
                "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": int(Vh.numel() * 4),
                        "d2h_bytes_per_step": int(Oh.numel() * 4)},
                "gpu_launches": int(round(launches_per_step * args.steps)),
                "roofline": {"bound": "alu", "kernel": f"k_{dom}<float, 3, 5, 32>",
                             "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak, "traffic": traffic,
                             "launch_ms": launch_ms, "flop_per_launch": flops_launch,
                             "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz "
                                            "(nominal maximum clock)"},
                "stages_ms_per_step": {s: prof[s]["ms"] / args.steps for s in prof},
                "stage_launches_per_step": {s: prof[s]["launches"] / args.steps for s in prof},
                "clocks": clocks, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--ref-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
