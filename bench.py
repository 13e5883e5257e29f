#!/usr/bin/env python
"""Benchmark of the CAC-MFZ-CDP solver on one GB300 (or N replicas).

One step = one complete solve of the 64-trial workload (N = 2000, M = 1200,
200 nonzeros, noise 0.01, lambda = 0.03, 30 outer iterations x 2000 Euler steps,
FP32): Gram formation, every outer iteration (persistent Euler kernel + refit),
the objective of every trial and the kept trial.

Prints one JSON line.  `value` is reconstructions/s over all ranks with A and y
already in HBM (CUDA events on the library's stream, L2 flushed between steps);
`e2e` is the same metric through the C ABI from pinned host buffers, host<->device
copies included.  `--impl reference` times the FP64 CPU oracle on a bounded
sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import cs_inputs  # noqa: E402

METRIC = "solved reconstructions/s and Euler spin-steps/s at oracle RMSE; p50/p99 latency; %roofline"
WORKLOAD = "trials64_n2000_fp32"
L2_FLUSH_BYTES = 512 << 20


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_simt_peak_tflops(sm_mhz, num_sms=152):
    """FP32 FMA throughput: SMs x 128 FP32 lanes x 2 flop x SM clock."""
    return num_sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def recorded_traffic(kernel_src):
    """DRAM bytes per Euler launch from the committed ncu summary, if it was taken on
    the current kernel source (its sha256 is recorded beside the figure)."""
    path = os.path.join(ROOT, "profiles", "euler_kernel_trials64_n2000.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    h = re.search(r"euler_source_sha256:\s*([0-9a-f]{64})", text)
    if not m or not h:
        return None
    sha = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()
    return float(m.group(1)) if sha == h.group(1) else None


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples taken while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        if self.proc is None:
            return None
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------ CPU oracle timing
def oracle_sample(w, target_s=12.0, min_steps=10):
    """Time the FP64 oracle on the first Euler steps of the first outer iteration of
    the workload (all trials) for about target_s seconds, and extrapolate one whole
    solve: the per-step cost comes from two calibration runs of different length
    (their difference removes the fixed cost of the Gram matrix and the refit)."""
    import numpy as np  # noqa: F401
    import oracle

    inst = cs_inputs.workload_instance(w)
    keys = {f.name for f in __import__("dataclasses").fields(oracle.Params)}
    prm = oracle.Params(**{k: v for k, v in w.items() if k in keys})
    prm.n_outer = 1

    def run(steps):
        t0 = time.perf_counter()
        oracle.solve(inst.A, inst.y, inst.lam, prm, trials=w["trials"], max_steps=steps)
        return time.perf_counter() - t0

    n1, n2 = min_steps, min(w["n_steps"], 12 * min_steps)
    t1 = run(n1)
    t2 = run(n2)
    per_step = max((t2 - t1) / max(n2 - n1, 1), 1e-6)
    fixed = max(t1 - n1 * per_step, 0.0)
    steps = int(max(min_steps, min(w["n_steps"], (target_s - fixed) / per_step)))
    t = run(steps)
    per_step = max((t - fixed) / steps, 1e-9)
    solve_s = fixed + per_step * w["n_outer"] * w["n_steps"]
    return {"value": 1.0 / solve_s, "unit": "reconstructions/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"FP64 NumPy oracle (BLAS on all host cores), first {steps} Euler steps (+ Gram, one refit) "
                       f"of outer iteration 0 of the {w['trials']}-trial N={w['N']} workload, {t:.1f} s; one solve "
                       f"extrapolated as {fixed:.2f} s + {w['n_outer']} x {w['n_steps']} x {per_step * 1e3:.2f} ms"),
            "spin_steps_per_s": w["N"] * w["trials"] / per_step, "seconds": t}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    w = cs_inputs.workload(WORKLOAD)
    vals, secs = [], []
    for i in range(args.warmup + args.steps):
        r = oracle_sample(w, target_s=args.reference_step_s)
        if i >= args.warmup:
            vals.append(r["value"])
            secs.append(r["seconds"])
    v = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "reconstructions/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(w, world),
        "cpu_baseline": {"value": v, "unit": "reconstructions/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": r["sample"]},
        "e2e": {"value": v, "unit": "reconstructions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def config_of(w, world):
    return {"workload": WORKLOAD, "N": w["N"], "M": w["M"], "nnz": w["nnz"], "noise": w["nu"], "lambda": w["lam"],
            "trials": w["trials"], "n_outer": w["n_outer"], "n_steps": w["n_steps"], "dt": w["dt"],
            "field": w["field"], "precision": w["precision"], "refit": w["refit"],
            "parallelism": f"replicas{world}" if world > 1 else "single",
            "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)"}


# ------------------------------------------------------------------ GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--reference-step-s", type=float, default=8.0)
    ap.add_argument("--n-outer", type=int, default=None,
                    help="override the workload's outer iterations (short runs for profiling only)")
    ap.add_argument("--n-steps", type=int, default=None,
                    help="override the workload's Euler steps per run (short runs for profiling only)")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: --warmup below 3 does not meet the timing rules", file=sys.stderr)

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch

    import oracle
    from paper_2405_00366_gb300 import build, cs

    if not os.path.exists(cs.LIB_PATH):
        build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w = cs_inputs.workload(WORKLOAD, seed=cs_inputs.WORKLOADS[WORKLOAD]["seed"] + rank)
    if args.n_outer:
        w["n_outer"] = args.n_outer
    if args.n_steps:
        w["n_steps"] = args.n_steps
    inst = cs_inputs.workload_instance(w)
    prm = cs.params_from_workload(w)
    T = w["trials"]
    stream = torch.cuda.Stream()
    A_dev = torch.from_numpy(inst.A).cuda()
    y_dev = torch.from_numpy(inst.y).cuda()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()

    def one_solve():
        h = cs.cs_problem_create(A_dev, y_dev, inst.lam, stream=stream)
        cs.cs_solve(h, prm, T)
        return h

    def finish(h):
        out = cs.cs_result(h)
        tm = cs.cs_problem_timing(h)
        cs.cs_problem_destroy(h)
        return out, tm

    for _ in range(args.warmup):
        out, tm = finish(one_solve())

    step_ms, euler_ms, launches = [], 0.0, 0
    phase_ms = [0.0, 0.0, 0.0, 0.0]
    results = None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            stream.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            h = one_solve()
            ev1.record(stream)
            results, tm = finish(h)
            step_ms.append(ev0.elapsed_time(ev1))
            euler_ms += tm[0][1]
            launches += tm[1]
            for k in range(4):
                phase_ms[k] += tm[0][k]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    total_s = sum(step_ms) / 1e3
    if dist:
        t = torch.tensor([total_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    value = world * args.steps / total_s

    # end to end through the C ABI from pinned host buffers
    A_pin = torch.from_numpy(inst.A).pin_memory()
    y_pin = torch.from_numpy(inst.y).pin_memory()
    e2e_s = []
    for i in range(max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = cs.cs_problem_create(A_pin, y_pin, inst.lam, stream=stream)
        cs.cs_solve(h, prm, T)
        x_e2e, s_e2e, E_e2e, st_e2e, _ = cs.cs_result(h)
        cs.cs_problem_destroy(h)
        e2e_s.append(time.perf_counter() - t0)
    e2e_total = sum(e2e_s)
    if dist:
        t = torch.tensor([e2e_total], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_total = float(t.item())

    if rank != 0:
        dist.destroy_process_group()
        return 0

    x_hat, sigma_hat, energy, stats, _ = results
    peaks, peak_kind = measured_peaks()
    ck = clocks.summary()
    n_launch_euler = args.steps * w["n_outer"]
    per_launch_s = euler_ms / 1e3 / n_launch_euler
    flops_per_launch = 2.0 * w["N"] * (w["N"] - 1) * T * w["n_steps"]
    achieved = flops_per_launch / per_launch_s / 1e12
    peak = fp32_simt_peak_tflops(float(peaks.get("sm_max_mhz", 2070.0)))
    traffic = recorded_traffic(os.path.join(ROOT, "paper_2405_00366_gb300", "csrc", "euler_impl.cuh"))
    ms_sorted = sorted(step_ms)
    line = {
        "metric": METRIC, "value": value, "unit": "reconstructions/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sum(step_ms) / len(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_of(w, world),
        "spin_steps_per_s": world * w["N"] * T * w["n_outer"] * w["n_steps"] / (total_s / args.steps),
        "latency_ms": {"p50": ms_sorted[len(ms_sorted) // 2],
                       "p99": ms_sorted[min(len(ms_sorted) - 1, int(math.ceil(0.99 * len(ms_sorted))) - 1)]},
        "quality": {"rmse": oracle.rmse(x_hat, inst.x0), "hamming": oracle.hamming_loss(sigma_hat, inst.xi),
                    "energy": energy, "support": int(stats[1])},
        "roofline": {"kernel": "euler_kernel<float, float, MR, STREAM=false, WIDE=true> "
                               "(FP32 G_off resident on chip, packed FMAs)",
                     "bound": "alu", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_source": (f"FP32 FMA: 152 SMs x 128 lanes x 2 flop x {peaks.get('sm_max_mhz', 2070.0)} MHz "
                                     f"(max SM clock, {peak_kind})"),
                     "launch_ms": per_launch_s * 1e3,
                     "flops_per_launch": flops_per_launch},
        "e2e": {"value": world * len(e2e_s) / e2e_total, "unit": "reconstructions/s",
                "h2d_bytes_per_step": (inst.A.size + inst.y.size) * 8,
                "d2h_bytes_per_step": inst.N * 8 + inst.N + 8 + cs.CS_STATS_LEN * 8},
        "gpu_launches": launches,
        "breakdown_ms_per_step": {k: v / args.steps for k, v in zip(["gram", "euler", "refit", "other"], phase_ms)},
        "clocks": ck,
    }
    if world == 1 and not args.no_cpu_baseline:
        cb = oracle_sample(w)
        cb.pop("seconds", None)
        line["cpu_baseline"] = cb
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
