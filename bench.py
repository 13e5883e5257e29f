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

Two further workloads print their own line (not the default):
  --workload batch_uneven_bf16   one step = one batched solve (cs_solve_batch) of
      512 uneven instances (N in [256, 4096], alpha in {0.3, 0.5, 0.7}, a in
      {0.05, 0.1, 0.2}, 16 trials, 30 x 2000 steps, BF16 storage of G_off),
      against plain FP32 solves of the same instances one at a time (cs_solve);
  --workload serve_mix           60 s Poisson request streams (200 requests/s,
      beyond one GPU's capacity, and 2 requests/s) mixing the single FP64 N=200
      shape, the 64-trial N=2000 shape and the uneven BF16 shape 60/30/10 over
      cached problems, through the continuous-batching server, against the same
      requests as plain FP32 solves one at a time; achieved against offered
      rate, p50/p99 latency;
  --workload sweep_random        the paper's random-data experiment: final RMSE
      against sparsity for alpha in {0.6, 0.8} and two noise levels, and the
      RMSE and Hamming loss after every outer iteration, both local fields.
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
# single-problem workloads the main path also measures (--workload): the FP64
# N = 200 single trial (latency-bound) and the MRI-shaped N = 16384 FP16 one
# (G_off streamed from HBM every step)
SINGLE_WORKLOADS = [WORKLOAD, "single_n200_fp64", "mri_n16384_fp16"]
FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 (nominal)
# mma.sync m16n8k16 FP16 (FP32 accumulate) throughput measured on GB300 with a
# register-only loop, 152 CTAs x 8-16 warps: the ceiling of the legacy MMA path
# the tensor-core Euler forms use (tcgen05 would be the 2.25 PFLOP/s nominal)
MMA_SYNC_F16_TFLOPS = 600.0
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


KERNEL_SOURCES = ["euler_kernel.cuh", "kernels_common.cuh", "mma.cuh", "tma.cuh", "common.cuh", "tcgen05.cuh"]


def kernel_source_sha256():
    """sha256 over the device sources of the Euler kernel (in KERNEL_SOURCES order)."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2405_00366_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def recorded_traffic():
    """DRAM bytes per Euler launch from the committed ncu summary, if it was taken on
    the current kernel sources (their sha256 is recorded beside the figure)."""
    path = os.path.join(ROOT, "profiles", "euler_kernel_trials64_n2000.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    h = re.search(r"euler_source_sha256:\s*([0-9a-f]{64})", text)
    if not m or not h:
        return None
    return float(m.group(1)) if kernel_source_sha256() == h.group(1) else None


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


def oracle_sample_single_thread(name, target_s=6.0):
    """oracle_sample on one host core: a child process with every BLAS thread pool
    limited to one thread (the pools are sized when NumPy loads)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "r = bench.oracle_sample(bench.replica_workload(0, %r), target_s=%r); r.pop('seconds', None); "
            "print(json.dumps(r))" % (ROOT, name, target_s))
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        r = json.loads(out.stdout.strip().splitlines()[-1])
        r["cores"] = 1
        r["sample"] = r["sample"].replace("BLAS on all host cores", "BLAS on one core")
        return r
    except Exception as exc:  # reported, never fatal to the GPU measurement
        return {"unavailable": str(exc)[:200]}


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


# ------------------------------------------------------------------ replicas (N > 1)
def replica_workload(rank, name=WORKLOAD):
    """The benchmark workload of one replica: the instance seed is offset by the rank,
    so the N replicas solve N independent problems (no data exchange between ranks)."""
    return cs_inputs.workload(name, seed=cs_inputs.WORKLOADS[name]["seed"] + rank)


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest of the ranks' values of x (the job's time is its slowest rank's)."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, units_per_rank, total_s):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / total_s


def config_of(w, world, name=WORKLOAD, autotune=1):
    return {"workload": name, "N": w["N"], "M": w["M"], "nnz": w["nnz"], "noise": w["nu"], "lambda": w["lam"],
            "trials": w["trials"], "n_outer": w["n_outer"], "n_steps": w["n_steps"], "dt": w["dt"],
            "field": w["field"], "precision": w["precision"], "refit": w["refit"],
            "parallelism": f"replicas{world}" if world > 1 else "single",
            "work_split": "cost model" if (name == "mri_n16384_fp16" or not autotune) else "autotuned",
            "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)"}


# ------------------------------------------------------------------ batched and served workloads
BATCH = dict(n_inst=512, n_min=256, n_max=4096, alphas=[0.3, 0.5, 0.7], sparsities=[0.05, 0.1, 0.2],
             nu=0.01, lam=0.03, trials=16, n_plain=16, seed=17)


def _run_params(cs, precision, **over):
    """Run parameters of the 64-trial workload (30 x 2000 steps) in another precision."""
    w = dict(cs_inputs.WORKLOADS["trials64_n2000_fp32"], precision=precision)
    w.update(over)
    return cs.params_from_workload(w)


def run_batch(args):
    """Batched BF16 solves of uneven instances vs plain FP32 solves one at a time."""
    import numpy as np
    import torch

    import oracle
    from paper_2405_00366_gb300 import build, cs

    if not os.path.exists(cs.LIB_PATH):
        build.build()
    b = dict(BATCH, n_inst=args.batch_instances or BATCH["n_inst"])
    insts = cs_inputs.uneven_batch(b["n_inst"], b["n_min"], b["n_max"], b["alphas"], b["sparsities"], b["nu"],
                                   b["lam"], seed=b["seed"])
    T = b["trials"]
    stream = torch.cuda.Stream()
    dev = [(torch.from_numpy(i.A).cuda(), torch.from_numpy(i.y).cuda()) for i in insts]
    torch.cuda.synchronize()
    over = {k: v for k, v in (("n_outer", args.n_outer), ("n_steps", args.n_steps)) if v}
    prm_b = _run_params(cs, "bf16", autotune=args.autotune, tensor_form=args.tensor_form, **over)
    prm_w = _run_params(cs, "bf16", autotune=args.autotune, tensor_form=args.tensor_form, **dict(over, n_outer=1))
    prm_p = _run_params(cs, "fp32", **over)
    # the problems (G formed once, kept resident) serve every batch
    hs = [cs.cs_problem_create(A, y, i.lam, stream=stream) for (A, y), i in zip(dev, insts)]

    phase = {}

    def batched(prm):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        cs.cs_solve_batch(hs, prm, T)
        ev1.record(stream)
        res = [cs.cs_result(h) for h in hs]
        ms, n = cs.cs_problem_timing(hs[0])  # the batch's phases (event nodes of its graph)
        phase.update(euler_s=ms[1] / 1e3, refit_s=ms[2] / 1e3, other_s=ms[3] / 1e3)
        return ev0.elapsed_time(ev1) / 1e3, res

    # warm-up batches of one outer iteration each: the same launches (and the
    # batch autotuner's timing runs) at a thirtieth of a full batch's time
    for _ in range(max(1, args.warmup)):
        batched(prm_w)
    times, res = [], None
    with ClockSampler(_env_int("LOCAL_RANK", 0)) as clocks:
        for _ in range(max(1, args.steps)):
            t, res = batched(prm_b)
            times.append(t)
        shapes = sorted({(int(r[3][8]), int(r[3][10])) for r in res})
        for h in hs:
            cs.cs_problem_destroy(h)
        # plain FP32 solves, one instance at a time, on n_plain instances spread
        # evenly over the batch's N distribution (every len/n_plain-th by N)
        by_n = sorted(range(len(insts)), key=lambda i: insts[i].N)
        step = len(insts) / b["n_plain"]
        picked = [by_n[int((j + 0.5) * step)] for j in range(b["n_plain"])]
        plain_s, plain_rmse = 0.0, []
        for k in picked:
            (A, y), inst = dev[k], insts[k]
            h = cs.cs_problem_create(A, y, inst.lam, stream=stream)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            cs.cs_solve(h, prm_p, T)
            ev1.record(stream)
            x, sgm, E, st, _ = cs.cs_result(h)
            cs.cs_problem_destroy(h)
            plain_s += ev0.elapsed_time(ev1) / 1e3
            plain_rmse.append(oracle.rmse(x, inst.x0))
    t_b = statistics.median(times)
    rmse_b = [oracle.rmse(r[0], i.x0) for r, i in zip(res, insts)]
    # roofline of the whole batched solve (Euler steps dominate): FP32 FMAs of the
    # coupling products against the FP32 FMA peak, and the G_off bytes streamed
    # (stored tiles, BF16, every step of every instance) against the HBM copy rate
    peaks, peak_kind = measured_peaks()
    steps_all = prm_b.n_outer * prm_b.n_steps
    flops = sum(2.0 * i.N * (i.N - 1) * T for i in insts) * steps_all
    gbytes = sum(((i.N + 127) // 128 * 128) * ((i.N + 31) // 32 * 32) * 2.0 for i in insts) * steps_all
    # rates over the Euler launches' own device time (event nodes around them)
    t_e = phase.get("euler_s") or t_b
    tflops = flops / t_e / 1e12
    gbs = gbytes / t_e / 1e9
    hpeak = float(peaks.get("hbm_gbs", 6800.0))
    form = int(res[0][3][10])
    if form == 6:
        # tcgen05 form: one M = 128, N = 2 x 16 MMA per 16 k and 128-row tile
        # (the two parts of X), against the dense BF16 tensor peak; and the G_off bytes
        tpk = float(peaks.get("bf16_tflops", 1900.0))
        executed = sum(((i.N + 127) // 128 * 128) * ((i.N + 31) // 32 * 32) * 2.0 * 2 * T for i in insts) * steps_all
        tfrac = executed / t_e / 1e12 / tpk
        hbm = gbs / hpeak >= tfrac
        roof = {"kernel": "euler_batch_kernel<__nv_bfloat16, float, 2, PAIR=false, TC=false, TC5=true>",
                "bound": "hbm" if hbm else "tensor", "achieved": gbs if hbm else executed / t_e / 1e12,
                "peak": hpeak if hbm else tpk, "unit": "GB/s" if hbm else "TFLOP/s",
                "frac": max(gbs / hpeak, tfrac), "hbm_frac": gbs / hpeak, "tensor_frac": tfrac,
                "algorithmic_tflops": tflops, "traffic": None,
                "peak_source": f"HBM copy bandwidth and dense BF16 tensor rate ({peak_kind})"}
    elif form == 4:
        # tensor-core form: two FP16/BF16 MMAs per product (the two parts of X) on
        # the mma.sync path, against its measured ceiling; and the G_off bytes
        mma = 2.0 * tflops
        hbm = gbs / hpeak > mma / MMA_SYNC_F16_TFLOPS
        roof = {"kernel": "euler_batch_kernel<__nv_bfloat16, float, 2, PAIR=false, TC=true>",
                "bound": "hbm" if hbm else "tensor", "achieved": gbs if hbm else mma,
                "peak": hpeak if hbm else MMA_SYNC_F16_TFLOPS, "unit": "GB/s" if hbm else "TFLOP/s",
                "frac": max(gbs / hpeak, mma / MMA_SYNC_F16_TFLOPS),
                "tensor_frac_of_mma_sync": mma / MMA_SYNC_F16_TFLOPS, "hbm_frac": gbs / hpeak,
                "algorithmic_tflops": tflops, "traffic": None,
                "peak_source": f"measured mma.sync FP16/BF16 ceiling and HBM copy bandwidth ({peak_kind})"}
    else:
        fpeak = fp32_simt_peak_tflops(float(peaks.get("sm_max_mhz", 2070.0)))
        hbm = gbs / hpeak > tflops / fpeak
        roof = {"kernel": "euler_batch_kernel<__nv_bfloat16, float, 8, PAIR=true, TC=false>",
                "bound": "hbm" if hbm else "alu", "achieved": gbs if hbm else tflops,
                "peak": hpeak if hbm else fpeak, "unit": "GB/s" if hbm else "TFLOP/s",
                "frac": max(gbs / hpeak, tflops / fpeak),
                "alu_frac": tflops / fpeak, "hbm_frac": gbs / hpeak, "traffic": None,
                "peak_source": f"FP32 FMA peak and HBM copy bandwidth ({peak_kind})"}
    v_b = len(insts) / t_b
    v_p = b["n_plain"] / plain_s
    Ns = [i.N for i in insts]
    line = {
        "metric": METRIC, "value": v_b, "unit": "reconstructions/s", "n_gpus": 1, "steps": len(times),
        "warmup": args.warmup, "ms_per_step": t_b * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 storage, f32 compute", "data": "synthetic",
        "config": {"workload": "batch_uneven_bf16", "instances": len(insts), "N_range": [min(Ns), max(Ns)],
                   "alphas": b["alphas"], "sparsities": b["sparsities"], "trials": T, "n_outer": prm_b.n_outer,
                   "n_steps": prm_b.n_steps, "precision": "bf16", "autotune": args.autotune,
                   "warmup_batches": "one outer iteration each",
                   "cluster_sizes_and_forms": shapes, "l2": "inputs larger than L2 (G_off of all instances)"},
        "spin_steps_per_s": sum(Ns) * T * prm_b.n_outer * prm_b.n_steps / t_b,
        "quality": {"rmse_mean": float(np.mean(rmse_b)),
                    "rmse_mean_plain_sample": float(np.mean([rmse_b[k] for k in picked])),
                    "plain_fp32_rmse_mean": float(np.mean(plain_rmse))},
        "plain_fp32": {"value": v_p, "unit": "reconstructions/s",
                       "sample": f"{b['n_plain']} instances spread evenly over the N distribution, solved one at "
                                 f"a time (cs_solve, FP32), "
                                 f"{plain_s:.1f} s"},
        "ratio_vs_plain_fp32": v_b / v_p,
        "breakdown_s_per_step": phase,
        "roofline": dict(roof, time_basis="the Euler launches' device time (breakdown_s_per_step.euler_s)"),
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


SERVE = dict(window_s=60.0, rates=[200.0, 2.0], mix=[0.6, 0.3, 0.1], pools=[64, 8, 32], slots=16, budget_gb=150,
             seed=23)


def _serve_pools(pools):
    """The problems requests are drawn from, per shape (config 1, 2, 3 of the
    benchmark set): (instances, workload dict, trials).  Shape 3 is the uneven
    batch's distribution (N uniform on [256, 4096], BF16, 16 trials)."""
    w1 = dict(cs_inputs.WORKLOADS["single_n200_fp64"])
    w2 = dict(cs_inputs.WORKLOADS["trials64_n2000_fp32"])
    w3 = dict(cs_inputs.WORKLOADS["trials64_n2000_fp32"], precision="bf16", trials=16)
    return [([cs_inputs.random_instance(200, 120, 20, 0.0, 0.05, seed=1000 + k) for k in range(pools[0])], w1, 1),
            ([cs_inputs.random_instance(2000, 1200, 200, 0.01, 0.03, seed=2000 + k) for k in range(pools[1])],
             w2, 64),
            (cs_inputs.uneven_batch(pools[2], 256, 4096, [0.3, 0.5, 0.7], [0.05, 0.1, 0.2], 0.01, 0.03, seed=3000),
             w3, 16)]


def _serve_arrivals(rate, window, mix, pools, seed):
    """A seeded Poisson stream over `window` seconds: (arrival_s, shape, pool index)."""
    rng = __import__("numpy").random.default_rng(seed)
    t, out = 0.0, []
    cum = [sum(mix[:i + 1]) for i in range(len(mix))]
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= window:
            return out
        u = float(rng.random())
        shape = next((i for i, c in enumerate(cum) if u < c), len(mix) - 1)
        out.append((t, shape, int(rng.integers(pools[shape]))))


def _pct(v, q):
    if not v:
        return None
    v = sorted(v)
    return v[min(len(v) - 1, int(math.ceil(q * len(v))) - 1)]


def run_serve(args):
    """Config 5: a Poisson request stream mixing the config 1-3 shapes 60/30/10,
    through the server (HBM-budget admission, G formed once per problem and cached,
    device-resident state) and as plain FP32 solves one at a time in arrival order,
    over the same 60 s window, at the offered rate of 200 requests/s (far above
    what one GPU completes: the achieved rate is the server's capacity) and at a
    sub-saturation rate.  Achieved rate = requests completed within the window /
    window; latencies over the completed requests (at the sub-saturation rate every
    request, the stream drained)."""
    import numpy as np
    import torch

    import oracle
    from paper_2405_00366_gb300 import build, cs

    if not os.path.exists(cs.LIB_PATH):
        build.build()
    cfg = SERVE
    window = args.serve_window or cfg["window_s"]
    pools = _serve_pools(cfg["pools"])
    stream = torch.cuda.Stream()
    handles = [[cs.cs_problem_create(torch.from_numpy(i.A).cuda(), torch.from_numpy(i.y).cuda(), i.lam, stream=stream)
                for i in insts] for insts, _, _ in pools]
    prms = [cs.params_from_workload(w) for _, w, _ in pools]
    prms_plain = [cs.params_from_workload(dict(w, precision="fp32")) for _, w, _ in pools]
    trials = [T for _, _, T in pools]
    budget = int(cfg["budget_gb"]) << 30

    # (time.monotonic is the clock of the server's request times)
    def wait_until(t0, t):
        while True:
            d = t - (time.monotonic() - t0)
            if d <= 0:
                return
            time.sleep(min(d, 0.002))

    # warm-up: every problem once through the server (plans, coupling copies in
    # every precision) and two of each shape as plain solves
    sv = cs.cs_server_create(budget, cfg["slots"])
    try:
        tks = [cs.cs_server_submit(sv, h, prms[s], trials[s]) for s in range(3) for h in handles[s]]
        for tk in tks:
            cs.cs_server_wait(sv, tk, 600000)
            cs.cs_server_result(sv, tk, 1 << 16)
    finally:
        cs.cs_server_destroy(sv)
    for s in range(3):
        for h in handles[s][:2]:
            cs.cs_solve(h, prms_plain[s], trials[s])
            cs.cs_result(h)

    def summary(n_offered, lat, in_window, rmse):
        in_window = int(in_window)
        return dict(offered=n_offered, completed=len(lat), completed_in_window=in_window,
                    achieved_rate=in_window / window,
                    latency_ms={"p50": None if not lat else float(_pct(lat, 0.5)) * 1e3,
                                "p99": None if not lat else float(_pct(lat, 0.99)) * 1e3},
                    rmse_mean=float(np.mean(rmse)) if rmse else None)

    def serve_arm(arr, drain):
        sv = cs.cs_server_create(budget, cfg["slots"])
        tickets = []
        lat, in_window, rmse = [], 0, []
        try:
            t0 = time.monotonic()
            for t, shape, k in arr:
                wait_until(t0, t)
                tickets.append((shape, k, cs.cs_server_submit(sv, handles[shape][k], prms[shape], trials[shape])))
            wait_until(t0, window)
            for shape, k, tk in tickets:
                if drain:
                    cs.cs_server_wait(sv, tk, 3600000)
                elif not cs.cs_server_poll(sv, tk):
                    continue
                x, sg, E, st, tm, _ = cs.cs_server_result(sv, tk, pools[shape][0][k].N)
                lat.append(tm[2] - tm[0])
                in_window += (tm[2] - t0) <= window
                rmse.append(oracle.rmse(x, pools[shape][0][k].x0))
        finally:
            cs.cs_server_destroy(sv)  # queued requests past the window are dropped
        return summary(len(arr), lat, in_window, rmse)

    def plain_arm(arr, drain):
        t0 = time.monotonic()
        lat, in_window, rmse = [], 0, []
        for t, shape, k in arr:
            if not drain and time.monotonic() - t0 >= window:
                break
            wait_until(t0, t)
            h = handles[shape][k]
            cs.cs_solve(h, prms_plain[shape], trials[shape])
            x, sg, E, st, _ = cs.cs_result(h)
            done = time.monotonic() - t0
            lat.append(done - t)
            in_window += done <= window
            rmse.append(oracle.rmse(x, pools[shape][0][k].x0))
        return summary(len(arr), lat, in_window, rmse)

    rates = [args.serve_rate] if args.serve_rate else cfg["rates"]
    results = []
    with ClockSampler(_env_int("LOCAL_RANK", 0)) as clocks:
        for ri, rate in enumerate(rates):
            arr = _serve_arrivals(rate, window, cfg["mix"], cfg["pools"], cfg["seed"] + ri)
            drain = rate < 20.0
            sv_r = serve_arm(arr, drain)
            pl_r = plain_arm(arr, drain)
            results.append(dict(offered_rate=rate, serve=sv_r, plain_fp32=pl_r,
                                ratio_vs_plain_fp32=(sv_r["achieved_rate"] / pl_r["achieved_rate"]
                                                     if pl_r["achieved_rate"] else None)))
    for hs in handles:
        for h in hs:
            cs.cs_problem_destroy(h)
    head = results[0]
    line = {
        "metric": METRIC, "value": head["serve"]["achieved_rate"], "unit": "reconstructions/s", "n_gpus": 1,
        "steps": 1, "warmup": 1, "ms_per_step": window * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "per request (f64 / f32 / bf16 storage)", "data": "synthetic",
        "config": {"workload": "serve_mix", "window_s": window, "rates_per_s": rates, "mix": "60/30/10 of the "
                   "config 1 (N=200 FP64, 1 trial), config 2 (N=2000 FP32, 64 trials) and config 3 (N in "
                   "[256, 4096] BF16, 16 trials) shapes", "problem_pools": cfg["pools"],
                   "slots": cfg["slots"], "hbm_budget_gb": cfg["budget_gb"],
                   "achieved": "requests completed within the window / window",
                   "latency": "over completed requests; the sub-saturation stream is drained"},
        "latency_ms": head["serve"]["latency_ms"],
        "rates": results,
        "ratio_vs_plain_fp32": head["ratio_vs_plain_fp32"],
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def run_sweep(args):
    """The paper's random-data experiment (its RMSE-against-sparsity figure and its
    per-iteration RMSE and Hamming-loss figure), on synthetic data of the same
    shape: N = 2000, alpha in {0.6, 0.8}, (nu, eta_end) in {(0.05, 0.18),
    (0.1, 0.35)}, a in {0.1, 0.2, 0.3, 0.4}, both local fields, `--sweep-datasets`
    random datasets per point, one trial each, the paper's schedules (workload
    paper_random_n2000: sigmoid pump, eta from 0.8 over 52 outer iterations,
    damped Jacobi CDP), FP32.  Prints one JSON line: reconstructions/s over the
    whole sweep, the final RMSE per point, and the mean RMSE and Hamming loss
    after every outer iteration at alpha = 0.6, a = 0.2, nu = 0.05."""
    import numpy as np
    import torch

    import oracle
    from paper_2405_00366_gb300 import build, cs

    if not os.path.exists(cs.LIB_PATH):
        build.build()
    torch.cuda.set_device(0)
    base = cs_inputs.WORKLOADS["paper_random_n2000"]
    N, n_outer = base["N"], base["n_outer"]
    alphas, noise, avals = [0.6, 0.8], [(0.05, 0.18), (0.1, 0.35)], [0.1, 0.2, 0.3, 0.4]
    fields = ["cn", "bn"]
    final, curves = {}, {}
    solves, t_gpu = 0, 0.0
    stream = torch.cuda.Stream()
    for field in fields:
        for alpha in alphas:
            for nu, eta_end in noise:
                for a in avals:
                    rm, hm = [], []
                    for ds in range(args.sweep_datasets):
                        lam = eta_end ** 2 / 2
                        inst = cs_inputs.random_instance(N, int(alpha * N), int(a * N), nu, lam,
                                                         seed=7919 * ds + int(1000 * a) + int(100 * alpha))
                        w = dict(base, field=field, eta_end=eta_end, lam=lam)
                        prm = cs.params_from_workload(w, record_outer=1)
                        A_d = torch.from_numpy(inst.A).cuda()
                        y_d = torch.from_numpy(inst.y).cuda()
                        torch.cuda.synchronize()
                        t0 = time.perf_counter()
                        h = cs.cs_problem_create(A_d, y_d, lam, stream=stream)
                        cs.cs_solve(h, prm, 1)
                        cs.cs_result(h)
                        t_gpu += time.perf_counter() - t0
                        solves += 1
                        sig, R = cs.cs_outer_history(h, n_outer, N, 1)
                        cs.cs_problem_destroy(h)
                        rm.append([oracle.rmse(sig[i, :, 0] * R[i, :, 0], inst.x0) for i in range(n_outer)])
                        hm.append([oracle.hamming_loss(sig[i, :, 0], inst.xi) for i in range(n_outer)])
                    key = f"{field}/alpha={alpha}/nu={nu}/a={a}"
                    final[key] = {"rmse": float(np.mean([r[-1] for r in rm])),
                                  "hamming": float(np.mean([h[-1] for h in hm]))}
                    if alpha == 0.6 and nu == 0.05 and a == 0.2:
                        curves[field] = {"rmse": np.mean(rm, axis=0).tolist(), "hamming": np.mean(hm, axis=0).tolist()}
    line = {
        "metric": METRIC, "value": solves / t_gpu, "unit": "reconstructions/s", "n_gpus": 1, "steps": solves,
        "warmup": 0, "ms_per_step": 1e3 * t_gpu / solves, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "sweep_random", "N": N, "alphas": alphas, "nu_eta_end": noise, "a": avals,
                   "fields": fields, "datasets_per_point": args.sweep_datasets, "trials": 1, "n_outer": n_outer,
                   "n_steps": base["n_steps"], "dt": base["dt"], "pump": "sigmoid d=0.4", "refit": "jacobi 0.1 x 100",
                   "timing": "host clock around create + solve + result of each solve"},
        "sweep": {"final": final, "per_iteration_alpha0.6_a0.2_nu0.05": curves},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tensor-form", type=int, choices=[0, 1, 2, 3, 4], default=0,
                    help="cs_params.tensor_form: 0 planner, 1 FMA forms only, 2 tensor cores only, 3 mma.sync forms only, 4 tcgen05 form only")
    ap.add_argument("--reference-step-s", type=float, default=8.0)
    ap.add_argument("--autotune", type=int, choices=[0, 1], default=1,
                    help="cs_params.autotune of the main workloads (0 for profiling: under ncu the tuning runs' "
                         "timings are distorted, so the cost model's split is the one to capture)")
    ap.add_argument("--n-outer", type=int, default=None,
                    help="override the workload's outer iterations (short runs for profiling only)")
    ap.add_argument("--n-steps", type=int, default=None,
                    help="override the workload's Euler steps per run (short runs for profiling only)")
    ap.add_argument("--workload", choices=SINGLE_WORKLOADS + ["batch_uneven_bf16", "serve_mix", "sweep_random"],
                    default=WORKLOAD)
    ap.add_argument("--sweep-datasets", type=int, default=2, help="random datasets per point of the sweep workload")
    ap.add_argument("--serve-window", type=float, default=None, help="seconds of request arrivals (serve_mix)")
    ap.add_argument("--serve-rate", type=float, default=None, help="one offered rate instead of 200 and 2 per s")
    ap.add_argument("--batch-instances", type=int, default=None,
                    help="instances of the batched workload (smaller batches for profiling only)")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: --warmup below 3 does not meet the timing rules", file=sys.stderr)

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batch_uneven_bf16":
        return run_batch(args)
    if args.workload == "serve_mix":
        return run_serve(args)
    if args.workload == "sweep_random":
        return run_sweep(args)

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

    name = args.workload
    w = replica_workload(rank, name)
    if args.n_outer:
        w["n_outer"] = args.n_outer
    if args.n_steps:
        w["n_steps"] = args.n_steps
    inst = cs_inputs.workload_instance(w)
    # work split timed on this GPU during the warm-up (the MRI-shaped problem keeps
    # the cost model's streamed split: its tuning runs would take seconds)
    tune = 0 if name == "mri_n16384_fp16" else args.autotune
    prm = cs.params_from_workload(w, autotune=tune, tensor_form=args.tensor_form)
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
    total_s = max_over_ranks(sum(step_ms) / 1e3, dist, "cuda")
    value = job_value(world, args.steps, total_s)

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
    e2e_total = max_over_ranks(sum(e2e_s), dist, "cuda")

    if rank != 0:
        dist.destroy_process_group()
        return 0

    x_hat, sigma_hat, energy, stats, _ = results
    form = int(stats[10])  # 0 / 1 FMA forms, 2 tensor cores (mma.sync), 5 tensor cores (tcgen05)
    peaks, peak_kind = measured_peaks()
    ck = clocks.summary()
    n_launch_euler = args.steps * w["n_outer"]
    per_launch_s = euler_ms / 1e3 / n_launch_euler
    flops_per_launch = 2.0 * w["N"] * (w["N"] - 1) * T * w["n_steps"]
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    if name == "mri_n16384_fp16":
        # every step streams the stored G_off (Npad x Npad FP16) from HBM
        npad = (w["N"] + 31) // 32 * 32
        bytes_per_launch = float(npad) * npad * 2 * w["n_steps"]
        roof = {"kernel": "euler_kernel<__half, float, MR, STREAM=true, WIDE=true, TC=%s> (FP16 G_off streamed%s)"
                          % (("true", ", mma.sync") if form == 2 else ("false", ", packed FMAs")),
                "bound": "hbm", "achieved": bytes_per_launch / per_launch_s / 1e9,
                "peak": float(peaks.get("hbm_gbs", 6800.0)), "unit": "GB/s",
                "peak_source": f"HBM copy bandwidth ({peak_kind})", "bytes_per_launch": bytes_per_launch,
                "bytes_note": "full stored matrix; the symmetric minimum is N(N-1)/2 x 2 B per step",
                "traffic": None}
    elif name == "single_n200_fp64":
        roof = {"kernel": "euler_kernel<double, double, MR, STREAM=false, WIDE=false> (FP64, latency-bound)",
                "bound": "alu", "achieved": flops_per_launch / per_launch_s / 1e12,
                "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                "peak_source": "GB300 FP64 nominal; a 1000-step dependent chain of 200 x 200 products: "
                               "the step latency is the figure of merit",
                "us_per_step": per_launch_s * 1e6 / w["n_steps"], "flops_per_launch": flops_per_launch,
                "traffic": None}
    elif form == 5:
        # FP32 problem on the tcgen05 tensor cores: one M = 128 MMA per 16-k block
        # on the stacked FP16 parts of G (64 rows hi over lo) and X (hi over lo);
        # the roofline is the product's own precision (FP32), the executed MMA
        # rate against the dense FP16 tensor rate beside it
        achieved = flops_per_launch / per_launch_s / 1e12
        C, ctas = int(stats[8]), int(stats[9])
        npad = (w["N"] + 31) // 32 * 32
        mma_flops = 2.0 * (ctas // max(C, 1)) * (npad // 16) * 128 * (2 * min(T, 64)) * 16 * ((T + 63) // 64)
        tpeak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0)))
        executed = mma_flops * w["n_steps"] / per_launch_s / 1e12
        roof = {"kernel": "euler_kernel<float, float, 1, STREAM=false, WIDE=true, TC=true, TC5=true> "
                          "(FP32 G_off resident on chip as FP16 hi/lo parts, one tcgen05 M=128 MMA per 16-k block, "
                          "TMEM accumulators)",
                "bound": "alu", "achieved": achieved, "peak": fp32_simt_peak_tflops(sm_mhz), "unit": "TFLOP/s",
                "peak_source": f"FP32, the precision of the product: 152 SMs x 128 lanes x 2 flop x {sm_mhz} MHz "
                               f"(max SM clock, {peak_kind})",
                "flops_per_launch": flops_per_launch,
                "tensor_pipe": {"executed_tflops": executed, "peak": tpeak, "frac": executed / tpeak,
                                "peak_source": f"dense BF16 (= FP16) tensor rate, cuBLAS sustained ({peak_kind})",
                                "executed_flops_per_step": mma_flops},
                "traffic": recorded_traffic()}
    elif form == 2:
        # FP32 problem on the tensor cores: three FP16 MMAs per tile on split
        # operands; the algorithmic figure counts the FP32 products once
        peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0)))
        achieved = flops_per_launch / per_launch_s / 1e12
        roof = {"kernel": "euler_kernel<float, float, MR, STREAM=false, WIDE=true, TC=true> "
                          "(FP32 G_off resident on chip, three FP16 mma.sync per tile)",
                "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "peak_source": f"dense BF16 (= FP16) tensor rate, cuBLAS sustained ({peak_kind}); "
                               "the kernel is timed inside a seconds-long solve",
                "flops_per_launch": flops_per_launch,
                "mma_tflops_executed": 3.0 * achieved,
                "mma_sync_peak_tflops": MMA_SYNC_F16_TFLOPS,
                "frac_of_mma_sync_peak": 3.0 * achieved / MMA_SYNC_F16_TFLOPS,
                "traffic": recorded_traffic()}
    else:
        roof = {"kernel": "euler_kernel<float, float, MR, STREAM=false, WIDE=true, TC=false> "
                          "(FP32 G_off resident on chip, packed FMAs)",
                "bound": "alu", "achieved": flops_per_launch / per_launch_s / 1e12,
                "peak": fp32_simt_peak_tflops(sm_mhz), "unit": "TFLOP/s",
                "peak_source": f"FP32 FMA: 152 SMs x 128 lanes x 2 flop x {sm_mhz} MHz (max SM clock, {peak_kind})",
                "flops_per_launch": flops_per_launch, "traffic": recorded_traffic()}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["launch_ms"] = per_launch_s * 1e3
    roof["form"] = form
    roof["plan"] = {"cluster": int(stats[8]), "ctas": int(stats[9])}
    roof["us_per_euler_step"] = per_launch_s * 1e6 / w["n_steps"]
    ms_sorted = sorted(step_ms)
    line = {
        "metric": METRIC, "value": value, "unit": "reconstructions/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sum(step_ms) / len(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"single_n200_fp64": "f64", "mri_n16384_fp16": "f16 storage, f32 compute"}.get(name, "f32"),
        "data": "synthetic", "config": config_of(w, world, name, args.autotune),
        "spin_steps_per_s": world * w["N"] * T * w["n_outer"] * w["n_steps"] / (total_s / args.steps),
        "latency_ms": {"p50": ms_sorted[len(ms_sorted) // 2],
                       "p99": ms_sorted[min(len(ms_sorted) - 1, int(math.ceil(0.99 * len(ms_sorted))) - 1)]},
        "quality": {"rmse": oracle.rmse(x_hat, inst.x0), "hamming": oracle.hamming_loss(sigma_hat, inst.xi),
                    "energy": energy, "support": int(stats[1])},
        "roofline": roof,
        "e2e": {"value": job_value(world, len(e2e_s), e2e_total), "unit": "reconstructions/s",
                "h2d_bytes_per_step": (inst.A.size + inst.y.size) * 8,
                "d2h_bytes_per_step": inst.N * 8 + inst.N + 8 + cs.CS_STATS_LEN * 8},
        "gpu_launches": launches,
        "host_submissions_per_step": int(tm[0][4]),
        "breakdown_ms_per_step": {k: v / args.steps for k, v in zip(["gram", "euler", "refit", "other"], phase_ms)},
        "clocks": ck,
    }
    if world == 1 and not args.no_cpu_baseline:
        cb = oracle_sample(w)
        cb.pop("seconds", None)
        cb["single_thread"] = oracle_sample_single_thread(name)
        line["cpu_baseline"] = cb
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
