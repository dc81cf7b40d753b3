#!/usr/bin/env python3
"""Benchmark: Kalman-MPC control steps per second on one B300 (or N replicas).

A step is one receding-horizon control step of Algorithm 1 -- ensemble
initialisation, H predictions through the CNN surrogate and H ensemble Kalman
analyses, then the plant update with the smoothed control -- on the
64 x 64 working workload (l = 8, CNN 2-32-32-1, N = 256 members, H = 10),
noise drawn on the device (Philox).  Inputs are resident in HBM when the timed
region starts; L2 is flushed (a 256 MB write) between timed steps, outside the
per-step events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl oic|reference]

Under torchrun each rank runs an independent replica (the problems are
independent; there is no collective on the data path) and rank 0 prints one
JSON line with the whole-job throughput.  `--impl reference` times the FP64
CPU oracle (the only reference this method has) on the host cores.
"""
from __future__ import annotations

import argparse
import collections
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "EnKS control steps/s (N×H CNN steps/s); p50/p99 solve latency vs plain FP32"
UNIT = "control steps/s"
SM_COUNT = 148
FP32_LANES_PER_SM = 128


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        p["source"] = "measured"
    except (OSError, ValueError):
        p = {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0,
             "sm_max_mhz": 2032.0, "source": "fallback"}
    return p


def fp32_alu_peak_tflops(sm_mhz):
    """FFMA peak: 148 SMs x 128 FP32 lanes x 2 flops x SM clock."""
    return SM_COUNT * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


# ------------------------------------------------------------- workload math
def conv_layer_flops(wl, cin, cout):
    return 2.0 * 9 * wl.n * wl.m * cin * cout


def cnn_flops_per_member_step(wl):
    f = 2.0 * wl.n * wl.l * wl.m                       # B U
    for cin, cout in zip(wl.channels[:-1], wl.channels[1:]):
        f += conv_layer_flops(wl, cin, cout)
    return f


def stage_work(wl, stage):
    """Algorithmic work of ONE launch of `stage` at the working size:
    (amount, unit, bound)."""
    N = wl.N
    if stage == "conv_hidden":
        c = wl.channels[1]
        return conv_layer_flops(wl, c, c) * N, "flop", "alu"
    if stage == "conv_first":
        return conv_layer_flops(wl, 2, wl.channels[1]) * N, "flop", "alu"
    if stage == "conv_out":
        return conv_layer_flops(wl, wl.channels[-2], 1) * N, "flop", "alu"
    if stage == "cnn_fused":
        # whole CNN step; the hidden layer (the bulk of the flops) runs on the
        # fp16 tensor pipe as three products per FP32 product
        return cnn_flops_per_member_step(wl) * N, "flop", "tensor"
    if stage == "cnn_bf16":
        # whole CNN step in BF16 (one kernel per layer), one product per product
        return cnn_flops_per_member_step(wl) * N, "flop", "tensor"
    return None


def kernel_traffic(stage, wl=None):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source of the kernel and on this workload (else None).  A
    line captured on fewer members (`members=`) is scaled by N / members: the
    kernels stream every member's rows once, so their traffic grows in
    proportion to the members."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    src_files = {"conv_hidden": "conv_tc.cu", "conv_first": "cnn_kernels.cu",
                 "conv_out": "cnn_kernels.cu", "cnn_fused": "cnn_fused_tc.cu", "cnn_bf16": "conv_bf16_tc.cu"}
    f = src_files.get(stage)
    if f is None:
        return None
    src = os.path.join(ROOT, "paper_2410_09663_b300", "csrc", f)
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    for line in open(path):
        if line.startswith("#"):
            continue
        parts = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        if parts.get("stage") != stage or parts.get("src_sha") != sha:
            continue
        if wl is not None and "workload" in parts and parts["workload"] != wl.name:
            continue
        scale = wl.N / float(parts["members"]) if (wl is not None and "members" in parts) else 1.0
        return float(parts["dram_bytes_per_launch"]) * scale
    return None
    src_files = {"conv_hidden": "conv_tc.cu", "conv_first": "cnn_kernels.cu",
                 "conv_out": "cnn_kernels.cu", "cnn_fused": "cnn_fused_tc.cu"}
    f = src_files.get(stage)
    if f is None:
        return None
    src = os.path.join(ROOT, "paper_2410_09663_b300", "csrc", f)
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    for line in open(path):
        parts = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        if parts.get("stage") == stage and parts.get("src_sha") == sha:
            return float(parts["dram_bytes_per_launch"])
    return None


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- the oracle
def oracle_step_seconds(wl, N_sample, k=0, noise=None):
    """Wall time of one control step of the FP64 oracle with N_sample members:
    one horizon solve from X_0 with the reference window of time k, then the
    plant step.  `noise` (the solve's random numbers) defaults to the device
    Philox stream of solve k, so the oracle consumes the same numbers as the
    CUDA path; it is drawn before the clock starts."""
    import oracle
    w = wl.with_(N=N_sample)
    net = oracle.Net(w.n, w.m, w.l, w.channels, w.weights(), w.B(), w.residual_scale)
    xr = w.X_ref_all(k + 1)
    if noise is None:
        from paper_2410_09663_b300 import workloads as W
        noise = W.philox_noise(w, solve=k)
    nz = np.asarray(noise, np.float32)[None]
    cons = oracle.Cons(w.cons.Gx, w.cons.Gu, w.cons.h, w.cons.alpha, w.cons.beta) if w.cons is not None else None
    t0 = time.perf_counter()
    oracle.run(net, w.N, w.H, 1, w.X0(), w.U_init(), xr[k:], w.U_ref(), nz, cons)
    return time.perf_counter() - t0


def host_threads():
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else (len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
                             else os.cpu_count())


def oracle_sample_members(wl, budget_s):
    """Members per timed oracle step: the whole ensemble when one full control
    step fits in `budget_s`, else the largest sample that does (the oracle's
    cost is linear in N; a tiny sample is dominated by fixed costs, so the
    sample is grown toward the budget rather than extrapolated once)."""
    n0 = max(8, -(-(wl.n + wl.l) // wl.m) + 2)   # (N - 1) m >= n + l keeps Sigma^Y definite
    n_s, t = n0, oracle_step_seconds(wl, n0)
    for _ in range(4):
        if n_s >= wl.N or t * wl.N / n_s <= budget_s or t >= 0.5 * budget_s:
            break
        n_s = int(min(wl.N, max(n_s + 1, n_s * budget_s / max(t, 1e-3))))
        t = oracle_step_seconds(wl, n_s)
    if t * wl.N / n_s <= budget_s:
        n_s = wl.N
    return n_s


def sample_text(wl, n_s, t_step):
    if n_s == wl.N:
        return (f"one whole control step (solve of {wl.N} members over H = {wl.H} + plant step) per timed "
                f"step, {t_step:.2f} s each; no extrapolation")
    return (f"one control step of {n_s} of {wl.N} members per timed step ({t_step:.2f} s), EXTRAPOLATED to "
            f"the full ensemble by {n_s}/{wl.N} (the oracle's cost is linear in N)")


def cpu_baseline(wl, budget_s=30.0):
    """The oracle as it stands on the host's cores: one control step of the
    same workload with the same device-Philox noise, measured the same way as
    the reference arm (whole ensemble where it fits the budget)."""
    n_s = oracle_sample_members(wl, budget_s)
    t = oracle_step_seconds(wl, n_s)
    value = (n_s / wl.N) / t
    return {"value": value, "unit": UNIT, "cores": host_threads(), "kind": "oracle",
            "extrapolated": n_s != wl.N, "sample": sample_text(wl, n_s, t)}


def reference_config(wl):
    """The workload keys the CUDA arm reports, with what differs in the oracle's
    implementation (not in the problem) stated beside them."""
    return config_dict(wl, {"precision": "fp64 (oracle)", "l2": "n/a (CPU)",
                            "history": "full smoothed history [X; U; dU] blocks k..k+H (the dropped rows do not "
                                       "change the kept rows' results)"})


def run_reference(args, wl):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2410_09663_b300 import workloads as W
    # every step: the whole ensemble if one control step takes <= 8 s, so
    # that --steps 20 --warmup 5 ends within a few minutes
    n_s = oracle_sample_members(wl, 8.0)
    w = wl.with_(N=n_s)
    cyc = min(5, wl.S)
    noises = [W.philox_noise(w, solve=k) for k in range(cyc)]
    for i in range(args.warmup):
        oracle_step_seconds(wl, n_s, k=i % cyc, noise=noises[i % cyc])
    times = [oracle_step_seconds(wl, n_s, k=i % cyc, noise=noises[i % cyc]) for i in range(args.steps)]
    t = sum(times)
    value = args.steps * (n_s / wl.N) / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / args.steps * wl.N / n_s, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": reference_config(wl),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": host_threads(), "kind": "oracle",
                             "extrapolated": n_s != wl.N,
                             "sample": sample_text(wl, n_s, t / args.steps) +
                             f"; control steps k = 0..{cyc - 1} in turn, from X_0; the device Philox "
                             f"stream's numbers, drawn on the host before each step's clock starts"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def replica_workload(wl, rank):
    """Each rank solves its own problem: the same workload, seed offset by
    the rank (no data is shared between ranks)."""
    return wl.with_(seed=wl.seed + rank)


def max_over_ranks(times, world, device=None):
    """Element-wise maximum of `times` over the ranks of the default process
    group (the job's time is that of its slowest replica)."""
    if world <= 1:
        return [float(t) for t in times]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x) for x in times], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def job_value(steps_per_rank, world, t_slowest):
    """Whole-job throughput: the control steps of every rank over the slowest
    rank's time (weak scaling: per-rank work is fixed)."""
    return world * steps_per_rank / t_slowest


def config_dict(wl, extra=None):
    d = {"workload": wl.name, "n": wl.n, "m": wl.m, "l": wl.l, "N": wl.N, "H": wl.H,
         "cnn": "-".join(str(c) for c in wl.channels), "precision": "fp32",
         "noise": "philox-4x32-10 (seed, solve, element)", "history": "U blocks + current X",
         "l2": "flushed between timed steps (256 MB write)"}
    if wl.cons is not None:
        d["constraint"] = ("|U| <= %g on every control entry: %d softplus-barrier rows (alpha %g, beta %g, "
                           "sigma_z %g), p = %d observed rows" % (float(wl.cons.h[0]), wl.c, wl.cons.alpha,
                                                                 wl.cons.beta, wl.cons.sigma_z, wl.p))
    if extra:
        d.update(extra)
    return d


# ------------------------------------------------------------------- our arm
def run_oic(args, wl):
    import torch
    import torch.distributed as dist
    import paper_2410_09663_b300 as oic

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    wl = replica_workload(wl, rank)                      # independent replica per rank
    w, b = wl.flat_weights()
    mixed = args.precision == "mixed"
    cfg = oic.config_from_workload(wl, noise_mode=oic.OIC_NOISE_PHILOX,
                                   precision=oic.OIC_PREC_MIXED if mixed else oic.OIC_PREC_FP32)
    stream = torch.cuda.Stream(device=dev)
    s = oic.Solver(cfg, w, b, wl.B(), device=dev, stream=stream, constraints=wl.cons)

    n_break = min(10, args.steps)                       # instrumented breakdown steps
    S_ref = args.steps + args.warmup + n_break + 5
    xr_all = torch.from_numpy(wl.X_ref_all(S_ref)).to(dev)
    ur = torch.from_numpy(wl.U_ref()).to(dev)
    X0 = torch.from_numpy(wl.X0()).to(dev)
    U0 = torch.from_numpy(wl.U_init()).to(dev)
    u_out = torch.zeros(wl.l, wl.m, device=dev)
    x_out = torch.zeros(wl.n, wl.m, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    H = wl.H

    def window(k):
        return xr_all[k:k + H + 1]

    with torch.cuda.stream(stream):
        s.oic_reset(X0, U0)
        for k in range(args.warmup):
            s.oic_step(window(k), ur, None, u_out, x_out)
        stream.synchronize()
        # stage breakdown: a few steps with every stage bracketed by events
        # (untimed); its largest stage is the one the timed region brackets
        s.oic_profile_begin(max_launches=256 * n_break)
        for i in range(n_break):
            s.oic_step(window(args.warmup + i), ur, None, u_out, x_out)
        breakdown = s.oic_profile_end()
        dominant = max(breakdown, key=lambda k: breakdown[k][0]) if breakdown else None
        # the timed region brackets one launch of the dominant stage per step
        # (the middle one of its per_step launches, all of the same size): an
        # event record between two kernels keeps the second from starting
        # early, so bracketing all of them would slow the step it measures
        per_step_l = max(1, round(breakdown[dominant][1] / n_break)) if dominant is not None else 1
        sample = (per_step_l, per_step_l // 2)
        if dominant is not None:                        # capture the timed variant's graph
            s.oic_profile_begin(stages=[dominant], max_launches=128)
            s.oic_profile_sample(*sample)
            s.oic_step(window(args.warmup + n_break), ur, None, u_out, x_out)
            s.oic_profile_end()

        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        launches0 = oic.oic_launch_count()
        if dominant is not None:
            s.oic_profile_begin(stages=[dominant], max_launches=128 * args.steps)
            s.oic_profile_sample(*sample)
        with ClockSampler(local) as clk:
            t0 = time.perf_counter()
            for i in range(args.steps):
                k = args.warmup + n_break + 1 + i
                flush.fill_(float(i))
                ev[i][0].record(stream)
                s.oic_step(window(k), ur, None, u_out, x_out)
                ev[i][1].record(stream)
            stream.synchronize()
            wall = time.perf_counter() - t0
        prof = s.oic_profile_end() if dominant is not None else {}
        launches = oic.oic_launch_count() - launches0
        s.oic_sync()
        per_step = [a.elapsed_time(c) for a, c in ev]
        # the same kind of step launched kernel by kernel instead of replayed
        # from its graph: the launch overhead the graph removes (not part of
        # the value above)
        n_eager = min(args.steps, 20)
        ev_e = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(n_eager)]
        os.environ["OIC_NO_GRAPH"] = "1"
        try:
            if dominant is not None:                    # the same event brackets as the timed graph
                s.oic_profile_begin(stages=[dominant], max_launches=128 * n_eager)
                s.oic_profile_sample(*sample)
            for i in range(n_eager):
                flush.fill_(float(i))
                ev_e[i][0].record(stream)
                s.oic_step(window(args.warmup + i), ur, None, u_out, x_out)
                ev_e[i][1].record(stream)
            stream.synchronize()
            if dominant is not None:
                s.oic_profile_end()
        finally:
            del os.environ["OIC_NO_GRAPH"]
        eager_ms = sum(a.elapsed_time(c) for a, c in ev_e) / max(n_eager, 1)
    t_dev = sum(per_step) / 1e3                         # seconds of device time in steps

    # e2e: the host-pointer entry point, pinned host buffers, copies inside
    xr_host = torch.from_numpy(wl.X_ref_all(S_ref)).pin_memory()
    ur_host = torch.from_numpy(wl.U_ref()).pin_memory()
    ua_host = torch.zeros(wl.l, wl.m).pin_memory()
    xn_host = torch.zeros(wl.n, wl.m).pin_memory()
    s.oic_reset_host(wl.X0(), wl.U_init())
    for k in range(min(3, args.warmup)):
        s.oic_step_host_ptr(xr_host[k].data_ptr(), ur_host.data_ptr(), None, ua_host.data_ptr(),
                            xn_host.data_ptr())
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for i in range(args.steps):
        k = args.warmup + i
        s.oic_step_host_ptr(xr_host[k].data_ptr(), ur_host.data_ptr(), None, ua_host.data_ptr(),
                            xn_host.data_ptr())
    torch.cuda.synchronize(dev)
    t_e2e = time.perf_counter() - t0
    h2d = (H + 1) * wl.n * wl.m * 4 + wl.l * wl.m * 4
    d2h = wl.l * wl.m * 4 + wl.n * wl.m * 4

    t_dev, t_e2e = max_over_ranks([t_dev, t_e2e], world, dev)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    peaks = load_peaks()
    clocks = clk.summary()
    total_ms = {k: v[0] for k, v in breakdown.items()}
    roof = None
    if dominant is not None and dominant in prof:
        work = stage_work(wl, dominant)
        ms, n_l = prof[dominant]
        if work is not None and n_l > 0:
            amount, unit, bound = work
            avg_s = ms / 1e3 / n_l
            if bound == "tensor":
                # a kernel timed inside a region shorter than a second runs at
                # the burst rate; a seconds-long region meets the power cap
                sustained = wall >= 1.0
                key = "bf16_tflops_sustained" if sustained else "bf16_tflops"
                peak = peaks.get(key, 1400.0 if sustained else 1800.0)
                ach = amount / avg_s / 1e12
                roof = {"bound": "tensor", "kernel": dominant, "achieved": ach, "peak": peak,
                        "unit": "TFLOP/s", "frac": ach / peak,
                        "peak_kind": "sustained" if sustained else "burst",
                        "peak_source": "%s bf16 dense %s (%s; timed region %.3f s; fp16 runs at the bf16 rate)"
                                       % (peaks["source"], "sustained" if sustained else "burst", key, wall),
                        "traffic": kernel_traffic(dominant, wl),
                        "algorithmic_per_launch": amount, "launches": n_l,
                        "avg_launch_ms": avg_s * 1e3,
                        "sampled": "launch %d of the %d %s launches of each timed step, bracketed by CUDA "
                                   "events" % (sample[1], sample[0], dominant),
                        "fp32_ffma_equiv_frac": ach / fp32_alu_peak_tflops(peaks.get("sm_max_mhz", 2032.0)),
                        "note": ("BF16 operands, FP32 accumulation" if dominant == "cnn_bf16" else
                                 "algorithmic FP32 flops; the tensor pipe executes 3 fp16 products each")}
            elif bound == "alu":
                peak = fp32_alu_peak_tflops(peaks.get("sm_max_mhz", 2032.0))
                roof = {"bound": "alu", "kernel": dominant, "achieved": amount / avg_s / 1e12,
                        "peak": peak, "unit": "TFLOP/s",
                        "frac": amount / avg_s / 1e12 / peak,
                        "peak_source": "derived: 148 SM x 128 FP32 lanes x 2 x %.0f MHz (%s sm_max_mhz)"
                                       % (peaks.get("sm_max_mhz", 2032.0), peaks["source"]),
                        "traffic": kernel_traffic(dominant, wl),
                        "algorithmic_per_launch": amount, "launches": n_l,
                        "avg_launch_ms": avg_s * 1e3,
                        "sampled": "launch %d of the %d %s launches of each timed step, bracketed by CUDA "
                                   "events" % (sample[1], sample[0], dominant)}
    share = {k: round(v / max(sum(total_ms.values()), 1e-12), 4) for k, v in total_ms.items()}
    steps_total = world * args.steps
    value = job_value(args.steps, world, t_dev)
    lat = sorted(per_step)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32+f64" if mixed else "f32", "data": "synthetic",
        "config": config_dict(wl, {
            "parallelism": "replicas" if world > 1 else "single",
            "precision": "mixed: BF16 conv, FP32 covariance, FP64 mean correction and gain" if mixed else "fp32",
            "member_steps_per_s": value * wl.N * wl.H,
            "cnn_tflops": value * wl.N * wl.H * cnn_flops_per_member_step(wl) / 1e12,
            "p50_step_ms": lat[len(lat) // 2], "p99_step_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
            "wall_s_timed_region": wall,
            "launch": "one CUDA graph per control step (events around one %s launch per step)" % dominant,
            "stage_share": share,
            "stage_ms_per_step": {k: v / n_break for k, v in total_ms.items()},
            "stage_breakdown": "%d instrumented steps before the timed region, every stage bracketed "
                               "by CUDA events" % n_break,
            "graph_vs_eager": {"graph_ms_per_step": 1e3 * t_dev / args.steps, "eager_ms_per_step": eager_ms,
                               "eager_steps": n_eager,
                               "note": "eager: the same step launched kernel by kernel (OIC_NO_GRAPH), "
                                       "with the same event brackets around the dominant stage, timed "
                                       "after the graph run"}}),
        "roofline": roof,
        "e2e": {"value": steps_total / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline(wl, budget_s=args.cpu_budget)
        except Exception as e:                          # the GPU line must still print
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": host_threads(),
                                    "kind": "oracle", "sample": f"failed: {e!r}"}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


MIX_METRIC = "aggregate control steps/s over a batch of uneven problems (one batch graph per step)"


def run_mix(args, name):
    """Batched uneven problems: every problem of the mix takes one control
    step per batch step (mixed precision, device noise); value = problems x
    steps / time.  The same problems stepped one after another on one stream
    are timed beside it."""
    import torch
    import torch.distributed as dist
    import paper_2410_09663_b300 as oic
    from paper_2410_09663_b300 import workloads
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wls = workloads.BATCHES[name](seed=2024 + 1000 * rank)
    P_ = len(wls)
    stream = torch.cuda.Stream(device=dev)
    solvers, refs = [], []
    S_ref = args.steps + args.warmup + 8
    with torch.cuda.stream(stream):
        for w in wls:
            wt, bs = w.flat_weights()
            cfg = oic.config_from_workload(w, noise_mode=oic.OIC_NOISE_PHILOX, precision=oic.OIC_PREC_MIXED)
            sv = oic.Solver(cfg, wt, bs, w.B(), device=dev, stream=stream)
            sv.oic_reset(torch.from_numpy(w.X0()).to(dev), torch.from_numpy(w.U_init()).to(dev))
            solvers.append(sv)
            refs.append(torch.from_numpy(w.X_ref_all(S_ref)).to(dev))
        batch = oic.Batch(solvers, stream=stream)
        slots = [sv.oic_io_slots() for sv in solvers]
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

        def fill(k):
            for w, r, (xr, ur, _, _) in zip(wls, refs, slots):
                xr.copy_(r[k:k + w.H + 1])
                ur.zero_()

        def time_batch(bt):
            for k in range(args.warmup):
                fill(k)
                bt.step()
            bt.sync()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize(dev)
            l0 = oic.oic_launch_count()
            with ClockSampler(local) as ck:
                for i in range(args.steps):
                    flush.fill_(float(i))
                    ev[i][0].record(stream)
                    fill(args.warmup + i)
                    bt.step()
                    ev[i][1].record(stream)
                bt.sync()
            return [a.elapsed_time(c) for a, c in ev], oic.oic_launch_count() - l0, ck

        per_step, launches, clk = time_batch(batch)
        t_rule = sum(per_step) / 1e3
        tuned = None
        if args.tune:
            # every problem's plan chosen by the autotuner (timed alone, cached
            # by shape), then the batch graph captured again with those plans
            t0 = time.perf_counter()
            ms_r, ms_t = batch.autotune(reps=2)
            t_tune = time.perf_counter() - t0
            plans = [sv.oic_get_plan()[0] for sv in solvers]
            per_step, launches, clk = time_batch(batch)
            tuned = {"tuner": "oic_batch_autotune: one choice for all problems, timed as whole batch steps",
                     "tuner_ms_rule": ms_r, "tuner_ms_tuned": ms_t,
                     "plans_distinct": len({tuple(sorted(p.items())) for p in plans}),
                     "plan_of_first_problem": plans[0],
                     "tuning_s": t_tune,
                     "rule_value": job_value(P_ * args.steps, world, t_rule),
                     "note": "value is with the tuned plans; rule_value the same batch with the built-in rules"}
        t_batch = sum(per_step) / 1e3
        # the same problems one after another, each through its own step graph
        k_seq = min(args.steps, 3)
        u_outs = [torch.zeros(w.l, w.m, device=dev) for w in wls]
        x_outs = [torch.zeros(w.n, w.m, device=dev) for w in wls]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for i in range(k_seq):
            k = args.warmup + args.steps + i
            for w, r, sv, uo, xo in zip(wls, refs, solvers, u_outs, x_outs):
                sv.oic_step(r[k:k + w.H + 1], torch.zeros(w.l, w.m, device=dev), None, uo, xo)
        e1.record(stream)
        stream.synchronize()
        t_seq = e0.elapsed_time(e1) / 1e3
        # end to end: host references in, controls and states out, every step
        host_refs = [r.cpu().pin_memory() for r in refs]
        host_out = [(torch.zeros(w.l, w.m).pin_memory(), torch.zeros(w.n, w.m).pin_memory()) for w in wls]
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for i in range(args.steps):
            k = i % (args.warmup + 1)
            for w, hr, (xr, ur, _, _) in zip(wls, host_refs, slots):
                xr.copy_(hr[k:k + w.H + 1], non_blocking=True)
                ur.zero_()
            batch.step()
            for (_, _, ua, xn), (hu, hx) in zip(slots, host_out):
                hu.copy_(ua, non_blocking=True)
                hx.copy_(xn, non_blocking=True)
            batch.sync()
        t_e2e = time.perf_counter() - t0
    h2d = sum((w.H + 1) * w.n * w.m * 4 for w in wls)
    d2h = sum((w.l + w.n) * w.m * 4 for w in wls)
    t_batch, t_seq, t_e2e, t_rule = max_over_ranks([t_batch, t_seq, t_e2e, t_rule], world, dev)
    if tuned is not None:
        tuned["rule_value"] = job_value(P_ * args.steps, world, t_rule)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    P = len(wls)
    lat = sorted(per_step)
    line = {
        "metric": MIX_METRIC, "value": job_value(P * args.steps, world, t_batch), "unit": "control steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_batch / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32+f64",
        "data": "synthetic",
        "config": {"workload": name, "problems": P,
                   "sizes": "grids {32,64,96,128}^2, l = m/8, N {64..512}, H 5..20, CNN 2-32-32-1",
                   "grids": {str(g): sum(1 for w in wls if w.m == g) for g in (32, 64, 96, 128)},
                   "member_steps_per_batch_step": sum(w.N * w.H for w in wls),
                   "precision": "mixed: BF16 conv, FP32 covariance, FP64 mean correction and gain",
                   "noise": "philox-4x32-10 on device, per-problem seeds",
                   "launch": "one CUDA graph per batch step, one branch per problem",
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single",
                   "sequential_value": job_value(P * k_seq, world, t_seq),
                   "sequential": "the same problems one after another, each through its own step graph",
                   "p50_step_ms": lat[len(lat) // 2], "p99_step_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                   "plans": tuned if tuned is not None else "built-in rules (no --tune)"},
        "roofline": None,
        "e2e": {"value": job_value(P * args.steps, world, t_e2e), "unit": "control steps/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "cpu_baseline": {"value": None, "unit": "control steps/s", "cores": host_threads(), "kind": "oracle",
                         "sample": "not run for the batch mode (the single-problem lines carry it)"},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


COV_METRIC = "control solves/s with Algorithm 1's optional covariance outputs (Sigma^X_{t|t-1}, Sigma^X_{t|t})"


def run_cov(args, wl):
    """Solves of the 64 x 64 workload (device noise, eager launches) with and
    without the optional covariance outputs of every assimilation time, timed
    with CUDA events on the solver's stream, L2 flushed between solves."""
    import torch
    import paper_2410_09663_b300 as oic
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    w, b = wl.flat_weights()
    stream = torch.cuda.Stream(device=dev)
    out = {}
    for full in (False, True):
        cfg = oic.config_from_workload(wl, noise_mode=oic.OIC_NOISE_PHILOX, keep_full_history=full)
        s = oic.Solver(cfg, w, b, wl.B(), device=dev, stream=stream)
        H, R = wl.H, s.oic_cov_rows(wl.H)
        with torch.cuda.stream(stream):
            X0 = torch.from_numpy(wl.X0()).to(dev)
            U0 = torch.from_numpy(wl.U_init()).to(dev)
            xr = torch.from_numpy(wl.X_ref_window(0)).to(dev)
            ur = torch.from_numpy(wl.U_ref()).to(dev)
            U_hat = torch.zeros(H + 1, wl.l, wl.m, device=dev)
            pred = torch.zeros(H * R * R, dtype=torch.float64, device=dev)
            post = torch.zeros_like(pred)
            flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
            times = {}
            for mode in ("plain", "cov"):
                def one():
                    if mode == "plain":
                        s.oic_solve(X0, U0, xr, ur, None, U_hat)
                    else:
                        s.oic_solve_cov(X0, U0, xr, ur, None, U_hat, None, 1.0, pred, post)
                for _ in range(args.warmup):
                    one()
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(args.steps)]
                stream.synchronize()
                for i in range(args.steps):
                    flush.fill_(float(i))
                    ev[i][0].record(stream)
                    one()
                    ev[i][1].record(stream)
                stream.synchronize()
                times[mode] = sum(a.elapsed_time(c) for a, c in ev) / args.steps
            s.oic_profile_begin(stages=["cov_out"], max_launches=4096)
            s.oic_solve_cov(X0, U0, xr, ur, None, U_hat, None, 1.0, pred, post)
            prof = s.oic_profile_end()
        s.close()
        rows = [s2 for s2 in range(1, H + 1)]
        flops = sum(2.0 * 2 * (wl.n * (t if full else 1) + (t + 1) * wl.l) ** 2 * wl.N * wl.m for t in rows)
        out["full_history" if full else "u_history"] = {
            "solve_ms": times["plain"], "solve_cov_ms": times["cov"],
            "cov_out_ms": prof.get("cov_out", (0.0, 0))[0], "cov_out_launches": prof.get("cov_out", (0.0, 0))[1],
            "kept_rows_at_H": R, "cov_flops_per_solve": flops,
            "cov_tflops": flops / (prof.get("cov_out", (1e30, 0))[0] / 1e3) / 1e12}
    line = {"metric": COV_METRIC, "value": 1e3 / out["u_history"]["solve_cov_ms"], "unit": "control solves/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": out["u_history"]["solve_cov_ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 products, f64 sums", "data": "synthetic",
            "config": config_dict(wl, {"launch": "eager (oic_solve / oic_solve_cov)", "modes": out})}
    print(json.dumps(line), flush=True)
    return 0


SERVE_METRIC = "served control requests/s (Poisson arrivals, continuous batching)"


def run_serve(args, rate=200.0):
    """Serving loop: Poisson arrivals of control requests (one control step
    of one problem each) over the mix64 problem population, served with
    continuous batching and admission by HBM footprint.  Reports the achieved
    request rate and p50/p99 latency (arrival to completion), next to the
    plain FP32 single-problem path (the 64 x 64 workload stepped alone)."""
    import torch
    import paper_2410_09663_b300 as oic
    from paper_2410_09663_b300 import serving, workloads
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0                                        # one server per node
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    budget_gb = args.budget_gb
    count = args.steps if args.steps != 200 else 10000
    wls = workloads.mix64(seed=2024)
    arrivals = serving.poisson_arrivals(rate, count, len(wls), seed=77)
    per = collections.Counter(pid for _, pid in arrivals)
    srv = serving.Server(dev, budget_bytes=budget_gb * 1e9, precision=oic.OIC_PREC_MIXED)
    for pid, w in enumerate(wls):
        srv.add(pid, w, steps_max=per[pid] + 1)
    footprint = sum(p.bytes for p in srv.problems.values())
    # warm-up: every problem admitted and stepped once (its step graph is
    # captured), then every resident problem back to its initial state
    srv.run([(0.0, pid) for pid in range(len(wls))])
    for p in srv.problems.values():
        if p.solver is not None:
            with torch.cuda.stream(p.stream):
                p.solver.oic_reset(torch.from_numpy(p.wl.X0()).to(dev), torch.from_numpy(p.wl.U_init()).to(dev))
        p.k, p.state, p.evictions = 0, None, 0
    torch.cuda.synchronize(dev)
    srv2 = srv
    launches0 = oic.oic_launch_count()
    with ClockSampler(0) as clk:
        rec, _, wall = srv2.run(arrivals)
    launches = oic.oic_launch_count() - launches0
    overlap = serving.max_overlap(srv2.device_intervals)
    lat = sorted(1e3 * (r[4] - r[2]) for r in rec)
    svc = sorted(1e3 * (r[4] - r[3]) for r in rec)
    span = max(r[4] for r in rec) - min(r[2] for r in rec)
    # the plain FP32 single-problem path, stepped alone back to back
    wl1 = workloads.working_64()
    w1, b1 = wl1.flat_weights()
    s1 = oic.Solver(oic.config_from_workload(wl1, noise_mode=oic.OIC_NOISE_PHILOX), w1, b1, wl1.B(), device=dev)
    xr1 = torch.from_numpy(wl1.X_ref_all(40)).to(dev)
    ur1 = torch.zeros(wl1.l, wl1.m, device=dev)
    uo1, xo1 = torch.zeros(wl1.l, wl1.m, device=dev), torch.zeros(wl1.n, wl1.m, device=dev)
    s1.oic_reset(torch.from_numpy(wl1.X0()).to(dev), torch.from_numpy(wl1.U_init()).to(dev))
    for k in range(5):
        s1.oic_step(xr1[k:k + wl1.H + 1], ur1, None, uo1, xo1)
    s1.oic_sync()
    t0 = time.perf_counter()
    lat1 = []
    for k in range(5, 35):
        a = time.perf_counter()
        s1.oic_step(xr1[k:k + wl1.H + 1], ur1, None, uo1, xo1)
        s1.oic_sync()
        lat1.append(1e3 * (time.perf_counter() - a))
    t1 = time.perf_counter() - t0
    lat1.sort()
    pick = lambda v, q: v[min(len(v) - 1, int(q * len(v)))]
    line = {
        "metric": SERVE_METRIC, "value": count / span, "unit": "requests/s", "n_gpus": 1, "steps": count,
        "warmup": len(wls), "ms_per_step": 1e3 * span / count, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16+f32+f64", "data": "synthetic",
        "config": {"workload": "serve200", "offered_rate": rate, "requests": count,
                   "problems": len(wls), "sizes": "mix64 (grids {32,64,96,128}^2, N {64..512}, H 5..20)",
                   "hbm_budget_bytes": int(budget_gb * 1e9), "footprint_all_problems_bytes": int(footprint),
                   "evictions": int(sum(p.evictions for p in srv2.problems.values())),
                   "max_steps_in_flight_on_device": int(overlap),
                   "latency_ms_p50": pick(lat, 0.5), "latency_ms_p99": pick(lat, 0.99),
                   "latency_ms_max": lat[-1], "service_ms_p50": pick(svc, 0.5), "service_ms_p99": pick(svc, 0.99),
                   "wall_s": wall,
                   "plain_fp32_single_problem": {
                       "workload": wl1.name, "steps_per_s": 30 / t1,
                       "latency_ms_p50": pick(lat1, 0.5), "latency_ms_p99": pick(lat1, 0.99)},
                   "latency": "arrival to completion (includes queueing); service = launch to completion"},
        "roofline": None,
        "e2e": {"value": count / span, "unit": "requests/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "cpu_baseline": {"value": None, "unit": "requests/s", "cores": host_threads(), "kind": "oracle",
                         "sample": "not run for the serving mode (the single-problem lines carry it)"},
    }
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["oic", "reference"], default="oic")
    ap.add_argument("--workload", default="working_64")
    ap.add_argument("--precision", choices=["fp32", "mixed"], default="fp32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tune", action="store_true",
                    help="batch mode: autotune every problem's plan and time the batch with the tuned plans")
    ap.add_argument("--budget-gb", type=float, default=150.0,
                    help="serving mode: HBM budget for admission (GB)")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--members", type=int, default=0,
                    help="ensemble size N other than the workload's (smaller cases for profiling)")
    ap.add_argument("--cov-outputs", action="store_true",
                    help="time solves with the optional covariance outputs against plain solves")
    ap.add_argument("--constraint", choices=["none", "u_box"], default="none",
                    help="u_box: |U| <= 0.1 on every control entry as 2 l softplus-barrier rows")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    from paper_2410_09663_b300 import workloads
    if args.workload == "serve200":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the serving mode has no oracle arm"}), flush=True)
            return 0
        return run_serve(args)
    if args.workload in workloads.BATCHES:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batch mode has no oracle arm"}), flush=True)
            return 0
        return run_mix(args, args.workload)
    wl = workloads.WORKLOADS[args.workload]()
    if args.members:
        wl = wl.with_(N=args.members, name=f"{wl.name}_N{args.members}")
    if args.constraint == "u_box":
        wl = wl.with_(cons=workloads.u_box(wl.n, wl.l, 0.1))
    if args.impl == "reference":
        return run_reference(args, wl)
    if args.cov_outputs:
        return run_cov(args, wl)
    return run_oic(args, wl)


if __name__ == "__main__":
    sys.exit(main())
