#!/usr/bin/env python3
"""Throughput of the in-place 1-D complex DFT on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c2|c3|c1|c4|c5|r1|m1]
                    [--impl ours|reference]

Default workload (the headline configuration, c3): one step = one in-place
transform of N = 2^33 complex128 points (128 GiB in HBM, no out-of-place
buffer), the forward (sign -1, Eq. 1) and the normalised inverse (sign +1,
times 1/N) alternating, input uniform[-1,1) re/im.  value = 5*N*log2(N)
flop per transform x transforms / time (GFLOP/s), whole job.  The input is
larger than the 129 MB L2, so no flush is needed between timed iterations.
The default line also carries `fp32_form`: the complex64 form at N = 2^31
(Gaussian input) against the complex128 form at the same N, timed, with the
complex64 error against the FP64 oracle on sampled bins and against the
complex128 result over the whole array.
Workload c2: forward then normalised inverse of N = 2^30 complex128 points
(16 GiB), uniform[-1,1) re/im plus 64 seeded tones.

Workload c5 (batched, mixed sizes): 256 complex64 transforms of 2^12..2^24
points in one arena, each direction one efft_batch_execute (one CUDA graph
launch); a step = forward + normalised conjugate-sign transform of all 256.

--impl reference times the CPU oracle (the FP64 radix-2 FFT, as it stands)
on the host cores; each step is a bounded sample of the workload's step
(the same transforms at a smaller N, named in `sample_of_step`), and
ms_per_step is the time that sample step took.

Multi-GPU: the transform does not shard across GPUs (one FFT
per GPU); under torchrun every rank runs an independent replica ("replicas
only") and value is the sum over ranks divided by the max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "5N·log2N GFLOP/s + HBM GB/s, in-place 1D FFT; FP32 vs FP64 at stated error"

WORKLOADS = {
    "c2": dict(log2n=30, dtype="c128", seed=2, tones=64, fwd_inv=True, gauss=False,
               desc="complex128 N=2^30 in place, forward then normalised inverse; "
                    "uniform[-1,1) re/im + 64 seeded tones"),
    "c3": dict(log2n=33, dtype="c128", seed=3, tones=0, fwd_inv=False, gauss=False,
               desc="complex128 N=2^33 (128 GiB) in place, one transform per step "
                    "(forward / normalised inverse alternating); uniform[-1,1) re/im"),
    "c1": dict(log2n=20, dtype="c128", seed=1, tones=0, fwd_inv=False, gauss=False,
               desc="complex128 N=2^20 in place, one transform per step; uniform[-1,1) re/im"),
    "c4": dict(log2n=31, dtype="c64", seed=4, tones=0, fwd_inv=False, gauss=True,
               desc="complex64 N=2^31 in place, one transform per step; Gaussian(0,1) re/im"),
    "m1": dict(log2n=30, n=3 << 28, dtype="c128", seed=7, tones=0, fwd_inv=True, gauss=False, normalize=False,
               desc="complex128 N=3*2^28 (12 GiB, the paper's size set N = M*2^s) in place, forward then the "
                    "unnormalised conjugate-sign transform (1/N is not exact); uniform[-1,1) re/im"),
    "r1": dict(log2n=31, real=True, dtype="c64", seed=6, tones=0, fwd_inv=True, gauss=False,
               desc="real float32 N=2^32 reals (16 GiB) in place, forward to the perm layout (Eq. 3) then the "
                    "normalised inverse; uniform[-1,1); GFLOP/s by the real-data count (5/2) N log2 N (Eq. 7)"),
    "c5": dict(batch=256, emin=12, emax=24, log2n=24, dtype="c64", seed=5, tones=0, fwd_inv=True, gauss=False,
               autotune=True,
               desc="256 complex64 transforms in place, N_i = 2^e_i with e_i uniform in {12..24} (seed 5), "
                    "one graph launch per direction: forward, then the normalised conjugate-sign transform; "
                    "radix schedules from the autotuner; uniform[-1,1) re/im"),
}
DTYPE_NAME = {"c128": "df32 (double-float f32 pairs; complex128 in/out)", "c64": "f32 (complex64)"}
DTYPE_NAME_REAL = {"c128": "df32 (double-float f32 pairs; float64 in/out)", "c64": "f32 (float32 reals)"}


def flops(n: int) -> float:
    return 5.0 * n * math.log2(n)


# Double-float (complex128) pass kernels: FP32 operations per element of one
# pass, from the fixed operation counts of the double-float method (FMA
# counted once; packed FP32x2 instructions count their two lanes):
#   complex add/sub (TwoSum on both parts, low parts added)     16
#   complex multiply (TwoProd by FMA, TwoSum, 4 cross terms)    32
#   multiply by exp(-2*pi*i/8) (add, then a real product)     24
#   renormalisation before an intermediate store               6
# A radix-2^LR pass (radix-16 stages, then one of radix 2^(LR mod 4)) does
# LR complex adds per element, the radix-16 constant multiplies (4 general
# and 6 by exp(-2*pi*i/8) per 16 elements per radix-16 stage; 2 by
# exp(-2*pi*i/8) per 8 in a radix-8 stage), 15/16 of a complex multiply per
# internal twiddle stage, and in strided passes the pass twiddle as two
# complex multiplies.
DF_OPS = {"add": 16, "mul": 32, "w8": 24, "norm": 6}
FP32_PEAK_OPS = 152 * 128 * 2.07e9  # SMs x FP32 lanes x maximum SM clock


def df_ops_per_element(log2r: int, kind: str) -> float:
    nfull, rem = divmod(log2r, 4)
    nst = nfull + (1 if rem else 0)
    ops = log2r * DF_OPS["add"]
    ops += nfull * (4 * DF_OPS["mul"] + 6 * DF_OPS["w8"]) / 16.0
    if rem == 3:
        ops += 2 * DF_OPS["w8"] / 8.0
    ops += (nst - 1) * 15.0 / 16.0 * DF_OPS["mul"]
    if kind in ("FIRST", "MID"):
        ops += 2 * DF_OPS["mul"] + DF_OPS["norm"]
    return ops


def flops_real(n: int) -> float:
    """The paper's count for n real points (Eq. 7)."""
    return 2.5 * n * math.log2(n)


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over all ranks (the job's time is its slowest rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, transforms_per_step: int, n: int, ms_per_step: float, real: bool = False) -> float:
    """Whole-job GFLOP/s: every rank transforms its own array (replicas);
    n complex points, or for real data 2n reals."""
    f = flops_real(2 * n) if real else flops(n)
    return world * transforms_per_step * f / (ms_per_step * 1e-3) / 1e9


KERNEL_SOURCES = {
    "c128": ("efft_kernels.cuh", "efft_arith.cuh", "efft_fx_df2.cu"),
    "c64": ("efft_kernels.cuh", "efft_arith.cuh", "efft_fx_f32.cu", "efft_fx32.cuh"),
    "mixed": ("efft_kernels.cuh", "efft_arith.cuh", "efft_mix.cuh", "efft_mix.cu"),
}


def scale_workload(wl: dict, log2n: int) -> dict:
    """The workload at another size (profiling captures on a smaller case):
    N = 2^log2n, or for N = M * 2^e the same M with e moved by as much as
    log2n moves (log2n is ceil(log2 N))."""
    wl = dict(wl)
    if "n" in wl:
        e = (wl["n"] & -wl["n"]).bit_length() - 1
        odd, e_new = wl["n"] >> e, e + log2n - wl["log2n"]
        wl["desc"] = wl["desc"].replace(f"{odd}*2^{e}", f"{odd}*2^{e_new}").replace(
            f"{(wl['n'] * 16) >> 30} GiB", f"{((odd << e_new) * 16) / 2**30:g} GiB")
        wl["n"] = odd << e_new
    wl["desc"] = wl["desc"].replace(f"2^{wl['log2n']}", f"2^{log2n}")
    wl["log2n"] = log2n
    return wl


def kernel_fingerprint(family: str) -> str:
    """sha1 (16 hex digits) of the sources of one kernel family: the
    complex128 or complex64 power-of-two pass kernels, or the mixed-radix
    middle-pass kernel."""
    import hashlib
    h = hashlib.sha1()
    files = KERNEL_SOURCES[family]
    for f in files:
        with open(os.path.join(ROOT, "paper_1409_5757_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload: str, log2n: int, kernel: str):
    """DRAM bytes per launch and pipe figures from the committed ncu summary,
    or None when there is none for this kernel or the kernel changed since."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        family = ("mixed" if workload == "m1" and kernel == "pass1"
                  else WORKLOADS[workload]["dtype"] if workload in WORKLOADS else "c128")
        fp = kernel_fingerprint(family)
        with open(path) as f:
            for line in f:
                if not line.strip() or line.startswith("#"):
                    continue
                w, e, k, b, fma, issue, src_fp, *src = line.split()
                if w == workload and int(e) == log2n and k == kernel and src_fp == fp:
                    # '-': the capture took DRAM bytes only
                    return {"bytes": float(b), "fma_pipe_pct": None if fma == "-" else float(fma),
                            "issue_pct": None if issue == "-" else float(issue), "source": " ".join(src)}
    except (OSError, ValueError):
        pass
    return None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------
def oracle_time(log2n: int, seed: int, reps: int = 1):
    """Time `reps` forward radix-2 transforms of 2^log2n points on the host."""
    import oracle
    o = oracle.get()
    x = o.gen_uniform(seed, 1 << log2n)
    best = None
    for _ in range(reps):
        t0 = time.perf_counter()
        o.fft_radix2(x, -1)
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    return best, o.threads


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_single_core(log2n: int, seed: int):
    """GFLOP/s of one forward oracle transform of 2^log2n points on one core
    (a fresh interpreter with OMP_NUM_THREADS=1)."""
    code = ("import sys, time; sys.path.insert(0, %r); import oracle; o = oracle.get(); "
            "x = o.gen_uniform(%d, 1 << %d); t = time.perf_counter(); o.fft_radix2(x, -1); "
            "print(time.perf_counter() - t, o.threads)") % (ROOT, seed, log2n)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
        dt, th = r.stdout.split()[-2:]
        return {"value": flops(1 << log2n) / float(dt) / 1e9, "unit": "GFLOP/s", "cores": int(th),
                "sample": f"one forward FP64 radix-2 oracle transform of N=2^{log2n}, {float(dt):.2f} s"}
    except Exception as ex:  # report, do not fail the benchmark line
        return {"value": None, "error": str(ex)[:200]}


def oracle_sample_log2n(target_s: float, cap: int) -> int:
    """Largest size <= 2^cap whose oracle transform fits in about target_s."""
    t20, _ = oracle_time(20, 1)
    for e in range(cap, 19, -1):
        est = t20 * (2.0 ** (e - 20)) * (e / 20.0) * 1.3
        if est <= target_s:
            return e
    return 20


def batch_sizes(wl):
    """The batch workload's log2 sizes: uniform integers in [emin, emax] from
    numpy's default generator seeded with the workload seed."""
    import numpy as np
    return [int(e) for e in np.random.default_rng(wl["seed"]).integers(wl["emin"], wl["emax"] + 1, wl["batch"])]


def oracle_batch_time(wl, budget_s: float):
    """The oracle's forward transforms of the batch's arrays, in batch order,
    until budget_s has passed: (flop, seconds, transforms, threads)."""
    import oracle
    o = oracle.get()
    fl, el, k = 0.0, 0.0, 0
    for i, e in enumerate(batch_sizes(wl)):
        x = o.gen_uniform(wl["seed"] * 1000 + i, 1 << e)
        t0 = time.perf_counter()
        o.fft_radix2(x, -1)
        el += time.perf_counter() - t0
        fl += flops(1 << e)
        k += 1
        if el >= budget_s:
            break
    return fl, el, k, o.threads


def run_reference_batch(args, wl):
    K, W = args.steps, args.warmup
    budget = 150.0 / max(K + W, 1)
    rates, step_s, cores, k = [], [], None, 0
    for i in range(W + K):
        t0 = time.perf_counter()
        fl, el, k, cores = oracle_batch_time(wl, budget)
        if i >= W:
            rates.append(fl / el)
            step_s.append(time.perf_counter() - t0)
    value = statistics.mean(rates) / 1e9
    ms = 1e3 * statistics.mean(step_s)
    sample = (f"FP64 radix-2 oracle, forward transforms of the first {k} arrays of the batch (in batch order) "
              f"per step, about {budget:.0f} s of host time; a full step is 2 x 256 transforms; ms_per_step is "
              f"that sample step's time")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": args.gpus,
        "steps": K, "warmup": W, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_of(wl),
        "sample_of_step": {"transforms": k, "of": 2 * len(batch_sizes(wl))},
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args, wl):
    import oracle  # noqa: F401
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if wl.get("batch"):
        return run_reference_batch(args, wl)
    import oracle
    o = oracle.get()
    K, W = args.steps, args.warmup
    tps = 2 if wl["fwd_inv"] else 1
    budget = 150.0 / max(K + W, 1) / tps
    e = oracle_sample_log2n(budget, wl["log2n"])
    x = o.gen_uniform(wl["seed"], 1 << e)
    times = []
    for i in range(W + K):
        # one step of the workload at N = 2^e: the forward transform, and for
        # forward-inverse workloads the conjugate-sign transform of its result
        t0 = time.perf_counter()
        y = o.fft_radix2(x, -1)
        if tps == 2:
            o.fft_radix2(y, +1)
        dt = time.perf_counter() - t0
        if i >= W:
            times.append(dt)
    cores = o.threads
    ms = 1e3 * statistics.mean(times)
    value = tps * flops(1 << e) / (ms * 1e-3) / 1e9
    sample = (f"each step: {'forward then conjugate-sign' if tps == 2 else 'one forward'} FP64 radix-2 oracle "
              f"transform{'s' if tps == 2 else ''} of N=2^{e} (the workload's step at N=2^{wl['log2n']} scaled "
              f"down to about {budget * tps:.0f} s of host time), seeded uniform input; ms_per_step is that "
              f"sample step's time")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": args.gpus,
        "steps": K, "warmup": W, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(wl), "sample_of_step": {"log2N": e, "N": 1 << e, "transforms": tps},
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def config_of(wl):
    if wl.get("batch"):
        es = batch_sizes(wl)
        return {"workload": wl["desc"], "transforms": len(es), "log2N_min": min(es), "log2N_max": max(es),
                "elements_total": sum(1 << e for e in es), "element": "complex64" if wl["dtype"] == "c64"
                else "complex128", "transforms_per_step": 2 * len(es), "in_place": True,
                "l2_between_steps": "inputs larger than L2 (no flush needed)", "seed": wl["seed"],
                "parallelism": "replicas only (one batch per GPU)"}
    if wl.get("real"):
        return {"workload": wl["desc"], "N_reals": 2 << wl["log2n"], "log2N": wl["log2n"] + 1,
                "element": "float32" if wl["dtype"] == "c64" else "float64", "layout": "perm (Eq. 3)",
                "transforms_per_step": 2 if wl["fwd_inv"] else 1, "in_place": True,
                "l2_between_steps": "inputs larger than L2 (no flush needed)",
                "seed": wl["seed"], "parallelism": "replicas only (one transform per GPU)"}
    return {"workload": wl["desc"], "N": wl.get("n", 1 << wl["log2n"]), "log2N": wl["log2n"],
            "element": "complex128" if wl["dtype"] == "c128" else "complex64",
            "transforms_per_step": 2 if wl["fwd_inv"] else 1, "in_place": True,
            "l2_between_steps": "inputs larger than L2 (no flush needed)" if wl["log2n"] >= 24
            else "inputs fit in L2 (latency-bound size)",
            "seed": wl["seed"], "parallelism": "replicas only (one transform per GPU)"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args, wl):
    import torch
    import torch.distributed as dist

    import paper_1409_5757_gb300 as efft
    from paper_1409_5757_gb300 import build as _build
    from paper_1409_5757_gb300 import inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()

    N = wl.get("n", 1 << wl["log2n"])
    c128 = wl["dtype"] == "c128"
    tdt = torch.complex128 if c128 else torch.complex64
    code = efft.EFFT_C128 if c128 else efft.EFFT_C64
    S = 16 if c128 else 8

    x = torch.empty(N, dtype=tdt, device=dev)
    if wl["gauss"]:
        inputs.fill_gaussian(x, wl["seed"])
    else:
        inputs.fill_uniform(x, wl["seed"])
    if wl["tones"]:
        f, a = inputs.tone_params(wl["seed"], N, wl["tones"])
        inputs.add_tones(x, f, a)
    torch.cuda.synchronize(dev)
    ref_norm = None
    keep = None
    if N * S <= (32 << 30):
        keep = x.clone()  # for the round-trip accuracy check after timing

    tune = efft.EFFT_FLAG_AUTOTUNE if args.autotune else 0
    real = bool(wl.get("real"))
    if real:
        # x holds 2N reals (the same bytes as N complex values)
        fwd = efft.Plan.real(2 * N, code, efft.EFFT_REAL_FORWARD, tune)
        inv = efft.Plan.real(2 * N, code, efft.EFFT_REAL_INVERSE, efft.EFFT_FLAG_NORMALIZE | tune)
    else:
        norm_flag = efft.EFFT_FLAG_NORMALIZE if wl.get("normalize", True) else 0
        rad = [int(v) for v in args.radices.split(",")] if args.radices else None
        fwd = efft.Plan(N, code, -1, 0 if rad else tune, radices=rad)
        inv = efft.Plan(N, code, +1, norm_flag | (0 if rad else tune), radices=rad)
        if args.variant:
            knobs = [int(v) for v in args.variant.split(",")]
            fwd.set_variant(*knobs)
            inv.set_variant(*knobs)
    fpt = flops_real(2 * N) if real else flops(N)  # flop per transform
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    tps = 2 if wl["fwd_inv"] else 1

    def step(i):
        if wl["fwd_inv"]:
            fwd.execute(x.data_ptr(), sp)
            inv.execute(x.data_ptr(), sp)
        elif i % 2 == 0:
            fwd.execute(x.data_ptr(), sp)
        else:
            inv.execute(x.data_ptr(), sp)

    K, W = args.steps, args.warmup
    for i in range(W):
        step(i)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)

    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(0.3)
    fwd.profile(True)
    inv.profile(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()  # a profiler run with --profile-from-start off sees the timed region only
    e0.record(stream)
    for i in range(K):
        step(W + i)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    torch.cuda.profiler.stop()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    elapsed_ms = e0.elapsed_time(e1)
    prof = {}
    for p in (fwd, inv):
        for k, (ms, n) in p.profile_read().items():
            a = prof.setdefault(k, [0.0, 0])
            a[0] += ms
            a[1] += n
    fwd.profile(False)
    inv.profile(False)

    elapsed_ms = max_over_ranks(elapsed_ms, dev)
    ms_per_step = elapsed_ms / K
    value = job_rate(world, tps, N, ms_per_step, real)
    hbm_passes = fwd.info()["hbm_passes"]
    hbm_gbs = world * tps * hbm_passes * 2 * N * S / (ms_per_step * 1e-3) / 1e9

    # accuracy: after W+K round trips the buffer should equal the input
    accuracy = None
    done = W + K
    if not wl["fwd_inv"] and done % 2 == 1:
        step(done)  # untimed: complete the last forward / inverse pair
        done += 1
    round_trips = done if wl["fwd_inv"] else done // 2
    tol_rt = 2e-14 * wl["log2n"] if c128 else 4e-6 * wl["log2n"]
    if keep is not None:
        # forward then inverse, round_trips times: x returns (times N per
        # round trip when the inverse is unnormalised)
        scale = 1.0 if wl.get("normalize", True) else float(N) ** (-round_trips)
        num, den = inputs.diff_norms(x, keep, scale)
        accuracy = {"roundtrip_rel_l2_after_all_steps": math.sqrt(num / den), "round_trips": round_trips,
                    "tolerance_per_round_trip": tol_rt}
    elif not wl["tones"] and not wl["gauss"] and not real and wl.get("normalize", True):
        # no room for a copy: the input regenerated chunk by chunk (the same
        # seeded stream) and compared with the buffer
        chunk = min(N, 1 << 28)
        y = torch.empty(chunk, dtype=tdt, device=dev)
        num = den = 0.0
        for c0 in range(0, N, chunk):
            inputs.fill_uniform(y, wl["seed"], n0=c0)
            a_, b_ = inputs.diff_norms(x[c0:c0 + chunk], y)
            num += a_
            den += b_
        del y
        accuracy = {"roundtrip_rel_l2_after_all_steps": math.sqrt(num / den), "round_trips": round_trips,
                    "tolerance_per_round_trip": tol_rt,
                    "reference": "the seeded input regenerated in 2^28-element chunks"}

    # roofline of the dominant kernel
    peak, peak_kind = peaks()
    dom = max(prof.items(), key=lambda kv: kv[1][0]) if prof else None
    roofline = None
    if dom:
        name, (tot_ms, nl) = dom
        per_launch_s = tot_ms / nl * 1e-3
        alg_bytes = (1 if name == "range_scan" else 2) * N * S
        achieved = alg_bytes / per_launch_s / 1e9
        tr = measured_traffic(args.workload, wl["log2n"], name)
        roofline = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": tr["bytes"] if tr else None,
                    "traffic_source": tr["source"] if tr else None,
                    "fp32_view": ({"fma_pipe_active_pct": tr["fma_pipe_pct"], "issue_active_pct": tr["issue_pct"],
                                   "note": ("the double-float pass kernels are bound by the FP32 pipe, not HBM"
                                            if c128 else "the FP32 pass kernels are bound by the L1/LSU data "
                                            "pipe and load latency, not HBM")}
                                  if tr and tr["fma_pipe_pct"] is not None else None),
                    "peak_kind": f"{peak_kind} STREAM-style copy (MEASURED_PEAKS.json hbm_gbs)",
                    "per_launch_ms": tot_ms / nl, "algorithmic_bytes_per_launch": alg_bytes,
                    "kernels_ms_per_step": {k: v[0] / K for k, v in prof.items()}}
        # the second roofline of a double-float power-of-two pass: FP32 arithmetic
        rad = fwd.radices() if hasattr(fwd, "radices") else []
        if c128 and name.startswith("pass") and rad and N & (N - 1) == 0 and not real:
            j = int(name[4:])
            kind = "SINGLE" if len(rad) == 1 else ("FIRST" if j == 0 else "LAST" if j == len(rad) - 1 else "MID")
            ope = df_ops_per_element(rad[j], kind)
            ach = ope * N / per_launch_s
            roofline["alu_view"] = {
                "bound": "alu", "achieved": ach / 1e12, "peak": FP32_PEAK_OPS / 1e12,
                "unit": "T FP32 operations/s (FMA counted once)", "frac": ach / FP32_PEAK_OPS,
                "ops_per_element": ope, "pass": f"2^{rad[j]} {kind}",
                "peak_kind": "152 SMs x 128 FP32 lanes x 2070 MHz (maximum SM clock)"}
    launches = sum(v[1] for v in prof.values())
    radices_now = fwd.radices()
    variant_now = fwd.variant()
    floor_gbs = world * tps * 2 * N * S / (ms_per_step * 1e-3) / 1e9

    # the FP32 form against the FP64 form at the same N (complex64 workloads)
    same_n_c128 = None
    if not c128 and not real and N * 16 <= (64 << 30) and not args.no_compare:
        del keep
        keep = None
        y = torch.empty(N, dtype=torch.complex128, device=dev)
        inputs.fill_gaussian(y, wl["seed"]) if wl["gauss"] else inputs.fill_uniform(y, wl["seed"])
        p128f = efft.Plan(N, efft.EFFT_C128, -1)
        p128i = efft.Plan(N, efft.EFFT_C128, +1, efft.EFFT_FLAG_NORMALIZE)
        for i in range(3):
            (p128f if i % 2 == 0 else p128i).execute(y.data_ptr(), sp)
        Kc = 4
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for i in range(Kc):
            (p128i if i % 2 == 0 else p128f).execute(y.data_ptr(), sp)
        c1.record(stream)
        torch.cuda.synchronize(dev)
        ms128 = c0.elapsed_time(c1) / Kc
        same_n_c128 = {"value": flops(N) / (ms128 * 1e-3) / 1e9, "unit": "GFLOP/s", "ms_per_transform": ms128,
                       "speedup_of_complex64": ms128 / (ms_per_step / tps)}
        for q in (p128f, p128i):
            q.destroy()
        del y

    # end to end: host buffers through efft_execute_host_stream (each step copies
    # its input from pinned host memory, transforms, copies the result back;
    # copies of neighbouring steps overlap the transforms of this one)
    e2e = None
    host_room = mem_available()
    # (one rank only: ranks share the host's memory, and each would pin the
    # whole array)
    if (N * S > (32 << 30) and not args.no_e2e and world == 1 and host_room is not None
            and host_room >= N * S + (24 << 30)):
        # the whole array does not fit twice in HBM: one device buffer (the
        # timed one) and one pinned host array that is both input and output,
        # so each step copies 2^33 x 16 B in, transforms, copies it back
        torch.cuda.synchronize(dev)
        t_pin = time.perf_counter()
        hbuf = inputs.PinnedHost(N, tdt)
        t_pin = time.perf_counter() - t_pin
        hbuf.tensor.copy_(x)
        Ke = 2
        efft.execute_host_stream([fwd], [hbuf.ptr], [hbuf.ptr], [x.data_ptr()], sp)  # warm
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        efft.execute_host_stream([fwd], [hbuf.ptr] * Ke, [hbuf.ptr] * Ke, [x.data_ptr()], sp)
        dt = (time.perf_counter() - t0) / Ke
        hbuf.free()
        del hbuf
        e2e = {"value": world * fpt / dt / 1e9, "unit": "GFLOP/s",
               "h2d_bytes_per_step": N * S, "d2h_bytes_per_step": N * S,
               "ms_per_step": dt * 1e3, "steps": Ke, "pin_seconds": t_pin,
               "api": "efft_execute_host_stream (one cudaHostAlloc host array as input and output, the one "
                      "device buffer: a second 128 GiB device buffer does not fit; the copy out of a step "
                      "and the copy in of the next share the link's two directions, 1 GiB piece by piece)"}
    elif (N * S <= (32 << 30) and not args.no_e2e
          and (world == 1 or (host_room is not None and host_room >= world * 2 * N * S + (24 << 30)))):
        src = keep if keep is not None else x
        hin = inputs.PinnedHost(N, tdt)
        hout = inputs.PinnedHost(N, tdt)
        hin.tensor.copy_(src)
        bufs = [x] + [torch.empty(N, dtype=tdt, device=dev) for _ in range(2)]
        chain = [fwd, inv] if wl["fwd_inv"] else [fwd]
        Ke = max(3, K)
        efft.execute_host_stream(chain, [hin.ptr] * 2, [hout.ptr] * 2, [b.data_ptr() for b in bufs], sp)  # warm
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        efft.execute_host_stream(chain, [hin.ptr] * Ke, [hout.ptr] * Ke, [b.data_ptr() for b in bufs], sp)
        dt = (time.perf_counter() - t0) / Ke
        hin.free()
        hout.free()
        tps_e2e = len(chain)
        e2e = {"value": world * tps_e2e * fpt / dt / 1e9, "unit": "GFLOP/s",
               "h2d_bytes_per_step": N * S, "d2h_bytes_per_step": N * S,
               "ms_per_step": dt * 1e3, "steps": Ke,
               "api": "efft_execute_host_stream (cudaHostAlloc host buffers, 3 device buffers, "
                      "copies in 1 GiB pieces overlapped with the transforms)"}
        del hin, hout, bufs
    elif not args.no_e2e:
        why = (f"{world} ranks would each pin a {N * S >> 30} GiB host array in the host's shared memory"
               if world > 1 else
               f"a pinned host copy of the {N * S >> 30} GiB array needs {(N * S >> 30) + 24} GiB of host memory; "
               f"MemAvailable is {'unknown' if host_room is None else str(host_room >> 30) + ' GiB'}")
        e2e = {"value": None, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0, "skipped": why}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        e = wl["log2n"] if wl["log2n"] <= 30 else 30
        e = min(e, oracle_sample_log2n(25.0, e))
        dt, cores = oracle_time(e, wl["seed"])
        # real data: the oracle transforms 2^e reals by a 2^e-point complex FFT,
        # i.e. the same time as this complex sample, counted by Eq. 7
        cval = (flops_real(1 << e) if real else flops(1 << e)) / dt / 1e9
        cpu = {"value": cval, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
               "sample": f"one forward FP64 radix-2 oracle transform of N=2^{e} (same seeded uniform input "
                         f"family) on the host cores, {dt:.1f} s",
               "nproc": os.cpu_count(), "cpu_model": cpu_model(),
               "single_core": oracle_single_core(min(e, 24), wl["seed"])}

    for p in (fwd, inv):
        p.destroy()
    fwd = inv = None
    fp32 = None
    if args.workload == "c3" and not args.no_fp32_form and args.log2n is None:
        del x
        keep = None
        import gc
        gc.collect()
        torch.cuda.empty_cache()
        fp32 = fp32_form(dev, stream, rank == 0 and world == 1 and not args.no_cpu)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": (DTYPE_NAME_REAL if real else DTYPE_NAME)[wl["dtype"]], "data": "synthetic",
            "config": config_of(wl),
            "hbm_gbs": hbm_gbs, "hbm_passes_per_transform": hbm_passes, "floor_equivalent_gbs": floor_gbs,
            "radices_log2": radices_now, "variant": variant_now,
            "fp64_form_same_n": same_n_c128, "fp32_form": fp32,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks, "accuracy": accuracy, "impl": "ours",
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def mem_available():
    """Host memory the kernel reports as available (bytes), or None."""
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return None


def fp32_form(dev, stream, with_oracle: bool):
    """The precision form against the FP64 form on the same GPU at the same
    N: complex64 (FP32 butterflies, FP64-generated twiddles, compensated
    products) and complex128 transforms of N = 2^31 points, Gaussian(0,1)
    re/im (seed 4), each timed over alternating forward / normalised inverse
    transforms (CUDA events); the complex64 forward result's error against
    the complex128 result of the same (FP32-rounded) input over the whole
    array, and against the FP64 oracle at sampled bins."""
    import torch

    import paper_1409_5757_gb300 as efft
    from paper_1409_5757_gb300 import inputs
    wl = WORKLOADS["c4"]
    e = wl["log2n"]
    N = 1 << e
    sp = stream.cuda_stream

    def timed(plans, buf, k):
        for i in range(3):
            plans[i % 2].execute(buf.data_ptr(), sp)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(k):
            plans[(i + 1) % 2].execute(buf.data_ptr(), sp)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / k

    out = {"workload": wl["desc"], "N": N, "log2N": e}
    x = torch.empty(N, dtype=torch.complex64, device=dev)
    inputs.fill_gaussian(x, wl["seed"])
    p64 = [efft.Plan(N, efft.EFFT_C64, -1), efft.Plan(N, efft.EFFT_C64, +1, efft.EFFT_FLAG_NORMALIZE)]
    ms64 = timed(p64, x, 10)
    inputs.fill_gaussian(x, wl["seed"])
    y = x.to(torch.complex128)  # the same FP32 values, promoted
    sumsq = inputs.diff_norms(y)[0]
    p128 = [efft.Plan(N, efft.EFFT_C128, -1), efft.Plan(N, efft.EFFT_C128, +1, efft.EFFT_FLAG_NORMALIZE)]
    p64[0].execute(x.data_ptr(), sp)
    p128[0].execute(y.data_ptr(), sp)
    xx = x.to(torch.complex128)
    num, den = inputs.diff_norms(xx, y)
    del xx
    ks = None
    if with_oracle:
        import numpy as np
        import oracle
        room = mem_available()
        if room is None or room >= 3 * N * 16 + (8 << 30):
            g = np.random.default_rng(44)
            ks = sorted({0, 1, N // 2, N - 1} | {int(v) for v in g.integers(0, N, 4)})
            got = x[torch.tensor(ks, device=dev)].cpu().numpy().astype(np.complex128)
            z = torch.empty(N, dtype=torch.complex64, device=dev)
            inputs.fill_gaussian(z, wl["seed"])
            zin = z.cpu().numpy()
            del z
            t0 = time.perf_counter()
            ref = oracle.get().dft_bins(zin.astype(np.complex128), np.array(ks, np.int64), -1)
            t_or = time.perf_counter() - t0
            del zin
            err_s = math.sqrt(float(np.mean(np.abs(got - ref) ** 2)) / sumsq)
            out["error_vs_fp64_oracle_sampled"] = {
                "rel_l2_estimate": err_s, "bins": ks, "oracle_seconds": t_or,
                "estimator": "sqrt(mean_k |F_k - Fe_k|^2 / sum_n |x_n|^2) (Eq. 9 with Parseval)"}
    inputs.fill_gaussian(y, wl["seed"])
    ms128 = timed(p128, y, 6)
    for p in p64 + p128:
        p.destroy()
    del x, y
    torch.cuda.empty_cache()
    out.update({
        "complex64": {"ms_per_transform": ms64, "gflops": flops(N) / (ms64 * 1e-3) / 1e9,
                      "hbm_gbs_floor_equivalent": 2 * N * 8 / (ms64 * 1e-3) / 1e9},
        "complex128": {"ms_per_transform": ms128, "gflops": flops(N) / (ms128 * 1e-3) / 1e9,
                       "hbm_gbs_floor_equivalent": 2 * N * 16 / (ms128 * 1e-3) / 1e9},
        "speedup_of_complex64": ms128 / ms64,
        "error_vs_complex128_full": math.sqrt(num / den),
        "tolerance_stated": 2e-6 * e,
    })
    return out


def run_batch(args, wl):
    """Workload c5: two batch executes per step over one arena."""
    import torch
    import torch.distributed as dist

    import paper_1409_5757_gb300 as efft
    from paper_1409_5757_gb300 import build as _build
    from paper_1409_5757_gb300 import inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()

    es = batch_sizes(wl)
    c128 = wl["dtype"] == "c128"
    tdt = torch.complex128 if c128 else torch.complex64
    code = efft.EFFT_C128 if c128 else efft.EFFT_C64
    S = 16 if c128 else 8
    total = sum(1 << e for e in es)
    offs = [0]
    for e in es:
        offs.append(offs[-1] + (1 << e))
    arena = torch.empty(total, dtype=tdt, device=dev)
    inputs.fill_uniform(arena, wl["seed"])
    keep = arena.clone()
    ptrs = [arena.data_ptr() + o * S for o in offs[:-1]]
    sizes = [1 << e for e in es]
    tune = efft.EFFT_FLAG_AUTOTUNE if (wl.get("autotune") or args.autotune) else 0
    fwd = efft.Batch(sizes, code, -1, tune)
    inv = efft.Batch(sizes, code, +1, efft.EFFT_FLAG_NORMALIZE | tune)
    schedules = {e: efft.Plan(1 << e, code, -1, tune).radices() for e in sorted(set(es))}
    kernels = fwd.info()["kernels"] + inv.info()["kernels"]
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream

    def step():
        fwd.execute(ptrs, sp)
        inv.execute(ptrs, sp)

    K, W = args.steps, args.warmup
    for _ in range(W):
        step()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(0.3)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * K + 1)]
    torch.cuda.profiler.start()  # a profiler run with --profile-from-start off sees the timed region only
    ev[0].record(stream)
    for i in range(K):
        fwd.execute(ptrs, sp)
        ev[2 * i + 1].record(stream)
        inv.execute(ptrs, sp)
        ev[2 * i + 2].record(stream)
    torch.cuda.synchronize(dev)
    torch.cuda.profiler.stop()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    elapsed_ms = ev[0].elapsed_time(ev[2 * K])
    graph_ms = [ev[j].elapsed_time(ev[j + 1]) for j in range(2 * K)]

    elapsed_ms = max_over_ranks(elapsed_ms, dev)
    ms_per_step = elapsed_ms / K
    step_flop = 2 * sum(flops(n) for n in sizes)
    value = world * step_flop / (ms_per_step * 1e-3) / 1e9
    passes = {}
    for e in sorted(set(es)):
        passes[e] = efft.Plan(1 << e, code, -1, tune).info()["hbm_passes"]
    step_bytes = 2 * sum(passes[e] * 2 * (1 << e) * S for e in es)
    hbm_gbs = world * step_bytes / (ms_per_step * 1e-3) / 1e9

    num, den = inputs.diff_norms(arena, keep, 1.0)
    accuracy = {"roundtrip_rel_l2_after_all_steps": math.sqrt(num / den), "round_trips": W + K,
                "tolerance_per_round_trip": 2e-14 * wl["emax"] if c128 else 4e-6 * wl["emax"]}

    peak, peak_kind = peaks()
    per_graph_s = statistics.median(graph_ms) * 1e-3
    achieved = step_bytes / 2 / per_graph_s / 1e9
    roofline = {"bound": "hbm", "kernel": "one batch graph launch (all kernels of 256 transforms)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                "peak_kind": f"{peak_kind} STREAM-style copy (MEASURED_PEAKS.json hbm_gbs)",
                "per_launch_ms": per_graph_s * 1e3, "algorithmic_bytes_per_launch": step_bytes / 2,
                "graph_kernel_nodes": kernels // 2}

    e2e = None
    if not args.no_e2e:
        # the public API with host data: every step copies the 256 host arrays
        # in, runs the forward and the inverse batch, copies the results out
        # (efft_batch_execute_host_stream: copies overlapped chunk by chunk)
        hin = inputs.PinnedHost(total, tdt)
        hout = inputs.PinnedHost(total, tdt)
        hin.tensor.copy_(keep)
        hp_in = [hin.ptr + int(o) * S for o in offs[:-1]]
        hp_out = [hout.ptr + int(o) * S for o in offs[:-1]]
        Ke = max(3, K)
        efft.batch_execute_host_stream([fwd, inv], hp_in, hp_out, ptrs, sp)  # warm
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(Ke):
            efft.batch_execute_host_stream([fwd, inv], hp_in, hp_out, ptrs, sp)
        dt = (time.perf_counter() - t0) / Ke
        e2e = {"value": world * step_flop / dt / 1e9, "unit": "GFLOP/s", "h2d_bytes_per_step": total * S,
               "d2h_bytes_per_step": total * S, "ms_per_step": dt * 1e3, "steps": Ke,
               "api": "efft_batch_execute_host_stream (cudaHostAlloc host arrays; per step the 256 "
                      "arrays in, the forward and inverse batches, the results out, copies overlapped "
                      "chunk by chunk)"}
        hin.free()
        hout.free()
        del hin, hout

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        fl, el, k, cores = oracle_batch_time(wl, 20.0)
        cpu = {"value": fl / el / 1e9, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
               "sample": f"forward FP64 radix-2 oracle transforms of the first {k} arrays of the batch, {el:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE_NAME[wl["dtype"]], "data": "synthetic", "config": config_of(wl),
            "hbm_gbs": hbm_gbs, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": K * kernels, "clocks": clocks, "accuracy": accuracy, "impl": "ours",
            "schedules_log2": {str(e): r for e, r in schedules.items()},
        }
        print(json.dumps(line), flush=True)
    fwd.destroy()
    inv.destroy()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    ap.add_argument("--autotune", action="store_true",
                    help="plans with EFFT_FLAG_AUTOTUNE (measured radix schedules; c5 always tunes)")
    ap.add_argument("--radices", default=None,
                    help="explicit schedule, log2 radices comma-separated (profiling of one kernel variant)")
    ap.add_argument("--variant", default=None,
                    help="kernel variant knobs wide,fused_swap,persistent (each -1 rule, 0 off, 1 on; "
                         "efft_plan_set_variant) for measuring one variant")
    ap.add_argument("--no-compare", action="store_true",
                    help="complex64 workloads: skip the complex128 run at the same N")
    ap.add_argument("--no-fp32-form", action="store_true",
                    help="c3: skip the complex64-vs-complex128 comparison at N = 2^31")
    ap.add_argument("--log2n", type=int, default=None,
                    help="override the workload's size (profiling captures on a smaller case)")
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.log2n is not None:
        wl = scale_workload(wl, args.log2n)
    if args.steps is None:
        args.steps = {"c2": 20, "c3": 6, "c1": 200, "c4": 40, "c5": 40, "r1": 20, "m1": 10}[args.workload]
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args, wl)
    if wl.get("batch"):
        return run_batch(args, wl)
    return run_ours(args, wl)


if __name__ == "__main__":
    sys.exit(main())
