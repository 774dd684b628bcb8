"""Benchmark of the fused electrofreezing LB step on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                [--precision f32|f64|f16s]
                [--workload production|precision|batched|serving|regimes]
                [--requests N --max-ny NY --budget-gb G] [--with-oracle]

A step is one pass of the whole hot path over the lattice: two launches, the
halo records of the tile-edge cells and the fused collide-and-stream kernel
(local macros, stencils, forces, four collisions, in-place streaming with
walls); every `--obs-every`-th step also reduces the observables of the
state it starts from inside the same kernel.  The default
workload is the precision case, the largest single-instance configuration:
1024 x 512 lattice, R = 160, theta = 60, PR+ (R_sigma = 2, S = 0.5),
CaE = 0.2, Ste = 0.5, rho_s/rho_l = 0.9, FP32.  L2 is flushed before every
timed step, outside the timed events: a 256 MB buffer is written, then
another 256 MB read, so none of the step's inputs is in L2 and no dirty
line of the flush is left for the step to write back.  Under torchrun
each rank advances its own instance (replicas, no collective on the data
path) and the slowest rank's time counts.

With N = 1 the line also carries, measured after the headline's timed
region: `production_fp32` (512 x 256), `plain_fp64` (the 128 x 64 and
512 x 256 cases in FP64), `fp16s` (the precision case in weight-shifted half
storage), `batched` (64 uneven instances, one launch per step, against the
same instances stepped one after another) and `serving` (a reduced Poisson
stream run to frozen fraction 0.99 under an HBM budget: p50/p99 time to
result); --no-extras leaves them out.

Other workloads (--workload): `production`, `plain` (128 x 64 FP64),
`batched`, `serving`, `regimes` (the production droplet to freezing with the
field off, prolate and oblate; --with-oracle adds the oracle on the
4x-coarsened lattice).  The roofline object is the HBM one for FP32 and
FP16S and the FP64 arithmetic one for FP64, whose step is bound by the FP64
pipe.

--impl reference times the FP64 CPU oracle on the same workload and metric.
"""
from __future__ import annotations

import argparse
import ctypes
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

BYTES_PER_LU = {"f64": 2 * (32 + 7) * 8, "f32": 2 * (32 + 7) * 4, "f16s": 2 * (9 * 4 + 23 * 2) + 2 * 7 * 4}
FALLBACK_HBM_GBS = 6800.0
NOMINAL_FP64_TFLOPS = 1.25     # FP64 rate of the part (nominal; no measured figure exists)


PROFILED_LATTICE = {"production": "512x256", "precision": "1024x512", "plain": "128x64"}


def profile_md(precision: str, workload: str = "production") -> str:
    return os.path.join(ROOT, "profiles", f"k_step_{precision}_{workload}_{PROFILED_LATTICE[workload]}.md")


def kernel_sources(precision: str):
    return ["lbm_kernels.cuh", "lbm_launch.cuh", f"step_{precision}.cu", "lbm_internal.h", "philox.h"]


def kernel_source_hash(precision: str = "f32") -> str:
    h = hashlib.sha256()
    for f in kernel_sources(precision):
        with open(os.path.join(ROOT, "paper_2410_06657_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def profiled(precision: str, workload: str, key: str):
    """A figure of the committed ncu summary of the step kernel (DRAM bytes
    per launch, FP64 flops per lattice update), if the summary was taken on
    the current kernel source; summaries cover the production and precision
    lattices."""
    if workload not in PROFILED_LATTICE:
        return None
    path = profile_md(precision, workload)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_b = re.search(key + r":\s*([0-9.eE+]+)", text)
    m_h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    if not m_b or not m_h or m_h.group(1) != kernel_source_hash(precision):
        return None
    return float(m_b.group(1))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while a region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


class L2Flush:
    """Flush of L2 (129 MB) between timed steps: a 256 MB buffer written,
    then another 256 MB read.  The read evicts the written lines, so the
    next step finds none of its inputs in L2 and no dirty line of the flush
    whose write-back would fall inside its timed region."""

    def __init__(self):
        import torch
        n = 256 * 1024 * 1024 // 4
        self.w = torch.empty(n, dtype=torch.float32, device="cuda")
        self.r = torch.ones(n, dtype=torch.float32, device="cuda")
        self.acc = torch.empty((), dtype=torch.float32, device="cuda")

    def __call__(self):
        import torch
        self.w.fill_(1.0)
        torch.sum(self.r, dim=0, out=self.acc)


def workload(name: str, precision: str):
    from paper_2410_06657_gb300 import workloads as W
    prec = W.PRECISIONS[precision]
    if name == "production":
        w = W.production(precision=prec)
        label = "production sessile droplet 512x256, R=80, theta=90, CaE=0.2, S=2, R_sigma=5, Ste=0.5"
    elif name == "precision":
        w = W.precision_case(precision=prec)
        label = "precision case 1024x512, R=160, theta=60, PR+ (R_sigma=2, S=0.5), CaE=0.2, Ste=0.5"
    elif name == "plain":
        w = W.plain_fp64_small()
        w["params"] = dict(w["params"], precision=prec)
        label = "plain sessile droplet 128x64, R=20, theta=90, CaE=0.2, S=2, R_sigma=5, Ste=0.5"
    else:
        raise SystemExit(f"unknown workload {name}")
    return w, label


def config_for(args, p: dict, label: str, world: int) -> dict:
    """The workload description both arms print (identical keys and values)."""
    return {"workload": label, "cells": p["nx"] * p["ny"], "precision": args.precision, "k_e": p["k_e"],
            "obs_every": args.obs_every, "observation": "fused into the step that reads the observed state",
            "streaming": "in place (AA pattern), one population copy",
            "l2": "flushed before every timed step (256 MB written, then 256 MB read)",
            "parallelism": f"replicas x{world}"}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(value: float, world: int) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# CPU oracle timing (the reported baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_mlups(params: dict, R: float, budget_s: float, max_steps=None):
    """Time the FP64 oracle, as it stands, on this workload's lattice: steps
    from the initial droplet until `budget_s` of CPU work (at least 2)."""
    import oracle
    from paper_2410_06657_gb300 import workloads as W
    o = oracle.Oracle(params)
    xc, yc = W.sessile_center(params["nx"], R, params["theta_deg"])
    o.init_droplet(R, xc, yc, 0)
    o.step(1)                      # warm the caches and pages
    n, t0 = 0, time.perf_counter()
    while True:
        o.step(1)
        n += 1
        el = time.perf_counter() - t0
        if (n >= 2 and el >= budget_s) or (max_steps and n >= max_steps):
            break
    cells = params["nx"] * params["ny"]
    return cells * n / el / 1e6, n, el


def run_reference(args, world, rank):
    from paper_2410_06657_gb300 import workloads as W
    if rank != 0:
        return
    w, label = workload(args.workload, args.precision)
    p = dict(w["params"])
    cells = p["nx"] * p["ny"]
    # one oracle step of the full lattice takes ~0.1-0.3 s; when K + W steps
    # would not fit in about two minutes, each step runs on a 128 x 64 sample
    # lattice with the same physics (the oracle's cost per cell is the same)
    import oracle
    probe = oracle.Oracle(p)
    xc, yc = W.sessile_center(p["nx"], w["R"], p["theta_deg"])
    probe.init_droplet(w["R"], xc, yc, 0)
    t0 = time.perf_counter()
    probe.step(1)
    per_step = time.perf_counter() - t0
    probe.close()
    sample = f"full {p['nx']}x{p['ny']} lattice"
    R = w["R"]
    if per_step * (args.steps + args.warmup) > 120.0:
        scale = p["ny"] / 64.0
        R = w["R"] / scale
        p.update(nx=128, ny=64, R0=R)
        sample = f"128x64 sample lattice, same physics (R={R:g}); full lattice step {per_step:.3f} s"
        cells = 128 * 64
    o = oracle.Oracle(p)
    xc, yc = W.sessile_center(p["nx"], R, p["theta_deg"])
    o.init_droplet(R, xc, yc, 0)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    el = time.perf_counter() - t0
    v = cells * args.steps / el / 1e6
    line = {
        "impl": "reference", "metric": "MLUPS", "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_for(args, dict(w["params"]), label, world),
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} FP64 oracle steps on the {sample}, 1 thread"},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args, world, rank, local):
    import numpy as np
    import torch
    from paper_2410_06657_gb300 import lbm, workloads as W

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lbm.load()
    w, label = workload(args.workload, args.precision)
    p = dict(w["params"])
    cells = p["nx"] * p["ny"]
    stream = torch.cuda.current_stream()
    sim = lbm.Simulation(p, stream)
    xc, yc = W.sessile_center(p["nx"], w["R"], p["theta_deg"])
    sim.init_droplet(w["R"], xc, yc, 0)
    flush_l2 = L2Flush()

    obs_every = args.obs_every
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    # the clock sampler starts before the warm-up steps, so the timed steps
    # follow the warm-up without an idle gap
    sampler = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
    sampler.start()
    time.sleep(0.3)
    # the warm-up's first two steps both observe, so the observing kernels of
    # both layout phases are loaded before the timed steps
    for i in range(args.warmup):
        flush_l2()
        if i % obs_every == 0 or i < 2:
            sim.observables_deferred()
        sim.step(1)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    # two events bracket each step.  Every obs_every-th step also reduces the
    # observables of the state it starts from, inside its own kernel
    # (lbm_observables_deferred): one pass over the lattice, not two.
    observe = [i % obs_every == 0 for i in range(args.steps)]
    for i in range(args.steps):
        flush_l2()
        a, _, c = ev[i]
        a.record(stream)
        if observe[i]:
            sim.observables_deferred()
        sim.step(1)
        c.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    # the plain step kernel's launches (the observing steps run another kernel)
    step_ms = [ev[i][0].elapsed_time(ev[i][2]) for i in range(args.steps) if not observe[i]]
    obs_step_ms = [ev[i][0].elapsed_time(ev[i][2]) for i in range(args.steps) if observe[i]]
    tot_ms = [ev[i][0].elapsed_time(ev[i][2]) for i in range(args.steps)]
    total_s = reduce_max(sum(tot_ms) / 1e3, world)
    obs = sim.observables_fetch()
    value = world * cells * args.steps / total_s / 1e6
    launch_us = 1e3 * statistics.mean(step_ms)

    # roofline of the dominant kernel (the fused step)
    bpl = BYTES_PER_LU[args.precision]
    alg_bytes = bpl * cells
    achieved = alg_bytes / (launch_us * 1e-6) / 1e9
    peak, peak_kind = measured_peak()
    traffic = profiled(args.precision, args.workload, "traffic_bytes_per_launch")

    # context for the fraction: a plain device copy moving the same bytes
    # (half read, half written), timed the same way (L2 flushed, events);
    # one launch of this size cannot reach the streaming bandwidth
    src = torch.ones(alg_bytes // 8, dtype=torch.float32, device="cuda")
    dst = torch.empty_like(src)
    cev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(50)]
    for _ in range(3):
        flush_l2()
        dst.copy_(src)
    for a, b in cev:
        flush_l2()
        a.record(stream)
        dst.copy_(src)
        b.record(stream)
    torch.cuda.synchronize()
    copy_us = 1e3 * statistics.mean(a.elapsed_time(b) for a, b in cev)
    del src, dst

    # steady state (informational): a long graph-replayed run, L2 warm
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_ss = 2048
    s0.record(stream)
    sim.step(n_ss)
    s1.record(stream)
    torch.cuda.synchronize()
    ss_mlups = cells * n_ss / (s0.elapsed_time(s1) / 1e3) / 1e6

    # end to end through the C ABI with host buffers: every step uploads the
    # whole state from pinned host memory, steps, and copies its observables
    # into pinned host memory (streamed: the host enqueues the steps without
    # a round trip each and waits once, then checks every record)
    nbytes = sim.state_bytes()
    host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    sim.export_state(host.numpy())
    k_e2e = max(10, min(args.steps, 200))
    osz = ctypes.sizeof(lbm.Obs)
    obs_host = torch.zeros(k_e2e * osz, dtype=torch.uint8, pin_memory=True)
    # untimed: the first import allocates its device buffers, and both layout
    # phases of the observables kernel get loaded
    for i in range(2):
        sim.import_state(host.data_ptr())
        sim.step(1)
        sim.observables_to_host(obs_host.data_ptr() + i * osz)
    sim.sync()
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for i in range(k_e2e):
        sim.import_state(host.data_ptr())
        sim.step(1)
        sim.observables_to_host(obs_host.data_ptr() + i * osz)
    sim.sync()
    e2e_s = reduce_max(time.perf_counter() - t0, world)
    e2e_value = world * cells * k_e2e / e2e_s / 1e6
    e2e_obs = [lbm.Obs.from_address(obs_host.data_ptr() + i * osz).as_dict() for i in range(k_e2e)]
    if any(o["status"] != 0 or o["step"] != e2e_obs[0]["step"] for o in e2e_obs):
        raise RuntimeError("end-to-end observables: a step diverged or read a wrong state")

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v, n, el = oracle_mlups(p, w["R"], budget_s=args.cpu_budget)
        cpu = {"value": v, "unit": "MLUPS", "cores": 1, "kind": "oracle",
               "sample": f"{n} FP64 oracle steps of the same {p['nx']}x{p['ny']} lattice from the "
                         f"initial droplet ({el:.1f} s, 1 thread)"}
    line = {
        "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": config_for(args, p, label, world),
        "observing_step_us": 1e3 * statistics.mean(obs_step_ms) if obs_step_ms else None,
        "roofline": roofline_f64(args, cells, launch_us, traffic) if args.precision == "f64" else {
                     "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": f"k_halo + k_step<{args.precision}> (one step, both launches timed)", "launch_us": launch_us,
                     "algorithmic_bytes_per_launch": alg_bytes, "bytes_per_lu": bpl,
                     "copy_same_bytes": {"launch_us": copy_us, "gbs": alg_bytes / (copy_us * 1e-6) / 1e9,
                                         "frac": alg_bytes / (copy_us * 1e-6) / 1e9 / peak,
                                         "note": "device-to-device copy of the same byte count, same timing"},
                     },
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": ctypes.sizeof(lbm.Obs), "steps": k_e2e,
                "note": "per step: lbm_import_state from pinned host memory, lbm_step(1), "
                        "lbm_observables_to_host into pinned host memory; one lbm_sync at the end"},
        # halo records + step (k_e - 1 sweeps more), and the finish launch of each observing step
        "gpu_launches": args.steps * (p["k_e"] + 1) + sum(observe),
        "clocks": clocks,
        "steady_state": {"value": ss_mlups, "unit": "MLUPS",
                         "note": f"lbm_step({n_ss}) graph replay, state resident in L2 (informational)"},
        "observables": {k: obs[k] for k in ("step", "mass", "frozen_fraction", "height", "width", "status")},
        "state_bytes_device": sim.device_bytes(),
    }
    sim.close()
    del flush_l2
    if world == 1 and not args.no_extras:
        line.update(extras(args))
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def roofline_f64(args, cells, launch_us, traffic):
    """The FP64 step is bound by FP64 arithmetic, not HBM: FP64 operations
    per launch (DADD, DMUL one each, DFMA two, counted by ncu on this kernel
    source) over the launch time, against the part's nominal FP64 rate."""
    flops_lu = profiled("f64", args.workload, "fp64_flops_per_lu")
    if flops_lu is None:
        return {"bound": "alu", "achieved": None, "peak": NOMINAL_FP64_TFLOPS, "unit": "TFLOP/s",
                "frac": None, "traffic": traffic, "peak_kind": "nominal",
                "kernel": "k_halo + k_step<f64> (one step, both launches timed)", "launch_us": launch_us,
                "note": "FP64 operation count not profiled for this source"}
    tflops = flops_lu * cells / (launch_us * 1e-6) / 1e12
    return {"bound": "alu", "achieved": tflops, "peak": NOMINAL_FP64_TFLOPS, "unit": "TFLOP/s",
            "frac": tflops / NOMINAL_FP64_TFLOPS, "traffic": traffic, "peak_kind": "nominal",
            "kernel": "k_halo + k_step<f64> (one step, both launches timed)", "launch_us": launch_us, "fp64_flops_per_lu": flops_lu}


# ---------------------------------------------------------------------------
# The other configurations, measured after the headline's timed region
# ---------------------------------------------------------------------------

def step_rate(name: str, precision: str, steps: int, warmup: int = 3):
    """MLUPS and the step kernel's roofline on one workload: `steps` timed
    steps, each bracketed by two events with L2 flushed before it."""
    import torch
    from paper_2410_06657_gb300 import lbm, workloads as W
    w, label = workload(name, precision)
    p = dict(w["params"])
    cells = p["nx"] * p["ny"]
    stream = torch.cuda.current_stream()
    sim = lbm.Simulation(p, stream)
    xc, yc = W.sessile_center(p["nx"], w["R"], p["theta_deg"])
    sim.init_droplet(w["R"], xc, yc, 0)
    flush = L2Flush()
    for _ in range(warmup):
        flush()
        sim.step(1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for a, b in ev:
        flush()
        a.record(stream)
        sim.step(1)
        b.record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    launch_us = 1e3 * statistics.mean(ms)
    o = sim.observables()
    out = {"workload": label, "precision": precision, "cells": cells, "steps": steps,
           "value": cells / (launch_us * 1e-6) / 1e6, "unit": "MLUPS", "launch_us": launch_us,
           "state_bytes_device": sim.device_bytes(), "status": o["status"]}
    if precision == "f64":
        out["roofline"] = roofline_f64(argparse.Namespace(workload=name), cells, launch_us,
                                       profiled("f64", name, "traffic_bytes_per_launch"))
    else:
        peak, kind = measured_peak()
        gbs = BYTES_PER_LU[precision] * cells / (launch_us * 1e-6) / 1e9
        out["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                           "peak_kind": kind, "bytes_per_lu": BYTES_PER_LU[precision],
                           "traffic": profiled(precision, name, "traffic_bytes_per_launch")}
    sim.close()
    return out


def extras(args):
    out = {}
    t0 = time.perf_counter()
    out["production_fp32"] = step_rate("production", "f32", 50)
    out["plain_fp64"] = {"128x64": step_rate("plain", "f64", 50), "512x256": step_rate("production", "f64", 20)}
    out["fp16s"] = step_rate("precision", "f16s", 20)
    out["batched"] = batched_rate("f32", steps=64, warmup=32)
    out["serving"] = serving_rate("f32", requests=args.extra_requests, max_ny=128, budget_gb=80.0)
    out["extras_wall_s"] = time.perf_counter() - t0
    return out


def batched_rate(precision: str, steps: int, warmup: int, rank: int = 0):
    """64 uneven instances (C4): one launch per step for all of them against
    the same instances advanced one after another (each replaying its own
    graph of 32 steps), both on the members' own data."""
    import torch
    from paper_2410_06657_gb300 import lbm, workloads as W
    stream = torch.cuda.current_stream()
    prec = W.PRECISIONS[precision]
    items = W.batched(n=64, seed=2410066570 + rank, precision=prec)
    sims = []
    for it in items:
        p = it["params"]
        s = lbm.Simulation(p, stream)
        xc, yc = W.sessile_center(p["nx"], it["R"], p["theta_deg"])
        s.init_droplet(it["R"], xc, yc, 0)
        sims.append(s)
    cells = sum(it["params"]["nx"] * it["params"]["ny"] for it in items)

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3

    for s in sims:
        s.step(warmup)
    t_plain = timed(lambda: [s.step(steps) for s in sims])
    batch = lbm.Batch(sims, stream, tile_rows=0)
    batch.step(warmup)
    t_batch = timed(lambda: batch.step(steps))
    v_batch, v_plain = cells * steps / t_batch / 1e6, cells * steps / t_plain / 1e6
    state = sum(s.device_bytes() for s in sims)
    tile_rows = batch.tile_rows
    batch.close()
    for s in sims:
        s.close()
    return {"workload": "64 instances, sizes uniform in {128x64 .. 512x256}, seeded CaE/R/S/theta/Ste draws",
            "precision": precision, "cells": cells, "steps": steps, "value": v_batch, "unit": "MLUPS",
            "plain_one_after_another": v_plain, "batched_over_plain": v_batch / v_plain, "tile_rows": tile_rows,
            "hbm_gbs_algorithmic": BYTES_PER_LU[precision] * cells * steps / t_batch / 1e9,
            "state_bytes_device": state}


def serving_rate(precision: str, requests: int, max_ny: int, budget_gb: float, rank: int = 0):
    """A Poisson stream (C5's arrival rate and parameter draws, a stated
    number of requests and largest lattice) served to frozen fraction 0.99."""
    import numpy as np
    import torch
    from paper_2410_06657_gb300 import workloads as W
    from paper_2410_06657_gb300.serving import Request, Server
    stream = torch.cuda.current_stream()
    prec = W.PRECISIONS[precision]
    items = W.serving_stream(n=requests, rate=20.0, seed=2410066571 + rank, max_ny=max_ny, precision=prec)
    reqs = []
    for it in items:
        p = it["params"]
        xc, yc = W.sessile_center(p["nx"], it["R"], p["theta_deg"])
        reqs.append(Request(id=it["id"], arrival=it["arrival"], params=p, R=it["R"], xc=xc, yc=yc))
    srv = Server(int(budget_gb * 1e9), stream, chunk=200)
    t0 = time.perf_counter()
    res = srv.run(reqs)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    lat = np.array([r.latency for r in res])
    lu = srv.lattice_updates
    return {"workload": f"{requests} Poisson arrivals at 20/s (seed 2410066571), sizes up to {2 * max_ny}x{max_ny}, "
                        f"C4 parameter draws, each run to frozen fraction 0.99", "precision": precision,
            "budget_gb": budget_gb, "chunk": 200, "value": lu / wall / 1e6, "unit": "MLUPS",
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "max": float(lat.max())},
            "hbm_gbs_algorithmic": lu * BYTES_PER_LU[precision] / wall / 1e9,
            "gpu_busy_fraction": srv.gpu_busy_s / wall if wall > 0 else None,
            "all_frozen": bool(all(r.frozen for r in res)), "wall_s": wall}


# ---------------------------------------------------------------------------
# Batched workload: 64 uneven instances, one launch per step, against the same
# instances advanced one after another
# ---------------------------------------------------------------------------

def run_batched(args, world, rank, local):
    import torch
    from paper_2410_06657_gb300 import lbm, workloads as W

    torch.cuda.set_device(local)
    lbm.load()
    stream = torch.cuda.current_stream()
    prec = W.PRECISIONS[args.precision]
    items = W.batched(n=64, seed=2410066570 + rank, precision=prec)
    sims = []
    for it in items:
        p = it["params"]
        s = lbm.Simulation(p, stream)
        xc, yc = W.sessile_center(p["nx"], it["R"], p["theta_deg"])
        s.init_droplet(it["R"], xc, yc, 0)
        sims.append(s)
    cells = sum(it["params"]["nx"] * it["params"]["ny"] for it in items)
    K = args.steps

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3

    # plain: each instance's K steps (graph-replayed) one after another
    for s in sims:
        s.step(args.warmup)
    t_plain = timed(lambda: [s.step(K) for s in sims])
    batch = lbm.Batch(sims, stream, tile_rows=0)
    batch.step(args.warmup)
    barrier(world)
    t_batch = timed(lambda: batch.step(K))
    t_batch = reduce_max(t_batch, world)
    v_batch = world * cells * K / t_batch / 1e6
    v_plain = cells * K / t_plain / 1e6
    state_gb = sum(s.state_bytes() for s in sims) / 1e9
    if rank == 0:
        print(json.dumps({
            "metric": "MLUPS", "value": v_batch, "unit": "MLUPS", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_batch / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": "batched: 64 instances, sizes uniform in {128x64 .. 512x256}, seeded "
                                   "CaE/R/S/theta/Ste draws", "cells": cells,
                       "tile_rows": batch.tile_rows,
                       "l2": f"state ({state_gb:.2f} GB) larger than L2"},
            "plain_one_after_another": {"value": v_plain, "unit": "MLUPS"},
            "batched_over_plain": v_batch / v_plain,
            "gpu_launches": K * (items[0]["params"]["k_e"] + 1),
        }))


# ---------------------------------------------------------------------------
# Serving: Poisson arrivals, continuous batching, p50/p99 time to result
# ---------------------------------------------------------------------------

def run_serving(args, world, rank, local):
    import numpy as np
    import torch
    from paper_2410_06657_gb300 import lbm, workloads as W
    from paper_2410_06657_gb300.serving import Request, Server

    torch.cuda.set_device(local)
    lbm.load()
    stream = torch.cuda.current_stream()
    prec = W.PRECISIONS[args.precision]
    stream_items = W.serving_stream(n=args.requests, rate=20.0, seed=2410066571 + rank,
                                    max_ny=args.max_ny, precision=prec)
    reqs = []
    for it in stream_items:
        p = it["params"]
        xc, yc = W.sessile_center(p["nx"], it["R"], p["theta_deg"])
        reqs.append(Request(id=it["id"], arrival=it["arrival"], params=p, R=it["R"], xc=xc, yc=yc))
    srv = Server(int(args.budget_gb * 1e9), stream, chunk=200)
    barrier(world)
    t0 = time.perf_counter()
    res = srv.run(reqs)
    torch.cuda.synchronize()
    wall = reduce_max(time.perf_counter() - t0, world)
    lat = np.array([r.latency for r in res])
    lu = srv.lattice_updates
    bpl = BYTES_PER_LU[args.precision]
    if rank == 0:
        print(json.dumps({
            "metric": "MLUPS", "value": world * lu / wall / 1e6, "unit": "MLUPS", "n_gpus": world,
            "steps": int(lu), "warmup": 0, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": f"serving: {args.requests} Poisson arrivals at 20/s, sizes up to "
                                   f"{2 * args.max_ny}x{args.max_ny}, run to frozen fraction 0.99",
                       "budget_gb": args.budget_gb, "chunk": 200},
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "max": float(lat.max())},
            "hbm_gbs_algorithmic": lu * bpl / wall / 1e9,
            "all_frozen": bool(all(r.frozen for r in res)), "wall_s": wall,
        }))


# ---------------------------------------------------------------------------
# Regimes: the production droplet run to freezing with the field off, prolate
# (PR+) and oblate (OB-); optionally the oracle on the 4x-coarsened lattice
# (128 x 64, R = 20, same tau: 16x fewer steps for the same Fourier number)
# ---------------------------------------------------------------------------

def _freeze(sim, every, max_steps):
    """Step until t_fre; return (t_fre, Fo_fre, aspect and height at t_fre, steps)."""
    while sim.t < max_steps:
        sim.step(every)
        o = sim.observables()
        if o["status"] != 0:
            break
        if o["t_fre"] >= 0:
            return o
    return sim.observables()


def run_regimes(args, world, rank, local):
    import torch
    from paper_2410_06657_gb300 import lbm, workloads as W

    torch.cuda.set_device(local)
    lbm.load()
    stream = torch.cuda.current_stream()
    prec = W.PRECISIONS[args.precision]
    # the configuration of Sec. 5.4, Fig. 14(b) (Ste = 0.2, theta = 120,
    # CaE = 1, the whole region initially at T_m + (T_m - T_w) / 2) on the
    # 512 x 256 lattice, R = 80
    cases = [("field off", None, 0.0), ("OB-", "OB-", 1.0), ("PR-", "PR-", 1.0), ("PR+", "PR+", 1.0)]
    out, lu, t_gpu = [], 0, 0.0
    t_off = None
    for name, regime, ca in cases:
        w = W.production(precision=prec, regime=regime, CaE=ca)
        p = dict(w["params"], Ste=0.2, theta_deg=120.0, alpha_lg=0.2, rho_sl=0.9,
                 T_init=0.5 * (w["params"]["T_m"] - w["params"]["T_w"]) + w["params"]["T_m"])
        sim = lbm.Simulation(p, stream)
        xc, yc = W.sessile_center(p["nx"], w["R"], p["theta_deg"])
        sim.init_droplet(w["R"], xc, yc, 0)
        sim.presolve(1e-6, 200000)
        probe = int(round(0.3125 * w["R"] ** 2 / p["alpha_l"]))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.step(probe)
        op = sim.observables()
        o = _freeze(sim, 50, 1000000)
        torch.cuda.synchronize()
        t_gpu += time.perf_counter() - t0
        lu += p["nx"] * p["ny"] * sim.t
        if regime is None:
            t_off = o["t_fre"]
        rec = {"case": name, "t_fre": o["t_fre"], "Fo_fre": o["Fo_fre"], "aspect": o["aspect"],
               "height": o["height"], "frozen_fraction": o["frozen_fraction"],
               "height_at_Fo_0.3125": op["height"], "R_tr_at_Fo_0.3125": op["R_tr"]}
        if t_off and o["t_fre"] > 0:
            rec["t_star"] = (o["t_fre"] - t_off) / t_off
        if args.with_oracle and rank == 0:
            import oracle
            pc = dict(p, nx=128, ny=64, R0=w["R"] / 4, precision=W.FP64)
            orc = oracle.Oracle(pc)
            xcc, ycc = W.sessile_center(128, w["R"] / 4, p["theta_deg"])
            orc.init_droplet(w["R"] / 4, xcc, ycc, 0)
            oo = orc.observables()
            while orc.t < 400000 // 16 and oo["t_fre"] < 0:
                orc.step(50)
                oo = orc.observables()
            rec["oracle_128x64"] = {"t_fre": oo["t_fre"], "Fo_fre": oo["Fo_fre"], "aspect": oo["aspect"],
                                    "height_x4": 4 * oo["height"]}
            if oo["Fo_fre"] > 0 and o["Fo_fre"] > 0:
                rec["Fo_fre_rel_diff"] = o["Fo_fre"] / oo["Fo_fre"] - 1
                rec["aspect_rel_diff"] = o["aspect"] / oo["aspect"] - 1
        out.append(rec)
        sim.close()
    if rank == 0:
        print(json.dumps({
            "metric": "MLUPS", "value": world * lu / t_gpu / 1e6, "unit": "MLUPS", "n_gpus": world,
            "steps": int(lu), "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": "droplet 512x256, R=80, run to frozen fraction 0.99 in the configuration of "
                                   "Fig. 14(b): Ste=0.2, theta=120, CaE=1, initial T = T_m + (T_m - T_w)/2; "
                                   "field off, OB- (R_sigma=2, S=5), PR- (5, 9.5), PR+ (2, 0.5)",
                       "observables_every": 50},
            "cases": out,
        }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="f32", choices=["f32", "f64", "f16s"])
    ap.add_argument("--workload", default="precision",
                    choices=["precision", "production", "plain", "batched", "serving", "regimes"])
    ap.add_argument("--no-extras", action="store_true", help="headline line only")
    ap.add_argument("--extra-requests", type=int, default=48, help="requests of the serving extra")
    ap.add_argument("--requests", type=int, default=32)
    ap.add_argument("--max-ny", type=int, default=128)
    ap.add_argument("--budget-gb", type=float, default=80.0)
    ap.add_argument("--obs-every", type=int, default=10)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--with-oracle", action="store_true",
                    help="regimes: also run the oracle on the 4x-coarsened lattice")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload == "batched":
        run_batched(args, world, rank, local)
        return
    if args.workload == "serving":
        run_serving(args, world, rank, local)
        return
    if args.workload == "regimes":
        run_regimes(args, world, rank, local)
        return
    run_gpu(args, world, rank, local)


if __name__ == "__main__":
    main()
