#!/usr/bin/env python
"""Benchmark of the RK-3 off-lattice Boltzmann step (node-updates/s).

Default workload: the planar liquid-vapour set-up between diffuse walls,
1024 x 8 nodes (walls at x = 0, 1, periodic y), T_w = 0.9,
n = 1 + 0.01 U(-1, 1), tau = 0.005, dt = 5e-5, in FP64; the FP32 + Kahan
variant is timed beside it and its error against the FP64 path stated.
A "step" is one full RK-3 step (3 x moments + fused stage) of the whole grid.

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events
on the context's stream, with a 256 MiB buffer written between steps so L2
(129 MB) holds nothing of the step's data; barrier + synchronize on both
sides; max over ranks.  With torchrun (N > 1) every rank runs an
independent replica (the path has no data exchange to shard): value is the
node-updates of all ranks per second.

Also reported: per-kernel roofline of the dominant kernel (CUDA events on
its launching stream), end-to-end throughput through the C ABI with pinned
host buffers, the FP64 oracle timed on the host cores, SM clocks sampled
during the timed region.  ``--impl reference`` times the FP64 oracle alone.
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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "node-updates/s (25-vel RK3 step) vs plain FP64 at stated error; % of roofline"
UNIT = "node-updates/s"

# Algorithmic flops of one stage per node (FMA = 2), counted formula by
# formula: moments 110, force stencils 172,
# equilibrium factors 104, local part of L and RK combination 25 x 30 = 750,
# WENO-5 faces 40 x 57 = 2280 (20 moving velocities per axis, one face per
# node), advection and output 155.  The FP32 variant adds the Kahan
# compensation of the four 25-term moment sums (+365).
STAGE_FLOPS_PER_NODE = 110 + 172 + 104 + 750 + 2280 + 155
STAGE_FLOPS_PER_NODE_FP32 = STAGE_FLOPS_PER_NODE + 365
# Population values moved per node and step: stage 1 reads f and writes f1
# (50), stages 2 and 3 read f^n and f_s and write (75 each): 200 per step.
VALUES_PER_NODE_STEP = 200

# Peaks from unit counts and the 2.07 GHz maximum SM clock: FP64 2 DFMA per
# SM per clock (1.20 TFLOP/s measured at 1.97 GHz with an FMA loop),
# 152 x 2 x 2 x 2.07e9 = 1.26 TFLOP/s; FP32 128 lanes per SM,
# 152 x 128 x 2 x 2.07e9 = 80.5 TFLOP/s.
PEAK_FP64_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# DRAM bytes (read + write) per stage launch, averaged over the three stages of
# a step, from one ncu capture of exactly this kernel build on this workload
# (stage 1: 1.71 MB, stages 2 and 3: 3.35 MB each; writes still in L2).  Any
# other kernel or workload reports null.
DRAM_TRAFFIC_PER_LAUNCH = {("planar", None, "k_fused<double,7,8,8>"): 2.81e6}
PEAK_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def workload(name, size=None):
    from paper_1702_01690_gb300 import inputs
    if name == "planar":
        p, f = inputs.planar_walls()
        desc = (f"planar liquid-vapour interface {p.nx}x{p.ny}, diffuse walls x=0,1, periodic y, Tw=0.9, "
                f"tau={p.tau:g}, dt={p.dt:g}")
    elif name == "shear":
        p, f = inputs.shear_64x4()
        desc = "shear-wave decay 64x4 periodic, T0=1.1, tau=0.01, dt=0.002"
    elif name == "laplace":
        n = size or 2048
        p, f = inputs.laplace(n, R=0.2)
        desc = f"Laplace drop {n}^2 periodic, R=0.2, T=0.9, tau=5e-3, dt={p.dt:g}"
    elif name == "phase":
        n = size or 4096
        p, f = inputs.phase_separation(n)
        desc = f"phase separation {n}^2, diffuse walls, Tw=0.7, tau=5e-3, dt={p.dt:g}"
    else:
        raise SystemExit(f"unknown workload {name}")
    return p, f, desc


# ------------------------------------------------------------------ clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.proc or not self.path:
            return None
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ oracle legs
def oracle_rate(p, fields, seconds: float, max_steps: int = 10 ** 6):
    """FP64 oracle node-updates/s on the host cores: whole-grid steps until
    `seconds` of CPU work (at least one step)."""
    import oracle
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    o = oracle.Oracle(p.nx, p.ny, p.ds, p.dt, p.tau, p.a, p.b, p.sigma, p.Tw, p.uw, p.side_x, p.side_y)
    o.init_fields(*fields)
    steps = 0
    t0 = time.perf_counter()
    while True:
        o.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds or steps >= max_steps:
            break
    return p.nx * p.ny * steps / el, steps, el, oracle.max_threads()


def oracle_sample_params(p, fields, max_nodes=1 << 16):
    """Bounded sample of a large workload: the top-left window of at most
    max_nodes nodes with the same parameters (walls kept)."""
    if p.nx * p.ny <= max_nodes:
        return p, fields, f"full grid {p.nx}x{p.ny}"
    from paper_1702_01690_gb300 import inputs
    w = int(math.sqrt(max_nodes))
    wx, wy = min(p.nx, w), min(p.ny, max_nodes // min(p.nx, w))
    q = inputs.RunParams(**{**p.as_dict(), "nx": wx, "ny": wy})
    sub = tuple(np.ascontiguousarray(a[:wy, :wx]) for a in fields)
    return q, sub, f"{wx}x{wy} window of the {p.nx}x{p.ny} grid"


def run_reference(args, rank, world):
    if rank != 0:
        return
    p, fields, desc = workload(args.workload, args.size)
    q, sub, what = oracle_sample_params(p, fields)
    # untimed warm-up steps, then K timed whole-grid steps of the sample
    import oracle
    oracle.set_threads(os.cpu_count() or 1)
    o = oracle.Oracle(q.nx, q.ny, q.ds, q.dt, q.tau, q.a, q.b, q.sigma, q.Tw, q.uw, q.side_x, q.side_y)
    o.init_fields(*sub)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    el = time.perf_counter() - t0
    v = q.nx * q.ny * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc, "sample": what},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": f"{args.steps} RK-3 steps of the {what}"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ranks
def rank_barrier():
    """Barrier over the ranks of the default process group (none without one)."""
    import torch.distributed as tdist
    if tdist.is_available() and tdist.is_initialized() and tdist.get_world_size() > 1:
        tdist.barrier()


def max_over_ranks(value: float) -> float:
    """Largest value over the ranks of the default process group (a CPU
    tensor for gloo, a CUDA tensor for NCCL); the value itself without one."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if tdist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, nodes: int, steps: int, ms: float) -> float:
    """Whole-job node-updates/s: every rank advanced `nodes` nodes `steps`
    times in the slowest rank's `ms` milliseconds."""
    return world * nodes * steps / (ms / 1e3)


# ------------------------------------------------------------------ GPU leg
def time_steps(ctx, steps, warmup, flush, stream):
    import torch
    for _ in range(warmup):
        ctx.step_async(1)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k & 0xFF)
        evs[k][0].record(stream)
        ctx.step_async(1)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in evs]
    st = ctx.status()
    if st != 0:
        raise RuntimeError(f"step status {st}")
    return sum(ms), ms


def run_ours(args, rank, world):
    import torch
    from paper_1702_01690_gb300 import olb

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    p, fields, desc = workload(args.workload, args.size)
    N = p.nx * p.ny
    olb.use_torch_allocator(True)
    dev_fields = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in fields]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    ctx = olb.create(p, olb.FP64, stream)
    ctx.init_fields(*dev_fields)
    torch.cuda.synchronize()
    rank_barrier()
    with ClockSampler(local) as clk:
        total_ms, _ = time_steps(ctx, args.steps, args.warmup, flush, stream)
    torch.cuda.synchronize()
    rank_barrier()
    total_ms = max_over_ranks(total_ms)
    ms_step = total_ms / args.steps
    value = job_value(world, N, args.steps, total_ms)
    m64 = ctx.moments()

    # dominant kernel: per-launch device time of each kernel kind
    prof = ctx.profile(max(3, min(args.steps, 50)))
    st_ms = prof["stage_ms"]
    achieved = STAGE_FLOPS_PER_NODE * N / (st_ms * 1e-3) / 1e12
    tile = ctx.get_tile()
    kname = f"k_fused<double,{tile[0]},{tile[1]},{tile[2]}>"
    roof = {"kernel": f"{kname} (moments + force + WENO-5 + BGK + RK-3 stage)",
            "bound": "alu", "achieved": achieved, "peak": PEAK_FP64_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / PEAK_FP64_TFLOPS,
            "traffic": DRAM_TRAFFIC_PER_LAUNCH.get((args.workload, args.size, kname)),
            "peak_source": "FP64 units x max SM clock (2 DFMA/SM/clk x 152 x 2.07 GHz)",
            "algorithmic_flops_per_launch": STAGE_FLOPS_PER_NODE * N,
            "stage_ms": st_ms, "stage_share": 3 * st_ms / ms_step if ms_step > 0 else None}

    # FP32 + Kahan variant on the same workload
    ctx32 = olb.create(p, olb.FP32_KAHAN, stream)
    ctx32.init_fields(*dev_fields)
    torch.cuda.synchronize()
    rank_barrier()
    total32, _ = time_steps(ctx32, args.steps, args.warmup, flush, stream)
    rank_barrier()
    total32 = max_over_ranks(total32)
    m32 = ctx32.moments()
    prof32 = ctx32.profile(max(3, min(args.steps, 50)))
    ach32 = STAGE_FLOPS_PER_NODE_FP32 * N / (prof32["stage_ms"] * 1e-3) / 1e12
    tile32 = ctx32.get_tile()
    us = max(np.max(np.abs(m64[1])), np.max(np.abs(m64[2])), 1e-300)
    err32 = {"n": float(np.max(np.abs(m32[0] - m64[0])) / np.max(np.abs(m64[0]))),
             "u": float(max(np.max(np.abs(m32[1] - m64[1])), np.max(np.abs(m32[2] - m64[2]))) / us),
             "T": float(np.max(np.abs(m32[3] - m64[3])) / np.max(np.abs(m64[3])))}
    v32 = job_value(world, N, args.steps, total32)
    fp32 = {"value": v32, "ms_per_step": total32 / args.steps, "speedup_vs_fp64": v32 / value,
            "max_rel_err_vs_fp64_after_steps": err32, "steps_compared": args.warmup + args.steps,
            "roofline": {"kernel": f"k_fused<float,{tile32[0]},{tile32[1]},{tile32[2]}>", "bound": "alu", "achieved": ach32,
                         "peak": PEAK_FP32_TFLOPS, "unit": "TFLOP/s", "frac": ach32 / PEAK_FP32_TFLOPS,
                         "stage_ms": prof32["stage_ms"]}}
    ctx32.close()

    # end to end through the C ABI with pinned host buffers
    host_in = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in fields]
    host_out = [torch.empty((p.ny, p.nx), dtype=torch.float64).pin_memory() for _ in range(4)]
    e2e_iters = max(3, min(args.steps, 50))
    ctx.init_fields(*[h.numpy() for h in host_in])
    torch.cuda.synchronize()
    rank_barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_iters):
        ctx.init_fields(*[h.numpy() for h in host_in])
        ctx.step_async(1)  # olb_moments synchronises; the status word is sticky
        olb._check(olb.library().olb_moments(ctx.handle, *[olb._VP(h.data_ptr()) for h in host_out]), "olb_moments")
    e2e_s = (time.perf_counter() - t0) / e2e_iters
    rank_barrier()
    e2e_s = max_over_ranks(e2e_s)
    if ctx.status() != 0:
        raise RuntimeError("e2e: step status")
    e2e = {"value": job_value(world, N, 1, 1e3 * e2e_s), "unit": UNIT, "h2d_bytes_per_step": 4 * N * 8,
           "d2h_bytes_per_step": 4 * N * 8,
           "what": "olb_init_fields (host, pinned) + olb_step_async(1) + olb_moments (host, pinned) per step"}
    ctx.close()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "nodes": N, "grid": [p.nx, p.ny],
                       "l2": "256 MiB buffer written between timed steps",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roof, "fp32_kahan": fp32, "e2e": e2e,
            "gpu_launches": 3 * args.steps, "clocks": clk.summary()}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, steps, el, cores = oracle_rate(p, fields, args.cpu_seconds)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{steps} whole-grid RK-3 steps of the {p.nx}x{p.ny} workload ({el:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_batch(args, rank, world):
    """64 independent runs of uneven sizes (32^2 .. 1024^2 shear and
    longitudinal waves, Laplace drops, planar wall runs; 13.5 M nodes) in one
    persistent launch per stage, replayed from CUDA graphs, shape autotuned.
    The working set (3 x 25 x 13.5 M values) is far larger than L2."""
    import torch
    from paper_1702_01690_gb300 import inputs, olb
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    runs = inputs.batch_sweep()
    nodes = sum(p.nx * p.ny for p, _ in runs)
    out = {}
    for name, prec in (("fp64", olb.FP64), ("fp32_kahan", olb.FP32_KAHAN)):
        b = olb.Batch([p for p, _ in runs], prec, stream)
        for r, (p, fl) in enumerate(runs):
            b.init_fields(r, *fl)
        shape = b.autotune(2)
        b.step(args.warmup)
        torch.cuda.synchronize()
        rank_barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            e0.record(stream)
            b.step_async(args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
        rank_barrier()
        ms = max_over_ranks(e0.elapsed_time(e1))
        rc, _ = b.status()
        if rc != 0:
            raise RuntimeError(f"batch diverged ({name})")
        stage_ms = b.profile(2)
        flops = (STAGE_FLOPS_PER_NODE if prec == olb.FP64 else STAGE_FLOPS_PER_NODE_FP32) * nodes
        peak = PEAK_FP64_TFLOPS if prec == olb.FP64 else PEAK_FP32_TFLOPS
        ach = flops / (stage_ms * 1e-3) / 1e12
        out[name] = {"value": job_value(world, nodes, args.steps, ms), "ms_per_step": ms / args.steps,
                     "shape": list(shape), "stage_ms": stage_ms,
                     "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                                  "frac": ach / peak}, "clocks": clk.summary()}
        b.close()
        del b
        torch.cuda.empty_cache()
    line = {"metric": METRIC, "value": out["fp64"]["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": out["fp64"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "batched sweep: 64 runs 32^2..1024^2 (waves, Laplace drops, planar walls)",
                       "runs": len(runs), "nodes": nodes, "l2": "working set 8.1 GB (FP64) > L2"},
            "roofline": out["fp64"]["roofline"], "fp32_kahan": out["fp32_kahan"], "fp64": out["fp64"],
            "gpu_launches": 3 * args.steps}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="planar", choices=["planar", "shear", "laplace", "phase", "batch"])
    ap.add_argument("--size", type=int, default=None, help="grid size of the laplace / phase workloads")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
    if args.workload == "batch":
        run_batch(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
