#!/usr/bin/env python
"""Benchmark of the RK-3 off-lattice Boltzmann step (node-updates/s).

Default workload: phase separation between cold plates, 4096 x 4096 nodes
(diffuse walls at x = 0, 1 with T_w = 0.7, periodic y), n = 1 + 0.01
band-limited noise, T0 = 1, u = 0, tau = 5e-3, dt = 6.25e-7, sigma = 1e-4
(Sec. 7 set-up).  `value` is the FP64 path.  Beside it, on the same grid and
GPU, each with its own stage time and roofline fraction:
  fp32          FP32 arithmetic with compensated (hi + lo) population storage
  learned_fp64  learned WENO weights (network in FP32, populations FP64)
  learned_fp32  learned WENO weights with the FP32 path
  batch_fp64/32 64 independent runs of uneven size (32^2 .. 1024^2, 13.5 M
                nodes) in one launch per stage, autotuned shape
A "step" is one full RK-3 step of the whole grid: three stages, each the
per-node moments pre-pass and the fused stage kernel (force, WENO-5 fluxes,
collision and RK combination), six launches in all.

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events
on the context's stream, with a 256 MiB buffer written between steps (the
10 GB of populations are far larger than the 129 MB L2 anyway); barrier +
synchronize on both sides; max over ranks.  With torchrun (N > 1) every rank
runs an independent replica (the path has no data exchange to shard): value
is the node-updates of all ranks per second.

Accuracy (rank 0, N = 1, in the oracle leg): every GPU leg is re-run for a few
steps from the initial state and compared on windows at both walls and in the
bulk with the FP64 oracle run on those windows (a window interior farther than
10 nodes per step from a cut edge is exact); the same oracle runs give the CPU
baseline (all host cores) and a single-threaded oracle figure.

Also reported: the roofline of the dominant kernel, end-to-end throughput
through the C ABI with pinned host buffers, the mass and energy sums of the
GPU's FP64 reduction before and after the timed steps, SM clocks sampled
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
# formula: moments 110, force stencils 172, equilibrium factors 104, local
# part of L and RK combination 25 x 30 = 750, WENO-5 faces 40 x 57 = 2280
# (20 moving velocities per axis, one face per node), advection and output
# 155.  The same count is used for the FP32 path (its compensation work is
# overhead, not algorithmic flops).
STAGE_FLOPS_PER_NODE = 110 + 172 + 104 + 750 + 2280 + 155
# One evaluation of the 5-32-32-3 network (FMA = 2): 2 x (5 x 32 + 32 x 32 +
# 32 x 3) = 2560 flops plus 64 tanh, 3 exp and the softmax (not counted).
MLP_FLOPS = 2 * (5 * 32 + 32 * 32 + 32 * 3)
# Population values moved per node and step: stage 1 reads f and writes f1
# (50), stages 2 and 3 read f^n and f_s and write (75 each): 200 per step,
# 8 bytes each in both paths (FP32 stores hi + lo pairs).
VALUES_PER_NODE_STEP = 200
# DRAM bytes (read + write) per stage launch from one ncu capture of exactly
# this kernel build, on the Laplace 2048^2 grid (4.19 M nodes; the 4096^2
# grid is too large to capture), scaled by 4 to the 16.8 M nodes of the
# 4096^2 grid (traffic grows with the node count).  Any other kernel or
# workload reports null.
DRAM_TRAFFIC_PER_LAUNCH = {
    # 2048^2, stages 1, 2, 3: 1.820, 2.669, 2.658 GB (FP64) and 1.818, 2.668, 2.655 GB (FP32); mean x 4
    ("phase", None, "k_fused<double,8,8,4>"): 4 * (1.820 + 2.669 + 2.658) / 3 * 1e9,
    ("phase", None, "k_fused<float,8,8,5>"): 4 * (1.818 + 2.668 + 2.655) / 3 * 1e9,
}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def alu_peaks(device_index: int = 0):
    """FP64 and FP32 peaks (TFLOP/s) from the unit counts of the SM and its
    maximum clock: FP64 2 DFMA per SM per clock, FP32 128 lanes per SM, each
    FMA 2 flops; SM count from the device, clock from MEASURED_PEAKS.json
    (else 2070 MHz, GB300's maximum)."""
    import torch
    sms = torch.cuda.get_device_properties(device_index).multi_processor_count
    mhz = float(load_peaks().get("sm_max_mhz", 2070.0))
    return (sms * 2 * 2 * mhz * 1e6 / 1e12, sms * 128 * 2 * mhz * 1e6 / 1e12, sms, mhz)


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
        desc = (f"phase separation between cold plates {n}^2, diffuse walls x=0,1 Tw=0.7, periodic y, "
                f"n=1+0.01 noise, T0=1, tau=5e-3, dt={p.dt:g}, sigma=1e-4")
    else:
        raise SystemExit(f"unknown workload {name}")
    return p, f, desc


def default_theta():
    """The trained network shipped with the package (None if absent)."""
    from paper_1702_01690_gb300 import learned
    try:
        return learned.load_theta()
    except FileNotFoundError:
        return None


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
            # let the sampler start (its first query) before the timed region
            t0 = time.time()
            while time.time() - t0 < 5.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.05)
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


# ------------------------------------------------------------------ oracle windows
def windows_for(p, steps):
    """Oracle windows of a workload after `steps` steps: (x0, y0, wx, wy,
    wall) with a margin of 10 nodes per step around a 40 x 40 interior (none
    on the wall side)."""
    m = 10 * steps
    w = 40 + 2 * m
    ww = 40 + m
    wins = []
    if p.side_x == 1:
        wins.append((0, p.ny // 7, ww, w, "left"))
        wins.append((p.nx - ww, (3 * p.ny) // 4, ww, w, "right"))
    wins.append((p.nx // 2 - w // 2 + 7, p.ny - w // 2, w, w, None))  # bulk, wrapping in y
    return wins, m


def crop(fields, x0, y0, wx, wy, nx, ny, periodic_x):
    ys = np.arange(y0, y0 + wy) % ny
    xs = np.arange(x0, x0 + wx)
    if periodic_x:
        xs = xs % nx
    return tuple(np.ascontiguousarray(a[np.ix_(ys, xs)]) for a in fields)


def oracle_windows(p, fields, steps, theta=None, threads=None):
    """Run the FP64 oracle on the windows of `p` for `steps` steps; returns
    the per-window oracle moments, the windows, the interior margin, the
    node-updates done and the seconds taken."""
    import oracle
    from paper_1702_01690_gb300 import inputs
    oracle.set_threads(threads or (os.cpu_count() or 1))
    wins, m = windows_for(p, steps)
    out, work = [], 0
    t0 = time.perf_counter()
    for (x0, y0, wx, wy, wall) in wins:
        wp = inputs.RunParams(**{**p.as_dict(), "nx": wx, "ny": wy})
        if wall is None:
            wp.side_x = 0
        o = oracle.Oracle(wp.nx, wp.ny, wp.ds, wp.dt, wp.tau, wp.a, wp.b, wp.sigma, wp.Tw, wp.uw, wp.side_x,
                          wp.side_y)
        if theta is not None:
            o.set_mlp(np.asarray(theta, dtype=np.float64))
        o.init_fields(*crop(fields, x0, y0, wx, wy, p.nx, p.ny, p.side_x == 0))
        o.step(steps)
        out.append(o.moments())
        o.close()
        work += wx * wy * steps
    return out, wins, m, work, time.perf_counter() - t0, oracle.max_threads()


def window_errors(m_gpu, p, ref, wins, margin):
    """Largest error of the GPU moments against the oracle windows over the
    window interiors, relative to each field's largest oracle value there
    (u: the largest |u_x|, |u_y|)."""
    worst = {"n": 0.0, "u": 0.0, "T": 0.0}
    for (x0, y0, wx, wy, wall), mo in zip(wins, ref):
        ys = np.arange(y0, y0 + wy) % p.ny
        xs = np.arange(x0, x0 + wx) % p.nx
        iy = slice(margin, wy - margin)
        ix = slice(0, wx - margin) if wall == "left" else (slice(margin, wx) if wall == "right"
                                                           else slice(margin, wx - margin))
        g = [a[np.ix_(ys, xs)][iy, ix] for a in m_gpu]
        r = [a[iy, ix] for a in mo]
        us = max(np.max(np.abs(r[1])), np.max(np.abs(r[2])), 1e-300)
        worst["n"] = max(worst["n"], float(np.max(np.abs(g[0] - r[0])) / np.max(np.abs(r[0]))))
        worst["u"] = max(worst["u"], float(max(np.max(np.abs(g[1] - r[1])), np.max(np.abs(g[2] - r[2]))) / us))
        worst["T"] = max(worst["T"], float(np.max(np.abs(g[3] - r[3])) / np.max(np.abs(r[3]))))
    return worst


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    p, fields, desc = workload(args.workload, args.size)
    steps = args.steps
    # untimed warm-up, then K timed steps of the oracle on the workload's
    # windows (all host cores); a sample of the same per-node work
    import oracle
    from paper_1702_01690_gb300 import inputs
    oracle.set_threads(os.cpu_count() or 1)
    wins, _ = windows_for(p, 1)
    x0, y0, wx, wy, wall = wins[0]
    wx, wy = min(p.nx, 256), min(p.ny, 256)
    wp = inputs.RunParams(**{**p.as_dict(), "nx": wx, "ny": wy})
    o = oracle.Oracle(wp.nx, wp.ny, wp.ds, wp.dt, wp.tau, wp.a, wp.b, wp.sigma, wp.Tw, wp.uw, wp.side_x, wp.side_y)
    o.init_fields(*crop(fields, 0, 0, wx, wy, p.nx, p.ny, p.side_x == 0))
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(steps)
    el = time.perf_counter() - t0
    v = wx * wy * steps / el
    what = f"{wx}x{wy} window (walls kept) of the {p.nx}x{p.ny} grid"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc, "sample": what},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": f"{steps} RK-3 steps of the {what}"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU legs
def time_steps(ctx, steps, warmup, flush, stream):
    """K graph-replayed steps, each bracketed by CUDA events on the context's
    stream; the flush buffer is written between steps (outside the events)."""
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


def timed_leg(olb, p, dev_fields, prec, steps, warmup, flush, stream, world, peak, weno=0, theta=None,
              clocks=None, mlp_acts=None):
    """One timed leg: value, ms per step, stage time and roofline of the stage
    kernel.  The step is exactly three launches of the stage kernel, so the
    average launch takes a third of the timed step."""
    import torch
    N = p.nx * p.ny
    ctx = olb.create(p, prec, stream, weno_mode=weno)
    if theta is not None:
        ctx.set_weno_mlp(theta)
    ctx.init_fields(*dev_fields)
    torch.cuda.synchronize()
    rank_barrier()
    if clocks is not None:
        with clocks:
            total, per = time_steps(ctx, steps, warmup, flush, stream)
    else:
        total, per = time_steps(ctx, steps, warmup, flush, stream)
    rank_barrier()
    total = max_over_ranks(total)
    ms_step = total / steps
    stage_ms = ms_step / 3.0
    flops = STAGE_FLOPS_PER_NODE * N
    if mlp_acts is not None:
        flops += mlp_acts * MLP_FLOPS
    ach = flops / (stage_ms * 1e-3) / 1e12
    tile = ctx.get_tile()
    kind = "double" if prec == olb.FP64 else "float"
    kname = f"k_fused<{kind},{tile[0]},{tile[1]},{tile[2]}{',learned' if weno else ''}>"
    prof = ctx.profile(3)
    leg = {"value": job_value(world, N, steps, total), "ms_per_step": ms_step,
           "roofline": {"kernel": kname, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                        "frac": ach / peak, "algorithmic_flops_per_launch": flops, "stage_ms": stage_ms,
                        "stage_ms_single_launches": prof["stage_ms"]}}
    return leg, ctx


def run_ours(args, rank, world):
    import torch
    from paper_1702_01690_gb300 import olb

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    p, fields, desc = workload(args.workload, args.size)
    N = p.nx * p.ny
    peak64, peak32, sms, mhz = alu_peaks(local)
    olb.use_torch_allocator(True)
    dev_fields = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in fields]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    legs_run = 0

    # ---- FP64 (value)
    clk = ClockSampler(local)
    fp64, ctx = timed_leg(olb, p, dev_fields, olb.FP64, args.steps, args.warmup, flush, stream, world, peak64,
                          clocks=clk)
    legs_run += 1
    value, ms_step = fp64["value"], fp64["ms_per_step"]
    roof = dict(fp64["roofline"])
    kname = roof["kernel"]
    roof["traffic"] = DRAM_TRAFFIC_PER_LAUNCH.get((args.workload, args.size, kname))
    roof["peak_source"] = (f"FP64 units x max SM clock: 2 DFMA/SM/clk x {sms} SMs x {mhz:.0f} MHz x 2 flop "
                           f"(no FP64 entry in MEASURED_PEAKS.json)")
    # mass and energy from the GPU's FP64 reduction after the timed steps
    # (the context is then at step warmup + steps + 3 profiled steps)
    tot_after = ctx.totals()
    ctx.init_fields(*dev_fields)
    tot0 = ctx.totals()
    ctx.close()
    del ctx
    torch.cuda.empty_cache()

    # ---- FP32 compensated
    fp32, c32 = timed_leg(olb, p, dev_fields, olb.FP32_KAHAN, args.steps, args.warmup, flush, stream, world, peak32)
    fp32["speedup_vs_fp64"] = fp32["value"] / value
    fp32["roofline"]["peak_source"] = f"FP32 lanes x max SM clock: 128/SM x {sms} SMs x {mhz:.0f} MHz x 2 flop"
    fp32["roofline"]["traffic"] = DRAM_TRAFFIC_PER_LAUNCH.get((args.workload, args.size, fp32["roofline"]["kernel"]))
    c32.close()
    del c32
    torch.cuda.empty_cache()

    # ---- learned weights (FP64 and FP32 populations)
    theta = default_theta()
    learned = {}
    if theta is not None and not args.no_learned:
        lsteps = max(1, min(args.steps, args.learned_steps))
        for name, prec, pk in (("learned_fp64", olb.FP64, peak64), ("learned_fp32", olb.FP32_KAHAN, peak32)):
            leg, c = timed_leg(olb, p, dev_fields, prec, lsteps, args.warmup, flush, stream, world, pk, weno=1,
                               theta=theta)
            leg["steps"] = lsteps
            leg["speedup_vs_fp64_js"] = leg["value"] / value
            leg["roofline"]["note"] = ("flops counted as for the Jiang-Shu stage; the network evaluations "
                                       "are extra work on the FP32 pipe")
            c.close()
            del c
            torch.cuda.empty_cache()
            learned[name] = leg

    # ---- batch sweep
    batch = {}
    if not args.no_batch:
        batch = run_batch_legs(args, world, stream, peak64, peak32)

    # ---- end to end through the C ABI with pinned host buffers
    ctx = olb.create(p, olb.FP64, stream)
    host_in = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in fields]
    host_out = [torch.empty((p.ny, p.nx), dtype=torch.float64).pin_memory() for _ in range(4)]
    e2e_iters = max(3, min(args.steps, 10))
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
    del ctx
    torch.cuda.empty_cache()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "nodes": N, "grid": [p.nx, p.ny],
                       "l2": "inputs (10 GB of populations) larger than L2; 256 MiB buffer also written "
                             "between timed steps",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roof, "fp32": fp32, **learned, **batch, "e2e": e2e,
            "totals_fp64_gpu": {"mass_initial": tot0[0], "energy_initial": tot0[3],
                                "mass_after_timed_steps": tot_after[0], "energy_after_timed_steps": tot_after[3],
                                "mass_rel_change": float((tot_after[0] - tot0[0]) / tot0[0])},
            "gpu_launches": 6 * args.steps, "clocks": clk.summary()}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line.update(oracle_leg(args, p, fields, dev_fields, theta, stream))
    if rank == 0:
        print(json.dumps(line), flush=True)


def oracle_leg(args, p, fields, dev_fields, theta, stream):
    """Accuracy of every GPU leg against the FP64 oracle on windows, and the
    oracle's own speed on the host cores (the CPU baseline)."""
    import torch
    from paper_1702_01690_gb300 import olb
    steps = args.check_steps
    ref, wins, margin, work, secs, cores = oracle_windows(p, fields, steps)
    out = {"cpu_baseline": {"value": work / secs, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{steps} RK-3 steps of {len(wins)} windows of the {p.nx}x{p.ny} workload "
                                      f"({work} node-updates, {secs:.1f} s), the windows the accuracy check uses"}}
    # single-threaded oracle on the first window for a few steps
    w0 = [wins[0]]
    x0, y0, wx, wy, wall = w0[0]
    import oracle
    from paper_1702_01690_gb300 import inputs
    oracle.set_threads(1)
    wp = inputs.RunParams(**{**p.as_dict(), "nx": wx, "ny": wy})
    if wall is None:
        wp.side_x = 0
    o = oracle.Oracle(wp.nx, wp.ny, wp.ds, wp.dt, wp.tau, wp.a, wp.b, wp.sigma, wp.Tw, wp.uw, wp.side_x, wp.side_y)
    o.init_fields(*crop(fields, x0, y0, wx, wy, p.nx, p.ny, p.side_x == 0))
    s1 = 2
    t0 = time.perf_counter()
    o.step(s1)
    el = time.perf_counter() - t0
    o.close()
    out["cpu_baseline_single_thread"] = {"value": wx * wy * s1 / el, "unit": UNIT, "cores": 1, "kind": "oracle",
                                         "sample": f"{s1} RK-3 steps of the {wx}x{wy} window at x0={x0}"}
    oracle.set_threads(os.cpu_count() or 1)
    acc = {"steps": steps, "windows": [list(w[:4]) + [w[4] or "bulk"] for w in wins],
           "interior_margin_nodes": margin}
    legs = [("fp64", olb.FP64, 0), ("fp32", olb.FP32_KAHAN, 0)]
    for name, prec, weno in legs:
        c = olb.create(p, prec, stream)
        c.init_fields(*dev_fields)
        assert c.step(steps) == 0
        acc[name] = window_errors(c.moments(), p, ref, wins, margin)
        c.close()
        del c
        torch.cuda.empty_cache()
    if theta is not None and not args.no_learned:
        lsteps = min(steps, 5)
        lref, lwins, lmargin, _, _, _ = oracle_windows(p, fields, lsteps, theta=theta)
        acc["learned_steps"] = lsteps
        for name, prec in (("learned_fp64", olb.FP64), ("learned_fp32", olb.FP32_KAHAN)):
            c = olb.create(p, prec, stream, weno_mode=olb.WENO_LEARNED)
            c.set_weno_mlp(theta)
            c.init_fields(*dev_fields)
            assert c.step(lsteps) == 0
            acc[name] = window_errors(c.moments(), p, lref, lwins, lmargin)
            c.close()
            del c
            torch.cuda.empty_cache()
    out["max_rel_err_vs_fp64_oracle_windows"] = acc
    return out


def run_batch_legs(args, world, stream, peak64, peak32):
    """64 independent runs of uneven sizes (32^2 .. 1024^2 shear and
    longitudinal waves, Laplace drops, planar wall runs; 13.5 M nodes) in one
    launch per stage (one CTA per tile of every run), replayed from CUDA
    graphs, shape autotuned.  The working set (3 x 25 x 13.5 M values) is far
    larger than L2."""
    import torch
    from paper_1702_01690_gb300 import inputs, olb
    runs = inputs.batch_sweep()
    nodes = sum(p.nx * p.ny for p, _ in runs)
    out = {}
    for name, prec, peak in (("batch_fp64", olb.FP64, peak64), ("batch_fp32", olb.FP32_KAHAN, peak32)):
        b = olb.Batch([p for p, _ in runs], prec, stream)
        for r, (p, fl) in enumerate(runs):
            b.init_fields(r, *fl)
        shape = b.autotune(2)
        b.step(args.warmup)
        torch.cuda.synchronize()
        rank_barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step_async(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        rank_barrier()
        ms = max_over_ranks(e0.elapsed_time(e1))
        rc, _ = b.status()
        if rc != 0:
            raise RuntimeError(f"batch diverged ({name})")
        stage_ms = ms / args.steps / 3.0
        ach = STAGE_FLOPS_PER_NODE * nodes / (stage_ms * 1e-3) / 1e12
        out[name] = {"value": job_value(world, nodes, args.steps, ms), "ms_per_step": ms / args.steps,
                     "runs": len(runs), "nodes": nodes, "shape": list(shape),
                     "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                                  "frac": ach / peak, "stage_ms": stage_ms}}
        b.close()
        del b
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="phase", choices=["planar", "shear", "laplace", "phase"])
    ap.add_argument("--size", type=int, default=None, help="grid size of the laplace / phase workloads")
    ap.add_argument("--check-steps", type=int, default=20, help="steps of the accuracy check against the oracle")
    ap.add_argument("--learned-steps", type=int, default=10, help="timed steps of the learned legs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
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
    run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
