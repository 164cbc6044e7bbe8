"""Benchmark: forward + adjoint X-ray transform of the 2D fan-beam workload
(512x512 pixels, 720 views over 2*pi, 768 flat-detector bins of 1.2, source-origin 1000,
source-detector 1500, a batch of 16 random-ellipse phantoms) on N GPUs of one node.

One step = the per-geometry ray setup + the forward projection of the 16-image batch +
the adjoint of the resulting sinograms, every kernel launched through the C ABI.
Metric: Grays/s = rays x images / (time of one step).  Each rank runs its own batch of 16
independent images (weak scaling, no collective on the data path).

``--impl reference`` times the double-precision CPU oracle on the host cores on a bounded
sample of the same workload (a subset of the views, all 16 images).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "fan2d_512x512_720views_768bins_batch16"
METRIC = "Grays/s forward+adjoint"
UNIT = "Grays/s"


def _config(extra=None):
    c = {"workload": WORKLOAD, "image": [512, 512], "views": 720, "bins": 768, "batch_per_gpu": 16,
         "geometry": "equispaced fan, flat detector, sod 1000, sdd 1500, du 1.2",
         "l2": "flushed between timed steps (256 MiB write)"}
    if extra:
        c.update(extra)
    return c


# ----------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------------------

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for name, val in zip(names, p[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clocks not sampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------------------
# our CUDA path
# ----------------------------------------------------------------------------------------

def _intersections(g, P, x):
    """Sum over rays of the units each ray crosses (counted on the GPU by projecting a
    constant image of ones through a unit-length indicator is not possible; use the sparse
    rows of a sample of rays and scale)."""
    rng = np.random.default_rng(0)
    rays = rng.choice(g.n_rays, size=4096, replace=False)
    rows = P.ray_units(rays)
    return float(np.mean([len(r[0]) for r in rows])) * g.n_rays


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2006_00686_gb300 import inputs, parallel
    from paper_2006_00686_gb300.xray import Projector, XR_ADJ_GATHER, XR_ADJ_SCATTER

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    g = inputs.fan2d_512()
    B = inputs.FAN2D_BATCH
    P = Projector(g)
    tune = {"batch_chunk": args.chunk, "adjoint": XR_ADJ_GATHER if args.adjoint == "gather" else XR_ADJ_SCATTER}
    P.set_tuning(block=args.block, **tune)
    x = inputs.phantom_batch(g, B, 10, seed0=parallel.rank_seeds(rank, B, 200)[0], device=str(dev))
    y = torch.empty(g.sino_shape(B), device=dev)
    z = torch.empty(g.image_shape(B), device=dev)
    flush = torch.empty(64 * 1024 * 1024, device=dev)  # 256 MiB > L2
    stream = torch.cuda.current_stream()

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(times=None):
        e = [ev() for _ in range(4)] if times is not None else None
        if e: e[0].record(stream)
        P.ray_setup(stream)
        if e: e[1].record(stream)
        P.forward(x, out=y, stream=stream)
        if e: e[2].record(stream)
        P.adjoint(y, out=z, stream=stream)
        if e: e[3].record(stream)
        if times is not None:
            times.append(e)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    recs = []
    with ClockSampler(local_rank) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1.0)  # evict L2 between timed steps (outside the step's events)
            step(recs)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    setup_ms = [a.elapsed_time(b) for a, b, c, d in recs]
    fwd_ms = [b.elapsed_time(c) for a, b, c, d in recs]
    adj_ms = [c.elapsed_time(d) for a, b, c, d in recs]
    step_ms = [a.elapsed_time(d) for a, b, c, d in recs]
    ms = float(np.mean(step_ms))
    ms = parallel.max_over_ranks(ms, dev)
    rays_step = g.n_rays * B
    value = rays_step * world / (ms * 1e-3) / 1e9

    # end to end through the C ABI with host buffers: pinned H2D of the images, the step,
    # D2H of the sinograms and the adjoint images, all inside the timed region
    x_h = x.cpu().pin_memory()
    y_h = torch.empty(y.shape, pin_memory=True)
    z_h = torch.empty(z.shape, pin_memory=True)
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        flush.fill_(1.0)
        a, b = ev(), ev()
        a.record(stream)
        x.copy_(x_h, non_blocking=True)
        step()
        y_h.copy_(y, non_blocking=True)
        z_h.copy_(z, non_blocking=True)
        b.record(stream)
        b.synchronize()
        if k >= args.warmup:
            e2e_ms.append(a.elapsed_time(b))
    e2e = float(np.mean(e2e_ms))
    e2e = parallel.max_over_ranks(e2e, dev)

    # roofline of the dominant kernel.  The path is bound by
    # neither HBM (the images and sinograms stay in L2; DRAM traffic is within ~15% of the
    # compulsory bytes) nor tensor cores: every unit costs scalar FP32 work.  "alu":
    # achieved = algorithmic FP32 FLOP per launch / launch time, with per (ray, unit)
    # intersection one subtraction for the length C_up - C_low and one FMA (2 FLOP) per
    # image; peak = 152 SMs x 128 FP32 lanes x 2 FLOP x maximum SM clock.
    peaks, peak_kind = _peaks()
    n_int = _intersections(g, P, x)
    fwd, adj = float(np.mean(fwd_ms)), float(np.mean(adj_ms))
    dom, dom_ms = ("forward", fwd) if fwd >= adj else ("adjoint", adj)
    flop = n_int * (1.0 + 2.0 * B)
    achieved = flop / (dom_ms * 1e-3) / 1e12
    peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    compulsory = 4.0 * (g.n_units + g.n_rays) * B
    # DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the current
    # forward and gather kernels, from one ncu capture of this workload
    traffic = {("adjoint", "gather"): 58.6e6, ("forward", "gather"): 61.9e6,
               ("forward", "scatter"): 61.9e6}.get((dom, args.adjoint))
    roof = {"bound": "alu", "kernel": dom, "achieved": round(achieved, 3), "peak": round(peak, 2),
            "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": traffic,
            "peak_source": f"derived: 152 SMs x 128 FP32 lanes x 2 x {peaks.get('sm_max_mhz', 2070.0):.0f} MHz "
                           f"({peak_kind} max clock)",
            "algorithmic_flop": flop, "intersections_per_image": n_int, "ms": round(dom_ms, 4),
            "hbm": {"compulsory_bytes": compulsory, "achieved_gbs": round(compulsory / (dom_ms * 1e-3) / 1e9, 1),
                    "peak_gbs": peaks["hbm_gbs"]}}

    out = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded random-ellipse phantoms)",
           "config": _config({"adjoint": args.adjoint, "batch_chunk": args.chunk, "block": args.block}),
           "e2e": {"value": round(rays_step * world / (e2e * 1e-3) / 1e9, 4), "unit": UNIT,
                   "h2d_bytes_per_step": int(x.numel() * 4),
                   "d2h_bytes_per_step": int(y.numel() * 4 + z.numel() * 4), "ms_per_step": round(e2e, 4)},
           # per step: detector setup, ray setup, image interleave, forward walk, then either
           # the scatter walk + its de-interleave (two accumulator memsets are not kernels)
           # or the sinogram interleave + gather
           "gpu_launches": args.steps * 6,
           "kernel_ms": {"ray_setup": round(float(np.mean(setup_ms)), 4), "forward": round(fwd, 4),
                         "adjoint": round(adj, 4)},
           "clocks": clk.summary(), "roofline": roof, "wall_s": round(wall, 3)}
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(g, x[:B].cpu().numpy(), budget_s=args.cpu_budget)
    P.close()
    return out


# ----------------------------------------------------------------------------------------
# the oracle on the host cores
# ----------------------------------------------------------------------------------------

def _oracle_step(O, g, f64, views):
    sub = g.subset_views(views)
    y = O.forward(sub, f64)
    O.adjoint(sub, y)
    return sub.n_rays * f64.shape[0]


def cpu_baseline(g, x_np, budget_s=15.0):
    from oracle import oracle as O

    f64 = x_np.reshape(x_np.shape[0], -1).astype(np.float64)
    views = np.arange(0, g.n_views, 180)  # 4 views: probe the rate
    t0 = time.perf_counter()
    rays = _oracle_step(O, g, f64, views)
    dt = time.perf_counter() - t0
    n = int(max(4, min(g.n_views, 4 * budget_s / max(dt, 1e-3))))
    views = np.linspace(0, g.n_views - 1, n).round().astype(np.int64)
    t0 = time.perf_counter()
    rays = _oracle_step(O, g, f64, views)
    dt = time.perf_counter() - t0
    return {"value": round(rays / dt / 1e9, 9), "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
            "sample": f"{len(views)} of {g.n_views} views, all {f64.shape[0]} images, forward+adjoint "
                      f"in float64 ({rays} rays, {dt:.1f} s)"}


def run_reference(args, rank, world):
    from oracle import oracle as O
    from paper_2006_00686_gb300 import inputs

    g = inputs.fan2d_512()
    B = inputs.FAN2D_BATCH
    x = inputs.phantom_batch(g, B, 10, seed0=200).numpy()
    f64 = x.reshape(B, -1).astype(np.float64)
    n_views = max(2, int(args.ref_views))
    times, rays = [], 0
    for k in range(args.warmup + args.steps):
        views = (np.arange(n_views) * (g.n_views // n_views) + k) % g.n_views
        t0 = time.perf_counter()
        rays = _oracle_step(O, g, f64, views)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    ms = 1e3 * float(np.mean(times))
    value = rays / (ms * 1e-3) / 1e9
    sample = f"{n_views} of {g.n_views} views per step, all {B} images, forward+adjoint in float64"
    return {"impl": "reference", "metric": METRIC, "value": round(value, 9), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded random-ellipse phantoms)",
            "config": _config({"sample": sample}),
            "cpu_baseline": {"value": round(value, 9), "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 9), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--adjoint", default="gather", choices=["gather", "scatter"])
    ap.add_argument("--chunk", type=int, default=16)
    ap.add_argument("--block", type=int, default=128)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-views", type=int, default=24)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args, rank, world)), flush=True)
        return

    import torch
    if world > 1:
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    import __graft_entry__
    if rank == 0 or not os.path.exists(os.path.join(ROOT, "paper_2006_00686_gb300", "libxray.so")):
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
    out = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
