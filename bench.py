"""Benchmark: forward + adjoint X-ray transform on N GPUs of one node.

Headline line: the 2D fan-beam workload (512x512 pixels, 720 views over 2*pi, 768
flat-detector bins of 1.2, source-origin 1000, source-detector 1500, a batch of 16
random-ellipse phantoms).  With no --workload, the same run also measures every other
scan configuration under ``extra.per_config``: the 2D parallel beam 64^2 (CUDA-graph
replay), the single-tilt-axis parallel beam 256^3 (with autograd and SIRT), the circular
cone 512^3, the helical cone 512^2 x 256, and 64 uneven fans as one persistent plan
against one launch set per problem.

One step = the per-geometry ray setup + the forward projection + the adjoint of the
resulting sinograms, every kernel launched through the C ABI.
Metric: Grays/s = rays x images / (time of one step).  Each rank runs its own batch of
independent images (weak scaling, no collective on the data path).

``--impl reference`` times the double-precision CPU oracle on the host cores on a bounded
sample of the same workload (a subset of the views, all images).
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
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []  # csv lines, each led by the sample's own timestamp
        self.window = None  # (start, end) wall-clock times of the timed region

    def mark(self, start: float, end: float):
        self.window = (start, end)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    @staticmethod
    def _when(ln: str) -> float:
        """Wall-clock time of a sample (nvidia-smi's 'YYYY/MM/DD HH:MM:SS.mmm'), -inf if unreadable."""
        import datetime
        try:
            return datetime.datetime.strptime(ln.split(",")[0].strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return float("-inf")

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        """Clocks of the samples taken during the timed region; a region shorter than the
        sampling interval takes the samples of the warm-up steps before it and of the timed
        steps (the same load), and says so."""
        lines = list(self.lines)
        window = "timed steps"
        if self.window is not None:
            t0, t1 = self.window
            inside = [ln for ln in lines if t0 - 0.01 <= self._when(ln) <= t1 + 0.01]
            if inside:
                lines = inside
            else:
                lines = [ln for ln in lines if self._when(ln) <= t1 + 0.01]
                window = "warm-up and timed steps (timed region shorter than the sampling interval)"
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 10:
                continue
            try:
                sm.append(float(p[2]))
                mx.append(float(p[3]))
            except ValueError:
                continue
            for name, val in zip(names, p[6:10]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clocks not sampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "window": window}


# ----------------------------------------------------------------------------------------
# our CUDA path
# ----------------------------------------------------------------------------------------

def _intersections(g, P, sample=4096):
    """Sum over rays of the units each ray crosses, estimated from the sparse rows (the
    walk's own unit lists) of a seeded sample of rays."""
    rng = np.random.default_rng(0)
    rays = rng.choice(g.n_rays, size=min(sample, g.n_rays), replace=False)
    rows = P.ray_units(rays)
    return float(np.mean([len(r[0]) for r in rows])) * g.n_rays


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


WORKLOADS = {
    # name: (geometry builder in inputs, images per rank, shapes per phantom, phantom seed base,
    #        description)
    "fan2d_512x16": ("fan2d_512", 16, 10, 200, None),
    "par2d_64": ("par2d_64", 1, 10, 1, "2D parallel 64x64, 90 views, 95 bins"),
    "par3d_256_tilt": ("par3d_256_tilt", 1, 30, 3,
                       "3D parallel 256^3, one tilt axis, 181 tilts -60..60 deg, 256x256 detector"),
    "cone_512": ("cone_512", 1, 30, 4, "circular cone 512^3 (0.8,0.8,1.0) centre (10,-5,3), 720 views, "
                 "1024x768 flat detector, sod 1000, sdd 1500"),
    "helix_512x256": ("helix_512x256", 1, 30, 5, "helical cone 512x512x256, 4 turns x 720 views, pitch 1, "
                      "736x64 flat detector, sod 600, sdd 1100"),
    "fans_uneven_64": (None, 64, 10, 500, "64 uneven 2D fans (sides 128..1024, seed 5), one persistent "
                       "launch each for forward and adjoint"),
    "fan2d_512x16_atten": ("fan2d_512", 16, 10, 200, "attenuated transform (exponential attenuation of a "
                           "0.02 + 0.05 x ellipse-phantom map) on the 512^2 x 16 fan scan"),
}


def _events(n):
    import torch
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def _timed_loop(step, args, flush, world, local_rank):
    """W untimed steps, then K timed steps (L2 flushed before each, outside its events);
    returns per-step lists of event pairs per phase, the clock summary and the wall time."""
    import torch
    recs = []
    with ClockSampler(local_rank) as clk:  # sampling from the warm-up on
        for _ in range(args.warmup):
            step(None)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0, w0 = time.perf_counter(), time.time()
        for _ in range(args.steps):
            flush.fill_(1.0)
            step(recs)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        clk.mark(w0, time.time())
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    return recs, clk.summary(), wall


def _e2e(sets, args, flush):
    """Mean ms per step of the end-to-end loop: every step copies its inputs host -> device
    (pinned), runs, and copies its results device -> host.  Host-to-device and
    device-to-host copies run on two more streams with two buffer sets, so the copies of
    steps k + 1 and k - 1 overlap step k's kernels; each step waits for its own inputs, and a
    buffer set is refilled only after its previous results were copied out.  The whole
    K-step loop is timed, from the first copy in to the last copy out.
    sets: two dicts with step() (launches on the current stream), host_in, dev_in, dev_out,
    host_out."""
    import torch
    comp = torch.cuda.current_stream()
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    n = len(sets)
    h2d = [torch.cuda.Event() for _ in range(n)]
    done = [torch.cuda.Event() for _ in range(n)]
    d2h = [torch.cuda.Event() for _ in range(n)]
    for e in done + d2h:
        e.record(comp)

    def copy_in(k):
        i = k % n
        s_in.wait_event(done[i])  # the set's previous step no longer reads its inputs
        with torch.cuda.stream(s_in):
            for d, h in zip(sets[i]["dev_in"], sets[i]["host_in"]):
                d.copy_(h, non_blocking=True)
        h2d[i].record(s_in)

    def run(K, start=None):
        if start is not None:
            start.record(s_in)
        copy_in(0)
        for k in range(K):
            i = k % n
            if k + 1 < K:
                copy_in(k + 1)  # prefetch the next step's inputs
            comp.wait_event(h2d[i])
            comp.wait_event(d2h[i])  # the set's previous results are out
            flush.fill_(1.0)  # L2 flushed before every step, inside the timed loop
            sets[i]["step"]()
            done[i].record(comp)
            s_out.wait_event(done[i])
            with torch.cuda.stream(s_out):
                for h, d in zip(sets[i]["host_out"], sets[i]["dev_out"]):
                    h.copy_(d, non_blocking=True)
            d2h[i].record(s_out)

    run(args.warmup)
    torch.cuda.synchronize()
    a, b = _events(2)
    run(args.steps, start=a)
    b.record(s_out)
    b.synchronize()
    return a.elapsed_time(b) / args.steps


_L2_PEAK = None


def _l2_peak():
    """Measured L2 read bandwidth (GB/s): a 64 MiB buffer read 20 times per launch with
    128-bit L2-only loads (xr_read_probe), best of 5 launches; measured once per process."""
    global _L2_PEAK
    if _L2_PEAK is None:
        from paper_2006_00686_gb300.xray import read_bandwidth
        _L2_PEAK = read_bandwidth(64 << 20, 20, 5)
    return _L2_PEAK


def _roofline(n_int, units_bytes, B, dom, dom_ms, peaks, peak_kind, traffic, traffic_note=None):
    """Roofline of the dominant kernel: the path is a gather (forward) or a
    scatter (adjoint) of 4 B per (ray, unit, image) along the rays, served from L1/L2, so
    the bound is memory, not tensor cores.  achieved = 4 B x intersections x images per
    launch / launch time; peak = the L2 read bandwidth measured in the same run.  The
    compulsory HBM bytes (images + sinograms) and the FP32 issue fraction are reported
    beside it."""
    gather = 4.0 * n_int * B
    gbs = gather / (dom_ms * 1e-3) / 1e9
    l2_peak = _l2_peak()
    flop = n_int * (1.0 + 2.0 * B)  # one subtraction per length, one FMA per image
    mhz = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * mhz * 1e6 / 1e12
    from paper_2006_00686_gb300.xray import fma_throughput
    global _FMA
    if "_FMA" not in globals():
        _FMA = fma_throughput()
    tflops = flop / (dom_ms * 1e-3) / 1e12
    out = {"bound": "l2", "kernel": dom, "achieved": round(gbs, 1), "peak": round(l2_peak, 1), "unit": "GB/s",
           "frac": round(gbs / l2_peak, 4), "traffic": traffic,
           "peak_source": "measured in this run: xr_read_probe, a 64 MiB buffer read 20x per launch with "
                          "L2-only 128-bit loads (MEASURED_PEAKS.json has no L2 figure)",
           "algorithmic_bytes": gather, "intersections_per_image": n_int, "images": B, "ms": round(dom_ms, 4),
           "hbm": {"compulsory_bytes": units_bytes,
                   "achieved_gbs": round(units_bytes / (dom_ms * 1e-3) / 1e9, 1),
                   "peak_gbs": peaks["hbm_gbs"], "peak_source": f"MEASURED_PEAKS.json ({peak_kind})",
                   "frac": round(units_bytes / (dom_ms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4)},
           "alu": {"achieved_tflops": round(tflops, 3), "peak_tflops": round(fp32_peak, 2),
                   "frac": round(tflops / fp32_peak, 4), "fp32_fma_measured_tflops": round(_FMA, 2),
                   "flop": flop,
                   "peak_source": f"derived: 152 SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz"}}
    if traffic_note:
        out["traffic_source"] = traffic_note
    return out


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the dominant
# kernel, from the ncu captures summarised under profiles/: (workload, phase, method) ->
# (bytes, note).  Only kernels unchanged since their capture are listed.
TRAFFIC = {
    ("fan2d_512x16", "adjoint", "gather"): (69.5e6, "profiles/gather_stage_fan2d_512x16.md (one launch of the staged "
                                                    "gather, full size; the records pass before it is not included)"),
    ("fan2d_512x16", "forward", "gather"): (62.4e6, "profiles/fwd_plane_fan2d_512x16.md (one launch, full size)"),
    ("par3d_256_tilt", "adjoint", "gather"): (118.4e6, "profiles/column_batch_par3d_256_tilt.md (one launch of the "
                                                        "staged gather, full size; the records pass is not included)"),
    ("cone_512", "adjoint", "scatter"): (79.91e9, "profiles/trace3d_cone_512_dram.md (one launch, full size)"),
    ("cone_512", "forward", "scatter"): (13.49e9, "profiles/trace3d_cone_512_dram.md (one launch of the two-part "
                                                 "forward, full size)"),
    ("helix_512x256", "adjoint", "scatter"): (3.378e9, "profiles/trace3d_helix_512x256_dram.md (one launch, full size)"),
}

GRAPHED = ("par2d_64",)  # launch-bound steps replayed from a CUDA graph
FUSED = ("par2d_64",)  # steps whose forward and adjoint run as one launch (xr_project_backproject)


def run_ours(args, rank, world, local_rank, workload=None, cpu_budget=None):
    import torch

    from paper_2006_00686_gb300 import inputs, parallel
    from paper_2006_00686_gb300.xray import Projector, XR_ADJ_GATHER, XR_ADJ_SCATTER

    workload = workload or args.workload
    cpu_budget = args.cpu_budget if cpu_budget is None else cpu_budget
    if workload == "fans_uneven_64":
        return run_uneven(args, rank, world, local_rank, cpu_budget)
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    builder, B, n_shapes, seed, desc = WORKLOADS[workload]
    g = getattr(inputs, builder)()
    P = Projector(g)
    tune = {}
    if args.adjoint:
        tune["adjoint"] = XR_ADJ_GATHER if args.adjoint == "gather" else XR_ADJ_SCATTER
    if args.chunk:
        tune["batch_chunk"] = args.chunk
    if args.order != "auto":
        from paper_2006_00686_gb300.xray import XR_ORDER_COLUMN, XR_ORDER_ROW, XR_ORDER_ROWBLOCK, XR_ORDER_VIEW
        tune["order"] = {"view": XR_ORDER_VIEW, "row": XR_ORDER_ROW, "column": XR_ORDER_COLUMN,
                         "rowblock": XR_ORDER_ROWBLOCK}[args.order]
    P.set_tuning(block=args.block, **tune)
    seed0 = parallel.rank_seeds(rank, B, seed)[0]
    if B > 1:
        x = inputs.phantom_batch(g, B, n_shapes, seed0=seed0, device=str(dev))
    else:
        x = inputs.phantom(g, n_shapes, seed0, device=str(dev)).float().contiguous()
    bshape = B if B > 1 else None
    y = torch.empty(g.sino_shape(bshape), device=dev)
    z = torch.empty(g.image_shape(bshape), device=dev)
    flush = torch.empty(64 * 1024 * 1024, device=dev)  # 256 MiB > L2
    stream = torch.cuda.current_stream()

    atten = workload.endswith("_atten")
    mu = (0.02 + 0.05 * inputs.phantom(g, 4, 900, device=str(dev))).float().contiguous() if atten else None

    def make_step(xb, yb, zb, fused=False):
        def step(recs=None):
            stream = torch.cuda.current_stream()  # the capture stream inside graphed()
            e = _events(4) if recs is not None else None
            if e: e[0].record(stream)
            P.ray_setup(stream)
            if e: e[1].record(stream)
            if fused:
                # forward and adjoint of its result in one launch; the adjoint phase is empty
                P.forward_adjoint(xb, sino_out=yb, img_out=zb, stream=stream)
                if e: e[2].record(stream)
            elif atten:
                P.forward_attenuated(xb, mu, out=yb, stream=stream)
            else:
                P.forward(xb, out=yb, stream=stream)
            if not fused:
                if e: e[2].record(stream)
                if atten:
                    P.adjoint_attenuated(yb, mu, out=zb, stream=stream)
                else:
                    P.adjoint(yb, out=zb, stream=stream)
            if e: e[3].record(stream)
            if recs is not None:
                recs.append(e)
        return step

    def graphed(step_fn):
        """The step captured once in a CUDA graph (after an eager call that reserves the
        workspace); each call replays it on the current stream."""
        step_fn(None)
        torch.cuda.synchronize()
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr):
            step_fn(None)
        torch.cuda.synchronize()

        def replay(recs=None):
            e = _events(2) if recs is not None else None
            if e: e[0].record()
            gr.replay()
            if e: e[1].record()
            if recs is not None:
                recs.append(e)
        return replay

    use_fused = workload in FUSED and not atten
    step = make_step(x, y, z, fused=use_fused)
    use_graph = workload in GRAPHED

    # per-phase kernel times from eager steps; the step time from the graph where used
    recs, clocks, wall = _timed_loop(step, args, flush, world, local_rank)
    setup_ms = [a.elapsed_time(b) for a, b, c, d in recs]
    fwd_ms = [b.elapsed_time(c) for a, b, c, d in recs]
    adj_ms = [c.elapsed_time(d) for a, b, c, d in recs]
    step_ms = [a.elapsed_time(d) for a, b, c, d in recs]
    eager_ms = float(np.mean(step_ms))
    if use_graph:
        grecs, clocks, wall = _timed_loop(graphed(step), args, flush, world, local_rank)
        step_ms = [a.elapsed_time(b) for a, b in grecs]
    ms = parallel.max_over_ranks(float(np.mean(step_ms)), dev)
    rays_step = g.n_rays * B
    value = rays_step * world / (ms * 1e-3) / 1e9
    separate = None
    if use_fused:
        # the same step with the forward and the adjoint as separate calls
        sep = make_step(x, y, z)
        srecs, _, _ = _timed_loop(graphed(sep) if use_graph else sep, args, flush, world, local_rank)
        sms = parallel.max_over_ranks(float(np.mean([r[0].elapsed_time(r[-1]) for r in srecs])), dev)
        separate = {"value": round(rays_step * world / (sms * 1e-3) / 1e9, 4), "ms_per_step": round(sms, 4),
                    "form": "ray setup, xr_project, xr_backproject" + (" (graph replay)" if use_graph else "")}

    # end to end through the C ABI with host buffers: pinned H2D of the images, the step,
    # D2H of the sinograms and the adjoint images, all inside the timed region
    x_h = x.cpu().pin_memory()
    sets = []
    for xb, yb, zb in ((x, y, z), (x.clone(), torch.empty_like(y), torch.empty_like(z))):
        st = make_step(xb, yb, zb, fused=use_fused)
        sets.append({"step": graphed(st) if use_graph else st, "host_in": [x_h], "dev_in": [xb],
                     "dev_out": [yb, zb],
                     "host_out": [torch.empty(yb.shape, pin_memory=True), torch.empty(zb.shape, pin_memory=True)]})
    e2e = parallel.max_over_ranks(_e2e(sets, args, flush), dev)
    plain = None
    if B > 1 and not atten:
        # the plain form: the same step with one launch set per image (single-image path)
        def plain_step(recs):
            stream = torch.cuda.current_stream()
            e = _events(4) if recs is not None else None
            if e: e[0].record(stream)
            P.ray_setup(stream)
            if e: e[1].record(stream)
            for b in range(B):
                P.forward(x[b], out=y[b], stream=stream)
            if e: e[2].record(stream)
            for b in range(B):
                P.adjoint(y[b], out=z[b], stream=stream)
            if e: e[3].record(stream)
            if recs is not None:
                recs.append(e)

        prec, _, _ = _timed_loop(plain_step, args, flush, world, local_rank)
        pms = parallel.max_over_ranks(float(np.mean([a.elapsed_time(d) for a, b, c, d in prec])), dev)
        plain = {"value": round(rays_step * world / (pms * 1e-3) / 1e9, 4), "ms_per_step": round(pms, 4),
                 "kernel_ms": {"ray_setup": round(float(np.mean([a.elapsed_time(b) for a, b, c, d in prec])), 4),
                               "forward": round(float(np.mean([b.elapsed_time(c) for a, b, c, d in prec])), 4),
                               "adjoint": round(float(np.mean([c.elapsed_time(d) for a, b, c, d in prec])), 4)},
                 "form": f"{B} single-image forward and adjoint launch sets per step"}

    peaks, peak_kind = _peaks()
    fwd, adj = float(np.mean(fwd_ms)), float(np.mean(adj_ms))
    dom, dom_ms = ("forward", fwd) if fwd >= adj else ("adjoint", adj)
    # the method the library's automatic choice takes: the gather on the 2D quad-plane path
    # (batches of 4 or more) and for single-tilt-axis scans run as 2D column problems, the
    # scatter elsewhere
    adj_mode = P.tuning()["adjoint"]
    if adj_mode == 0:
        method = "gather" if ((not g.is3d and B >= 4) or P.column_batch) else "scatter"
    else:
        method = "gather" if adj_mode == XR_ADJ_GATHER else "scatter"
    traffic, note = TRAFFIC.get((workload, dom, method), (None, None))
    n_int = _intersections(g, P)
    if use_fused:
        # one launch walks every ray twice: the forward's and the adjoint's bytes
        dom, dom_ms, method = "forward+adjoint (one launch)", fwd, "scatter"
        roof = _roofline(2 * n_int, 4.0 * (g.n_units + g.n_rays) * B, B, dom, dom_ms, peaks, peak_kind, None, None)
    else:
        roof = _roofline(n_int, 4.0 * (g.n_units + g.n_rays) * B, B, dom, dom_ms, peaks, peak_kind, traffic, note)

    extra = {}
    if atten:
        config = _config({"workload": workload, "geometry": desc, "adjoint": "scatter (attenuated)"})
        # detector setup, ray setup, gather constants; forward: image planes, the map's two
        # padded copies, the walk; adjoint: the map's copies, the walk, the de-interleave
        launches = 9
    elif workload == "fan2d_512x16":
        config = _config({"adjoint": method, "batch_chunk": P.tuning()["batch_chunk"], "block": args.block})
        # per step: detector setup, ray setup, the gather's per-ray constants, image
        # interleave, forward walk, then either the scatter walk + its de-interleave (two
        # accumulator memsets are not kernels) or the gather records + the staged gather
        launches = 7
    else:
        config = {"workload": workload, "geometry": desc, "image": list(g.image_shape()),
                  "views": g.n_views, "detector": [g.n_rows, g.n_cols], "batch_per_gpu": B,
                  "adjoint": method + (" (2D column problems)" if P.column_batch else ""),
                  "ray_order": {0: "auto", 1: "view", 2: "row", 3: "column", 4: "rowblock"}[P.tuning()["order"]],
                  "l2": "flushed between timed steps (256 MiB write)"}
        if use_graph:
            config["cuda_graph"] = "each step replayed from one captured graph"
        launches = _launch_count(P, g, B, fused=use_fused)
        if use_fused:
            config["adjoint"] = "scatter, in the forward's launch (xr_project_backproject)"
        if workload == "par3d_256_tilt":
            extra = _autograd_and_sirt(P, x, y, args)
    out = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded random-ellipse phantoms)",
           "config": config,
           "e2e": {"value": round(rays_step * world / (e2e * 1e-3) / 1e9, 4), "unit": UNIT,
                   "h2d_bytes_per_step": int(x.numel() * 4),
                   "d2h_bytes_per_step": int(y.numel() * 4 + z.numel() * 4), "ms_per_step": round(e2e, 4),
                   "method": "pinned copies in and out on two more streams, two buffer sets, L2 flushed "
                             "per step, whole loop timed"},
           "gpu_launches": args.steps * launches,
           "kernel_ms": ({"ray_setup": round(float(np.mean(setup_ms)), 4), "forward_adjoint": round(fwd, 4)}
                         if use_fused else
                         {"ray_setup": round(float(np.mean(setup_ms)), 4), "forward": round(fwd, 4),
                          "adjoint": round(adj, 4)}),
           "clocks": clocks, "roofline": roof, "wall_s": round(wall, 3)}
    if use_graph:
        out["eager_ms_per_step"] = round(eager_ms, 4)
    if separate is not None:
        out["separate"] = separate
        out["fused_over_separate"] = round(separate["ms_per_step"] / ms, 3)
    if plain is not None:
        out["plain"] = plain
        out["batched_over_plain"] = round(plain["ms_per_step"] / ms, 3)
    if "autograd_fwd_bwd_ms" in extra:
        # the differentiable form against the plain forward + adjoint through the C ABI
        extra["plain_fwd_adj_ms"] = round(fwd + adj, 3)
        extra["autograd_over_plain"] = round((fwd + adj) / extra["autograd_fwd_bwd_ms"], 3)
    if extra:
        out["extra"] = extra
    if rank == 0 and not args.no_cpu_baseline:
        xs = x if B > 1 else x[None]
        out["cpu_baseline"] = cpu_baseline(g, xs.cpu().numpy(), budget_s=cpu_budget)
    P.close()
    return out


def _launch_count(P, g, B, fused=False):
    """Kernels of the repo launched per step on the single-image and column paths."""
    # detector setup, ray setup (2D scans and ray lists: a per-ray table; parallel beams and ray
    # lists build both tables in one launch), and for 2D scans reserved for 4 or more images the
    # gather's per-ray constants
    setup = 1 + (0 if g.kind in ("par3d", "cone", "cone_arc", "helix", "helix_arc", "par2d", "rays2d") else 1) + \
        (1 if not g.is3d and P.reserved >= 4 else 0)
    if fused:
        return setup + 1  # the fused forward + adjoint (its zero fill is a memset)
    if P.column_batch:
        # detector setup, the column problem's ray records and gather constants, then per
        # image: the slice planes, the forward, the gather records, the staged gather
        return 3 + 4 * B
    if P.trace_walk:
        # detector setup (no per-ray table), then per image: the padded z-fastest copy, the
        # trace forward, the trace adjoint and the fold of the accumulator (its zero fill is a
        # memset)
        return 1 + 4 * B
    # then per image: the layout copy, the forward walk, the scatter walk and the fold of the
    # accumulator (zero fills are memsets)
    return setup + 4 * B


def run_split(args, rank, world, local_rank):
    """One scan split by views over the ranks (strong scaling): each rank sets up and projects
    its contiguous block of views, back-projects it into a partial image, and one all-reduce
    (NCCL) sums the partial images.  value = rays of the whole scan x images / step time
    (max over ranks)."""
    import torch

    from paper_2006_00686_gb300 import inputs, parallel

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    builder, B, n_shapes, seed, desc = WORKLOADS[args.workload]
    g = getattr(inputs, builder)()
    S = parallel.ShardedProjector(g)
    if B > 1:
        x = inputs.phantom_batch(g, B, n_shapes, seed0=seed, device=str(dev))
    else:
        x = inputs.phantom(g, n_shapes, seed, device=str(dev)).float().contiguous()
    flush = torch.empty(64 * 1024 * 1024, device=dev)
    yb = None
    if S.local is not None:
        yb = torch.empty(S.local_geom.sino_shape(B if B > 1 else None), device=dev)

    def make_step(xb, yblk):
        def step(recs=None):
            st = torch.cuda.current_stream()
            e = _events(2) if recs is not None else None
            if e: e[0].record(st)
            if S.local is not None:
                S.local.ray_setup(st)
                S.forward(xb, out=yblk)
            z = S.adjoint(yblk, like=xb)
            if e: e[1].record(st)
            if recs is not None:
                recs.append(e)
            return z
        return step

    step = make_step(x, yb)
    recs, clocks, wall = _timed_loop(step, args, flush, world, local_rank)
    ms = parallel.max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in recs])), dev)
    rays = g.n_rays * B
    out = {"metric": METRIC, "value": round(rays / (ms * 1e-3) / 1e9, 4), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True,
           "scaling": "strong", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded random-ellipse phantoms)",
           "config": {"workload": args.workload, "geometry": desc, "split": "views",
                      "views_per_rank": [len(v) for v in parallel.view_shards(g.n_views, world)],
                      "collective": "one all-reduce of the partial adjoint images per step",
                      "l2": "flushed between timed steps (256 MiB write)"},
           "gpu_launches": None, "clocks": clocks, "wall_s": round(wall, 3)}
    S.close()
    return out


def _autograd_and_sirt(P, x, y, args):
    """Differentiable forms on the same scan: one autograd forward + backward of
    0.5 ||A x - b||^2, and one SIRT iteration replayed from a CUDA graph."""
    import torch

    from paper_2006_00686_gb300 import recon
    from paper_2006_00686_gb300.xray import project

    b = y.clone()
    xr = torch.zeros_like(x, requires_grad=True)

    def ad():
        xr.grad = None
        loss = 0.5 * (project(xr, P) - b).square().sum()
        loss.backward()

    for _ in range(3):
        ad()
    torch.cuda.synchronize()
    a, e = _events(2)
    n = max(3, min(args.steps, 10))
    a.record()
    for _ in range(n):
        ad()
    e.record()
    e.synchronize()
    ad_ms = a.elapsed_time(e) / n
    s = recon.SIRT(P, b)
    s.capture()
    for _ in range(3):
        s._graph.replay()
    torch.cuda.synchronize()
    a.record()
    for _ in range(n):
        s._graph.replay()
    e.record()
    e.synchronize()
    sirt_ms = a.elapsed_time(e) / n
    # ordered-subset SIRT (8 interleaved view subsets) and Tikhonov CGLS on the same scan
    os = recon.OSSIRT(P.geom, b, 8)
    os.sweep()
    torch.cuda.synchronize()
    a.record()
    for _ in range(n):
        os.sweep()
    e.record()
    e.synchronize()
    os_ms = a.elapsed_time(e) / n
    os.close()
    recon.cgls(P, b, 2, lam=1.0)
    torch.cuda.synchronize()
    a.record()
    recon.cgls(P, b, n, lam=1.0)
    e.record()
    e.synchronize()
    cg_ms = a.elapsed_time(e) / n  # one CGLS iteration: a forward, an adjoint and 3 reductions
    rays = P.geom.n_rays
    return {"os_sirt_sweep_ms": round(os_ms, 3), "cgls_iter_ms": round(cg_ms, 3),
            "autograd_fwd_bwd_ms": round(ad_ms, 3),
            "autograd_grays_s": round(rays / (ad_ms * 1e-3) / 1e9, 4),
            "sirt_iter_ms_graph": round(sirt_ms, 3),
            "sirt_grays_s": round(rays / (sirt_ms * 1e-3) / 1e9, 4)}


def run_uneven(args, rank, world, local_rank, cpu_budget=None):
    """64 uneven fans: one persistent launch for all forwards and one for all adjoints,
    against the plain form (one launch per problem and operator)."""
    import torch

    from paper_2006_00686_gb300 import inputs, parallel
    from paper_2006_00686_gb300.xray import BatchPlan, Projector

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    _, n, n_shapes, seed, desc = WORKLOADS["fans_uneven_64"]
    cpu_budget = args.cpu_budget if cpu_budget is None else cpu_budget
    geoms = inputs.fans_uneven(n)
    Ps = [Projector(gq) for gq in geoms]
    seeds = parallel.rank_seeds(rank, n, seed)
    xs = [inputs.phantom(gq, n_shapes, s, device=str(dev)).float().contiguous() for gq, s in zip(geoms, seeds)]
    ys = [torch.empty(gq.sino_shape(), device=dev) for gq in geoms]
    zs = [torch.empty(gq.image_shape(), device=dev) for gq in geoms]
    for p, xq, yq, zq in zip(Ps, xs, ys, zs):  # workspaces of the plain form, outside the timing
        p.forward(xq, out=yq)
        p.adjoint(yq, out=zq)
    tuned = None
    if not args.tile and not args.plan_block:  # the autotuner picks the plan's work items
        from paper_2006_00686_gb300 import tune as T
        tuned = T.tune_batch_plan(Ps, xs, ys)
        args.tile, args.plan_block = tuned["tile"], tuned["block"]
    fwd_plan = BatchPlan(Ps, xs, ys, tile=args.tile, block=args.plan_block)
    adj_plan = BatchPlan(Ps, zs, ys, tile=args.tile, block=args.plan_block)
    flush = torch.empty(64 * 1024 * 1024, device=dev)
    stream = torch.cuda.current_stream()
    rays_step = sum(gq.n_rays for gq in geoms)

    def batched(recs):
        e = _events(4) if recs is not None else None
        if e: e[0].record(stream)
        fwd_plan.ray_setup(stream)  # every problem's ray setup in two launches
        if e: e[1].record(stream)
        fwd_plan.project(stream)
        if e: e[2].record(stream)
        adj_plan.backproject(stream)
        if e: e[3].record(stream)
        if recs is not None:
            recs.append(e)

    def plain(recs):
        e = _events(4) if recs is not None else None
        if e: e[0].record(stream)
        for p in Ps:
            p.ray_setup(stream)
        if e: e[1].record(stream)
        for p, xq, yq in zip(Ps, xs, ys):
            p.forward(xq, out=yq, stream=stream)
        if e: e[2].record(stream)
        for p, yq, zq in zip(Ps, ys, zs):
            p.adjoint(yq, out=zq, stream=stream)
        if e: e[3].record(stream)
        if recs is not None:
            recs.append(e)

    res = {}
    for name, fn in (("plain", plain), ("batched", batched)):
        recs, clocks, wall = _timed_loop(fn, args, flush, world, local_rank)
        ms = parallel.max_over_ranks(float(np.mean([a.elapsed_time(d) for a, b, c, d in recs])), dev)
        res[name] = {"ms": ms, "clocks": clocks, "wall": wall,
                     "setup": float(np.mean([a.elapsed_time(b) for a, b, c, d in recs])),
                     "fwd": float(np.mean([b.elapsed_time(c) for a, b, c, d in recs])),
                     "adj": float(np.mean([c.elapsed_time(d) for a, b, c, d in recs]))}
    ms = res["batched"]["ms"]
    value = rays_step * world / (ms * 1e-3) / 1e9
    # end to end: two buffer sets, each with its own pair of plans (plans hold their buffers)
    xh = [t.cpu().pin_memory() for t in xs]
    xs1 = [t.clone() for t in xs]
    ys1 = [torch.empty_like(t) for t in ys]
    zs1 = [torch.empty_like(t) for t in zs]
    plans1 = (BatchPlan(Ps, xs1, ys1, tile=args.tile, block=args.plan_block),
              BatchPlan(Ps, zs1, ys1, tile=args.tile, block=args.plan_block))

    def batched_on(fp, ap):
        def step():
            fp.ray_setup(stream)
            fp.project(stream)
            ap.backproject(stream)
        return step

    sets = []
    for (fp, ap), xb, yb, zb in (((fwd_plan, adj_plan), xs, ys, zs), (plans1, xs1, ys1, zs1)):
        sets.append({"step": batched_on(fp, ap), "host_in": xh, "dev_in": xb, "dev_out": yb + zb,
                     "host_out": [torch.empty(t.shape, pin_memory=True) for t in yb + zb]})
    e2e = parallel.max_over_ranks(_e2e(sets, args, flush), dev)
    for pl in plans1:
        pl.close()
    peaks, peak_kind = _peaks()
    rb = res["batched"]
    dom, dom_ms = ("forward", rb["fwd"]) if rb["fwd"] >= rb["adj"] else ("adjoint", rb["adj"])
    # intersections of all problems (one image each), each problem's rate sampled on 256 rays
    n_int = sum(_intersections(gq, p, sample=256) for gq, p in zip(geoms, Ps))
    compulsory = 4.0 * sum(gq.n_units + gq.n_rays for gq in geoms)
    roof = _roofline(n_int, compulsory, 1, "batched " + dom, dom_ms, peaks, peak_kind, None)
    out = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded random-ellipse phantoms)",
           "config": {"workload": "fans_uneven_64", "geometry": desc, "problems": n,
                      "sides": [gq.nx for gq in geoms][:8] + ["..."], "rays_per_step": rays_step,
                      "tile": args.tile, "plan_block": args.plan_block,
                      "plan_tuning": "autotuned" if tuned else "given",
                      "l2": "flushed between timed steps (256 MiB write)"},
           "e2e": {"value": round(rays_step * world / (e2e * 1e-3) / 1e9, 4), "unit": UNIT,
                   "h2d_bytes_per_step": int(sum(t.numel() for t in xs) * 4),
                   "d2h_bytes_per_step": int(sum(t.numel() for t in ys + zs) * 4), "ms_per_step": round(e2e, 4),
                   "method": "pinned copies in and out on two more streams, two buffer sets, L2 flushed "
                             "per step, whole loop timed"},
           # per step: the plan's two setup kernels (every problem's detector samples, then rays);
           # the copies and the persistent forward; the zero fill, the persistent adjoint and the
           # fold of the transposed accumulators
           "gpu_launches": args.steps * 7,
           "kernel_ms": {"ray_setup": round(rb["setup"], 4), "forward": round(rb["fwd"], 4),
                         "adjoint": round(rb["adj"], 4)},
           "plain": {"value": round(rays_step * world / (res["plain"]["ms"] * 1e-3) / 1e9, 4),
                     "ms_per_step": round(res["plain"]["ms"], 4),
                     "kernel_ms": {"forward": round(res["plain"]["fwd"], 4), "adjoint": round(res["plain"]["adj"], 4)}},
           "batched_over_plain": round(res["plain"]["ms"] / ms, 3),
           "clocks": rb["clocks"], "roofline": roof, "wall_s": round(rb["wall"], 3)}
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_uneven(geoms, xs, budget_s=cpu_budget)
    fwd_plan.close()
    adj_plan.close()
    for p in Ps:
        p.close()
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
    n_probe = 1 if g.is3d else 4  # a 3D view is ~1e6 rays
    views = np.arange(0, g.n_views, max(1, g.n_views // n_probe))[:n_probe]  # probe the rate
    t0 = time.perf_counter()
    rays = _oracle_step(O, g, f64, views)
    dt = time.perf_counter() - t0
    n = int(max(len(views), min(g.n_views, len(views) * budget_s / max(dt, 1e-3))))
    if n > len(views):  # else the probe is the sample
        views = np.linspace(0, g.n_views - 1, n).round().astype(np.int64)
        t0 = time.perf_counter()
        rays = _oracle_step(O, g, f64, views)
        dt = time.perf_counter() - t0
    return {"value": round(rays / dt / 1e9, 9), "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
            "sample": f"{len(views)} of {g.n_views} views, all {f64.shape[0]} images, forward+adjoint "
                      f"in float64 ({rays} rays, {dt:.1f} s)"}


def _uneven_sample(O, geoms, imgs, n_views):
    rays = 0
    for gq, xq in zip(geoms, imgs):
        views = np.linspace(0, gq.n_views - 1, n_views).round().astype(np.int64)
        rays += _oracle_step(O, gq, xq.reshape(1, -1).astype(np.float64), views)
    return rays


def cpu_baseline_uneven(geoms, xs, budget_s=15.0):
    from oracle import oracle as O

    imgs = [t.cpu().numpy() for t in xs]
    t0 = time.perf_counter()
    _uneven_sample(O, geoms, imgs, 2)
    dt = time.perf_counter() - t0
    nv = int(max(2, min(geoms[0].n_views, 2 * budget_s / max(dt, 1e-3))))
    t0 = time.perf_counter()
    rays = _uneven_sample(O, geoms, imgs, nv)
    dt = time.perf_counter() - t0
    return {"value": round(rays / dt / 1e9, 9), "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
            "sample": f"{nv} of 720 views of each of the {len(geoms)} problems, forward+adjoint in float64 "
                      f"({rays} rays, {dt:.1f} s)"}


def run_reference(args, rank, world):
    from oracle import oracle as O
    from paper_2006_00686_gb300 import inputs

    builder, B, n_shapes, seed, desc = WORKLOADS[args.workload]
    if builder is None:
        geoms = inputs.fans_uneven(B)
        imgs = [inputs.phantom(gq, n_shapes, seed + q).numpy() for q, gq in enumerate(geoms)]
        n_views = max(1, int(args.ref_views) // 8)

        def sample(k):
            return _uneven_sample(O, geoms, imgs, n_views)
        what = f"{n_views} of 720 views of each of the {B} problems per step, forward+adjoint in float64"
        config = {"workload": args.workload, "geometry": desc, "problems": B}
    else:
        g = getattr(inputs, builder)()
        if B > 1:
            x = inputs.phantom_batch(g, B, n_shapes, seed0=seed).numpy()
        else:
            x = inputs.phantom(g, n_shapes, seed).numpy()[None]
        f64 = x.reshape(B, -1).astype(np.float64)
        n_views = max(1, min(g.n_views, int(args.ref_views) if g.is3d is False else max(1, int(args.ref_views) // 8)))

        def sample(k):
            views = (np.arange(n_views) * (g.n_views // n_views) + k) % g.n_views
            return _oracle_step(O, g, f64, views)
        what = f"{n_views} of {g.n_views} views per step, all {B} images, forward+adjoint in float64"
        config = _config({"sample": what}) if args.workload == "fan2d_512x16" else {
            "workload": args.workload, "geometry": desc, "image": list(g.image_shape()), "views": g.n_views,
            "detector": [g.n_rows, g.n_cols], "batch_per_gpu": B, "sample": what}
    times, rays = [], 0
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        rays = sample(k)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    ms = 1e3 * float(np.mean(times))
    value = rays / (ms * 1e-3) / 1e9
    return {"impl": "reference", "metric": METRIC, "value": round(value, 9), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded random-ellipse phantoms)",
            "config": config,
            "cpu_baseline": {"value": round(value, 9), "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
                             "sample": what},
            "e2e": {"value": round(value, 9), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ----------------------------------------------------------------------------------------
# profiling cases: single kernels on reduced scans (one warm-up pass, one timed pass), sized so
# that one launch takes milliseconds and the volume exceeds L2 where DRAM figures matter
#   python bench.py --case cone_384     forward, scatter and tiled-gather adjoints
#   python bench.py --case uneven_16    16 uneven fans: plain launches, then one plan
# ----------------------------------------------------------------------------------------

def case_cone_384():
    """Circular cone, 384^3 voxels (226 MB) spanning the 512^3 scan's field of view, 90 views,
    512 x 384 detector of spacing 2."""
    v = np.arange(90, dtype=np.float64)
    s = 512 / 384
    import torch

    from paper_2006_00686_gb300 import inputs
    from paper_2006_00686_gb300.xray import Projector

    g = inputs.Geometry("cone", 384, 384, 384, dx=0.8 * s, dy=0.8 * s, dz=1.0 * s, cx=10.0, cy=-5.0, cz=3.0,
                        angles=2 * math.pi * v / 90, n_cols=512, n_rows=384, du=2.0, dv=2.0, sod=1000.0, sdd=1500.0)
    P = Projector(g)
    x = inputs.phantom(g, 30, 4, device="cuda").float().contiguous()
    y = torch.empty(g.sino_shape(), device="cuda")
    z = torch.empty(g.image_shape(), device="cuda")
    times = []
    for rep in range(2):
        e = _events(4)
        e[0].record()
        P.forward(x, out=y)
        e[1].record()
        P.adjoint(y, out=z, method=1)
        e[2].record()
        P.adjoint(y, out=z, method=2)
        e[3].record()
        e[3].synchronize()
        times = [e[i].elapsed_time(e[i + 1]) for i in range(3)]
    print(f"cone_384: rays {g.n_rays}, forward {times[0]:.3f} ms, scatter {times[1]:.3f} ms, "
          f"tiled gather {times[2]:.3f} ms")


def case_uneven_16():
    """The first 16 of the 64 uneven fans: the plain adjoint (one launch set per problem),
    then the same adjoints as one persistent plan."""
    import torch

    from paper_2006_00686_gb300 import inputs
    from paper_2006_00686_gb300.xray import BatchPlan, Projector

    geoms = inputs.fans_uneven()[:16]
    Ps = [Projector(g) for g in geoms]
    xs = [inputs.phantom(g, 10, 500 + q, device="cuda").float().contiguous() for q, g in enumerate(geoms)]
    ys = [torch.empty(g.sino_shape(), device="cuda") for g in geoms]
    zs = [torch.empty(g.image_shape(), device="cuda") for g in geoms]
    for p, x, y, z in zip(Ps, xs, ys, zs):
        p.forward(x, out=y)
        p.adjoint(y, out=z)
    plan = BatchPlan(Ps, zs, ys, tile=64, block=256)
    torch.cuda.synchronize()
    e = _events(3)
    e[0].record()
    for p, y, z in zip(Ps, ys, zs):
        p.adjoint(y, out=z)
    e[1].record()
    plan.backproject()
    e[2].record()
    e[2].synchronize()
    print(f"uneven_16: plain adjoints {e[0].elapsed_time(e[1]):.3f} ms, one plan {e[1].elapsed_time(e[2]):.3f} ms")


CASES = {"cone_384": case_cone_384, "uneven_16": case_uneven_16}


# the other scan configurations measured in the default run, with the same K and W (the
# 3D scans at most PER_CONFIG_3D_STEPS timed steps) and a shorter oracle sample
PER_CONFIG = ("par2d_64", "par3d_256_tilt", "cone_512", "helix_512x256", "fans_uneven_64")
PER_CONFIG_3D_STEPS = 20
PER_CONFIG_SHORT_STEPS = 20000
PER_CONFIG_CPU_S = 5.0


def per_config(args, rank, world, local_rank):
    import copy

    import torch
    res = {}
    for wl in PER_CONFIG:
        a = copy.copy(args)
        a.workload = wl
        if wl in ("cone_512", "helix_512x256"):
            a.steps = min(args.steps, PER_CONFIG_3D_STEPS)
        if wl == "par2d_64":  # 0.03 ms steps: enough of them for the clock sampler (~0.6 s)
            a.steps = max(args.steps, PER_CONFIG_SHORT_STEPS)
        if wl == "fans_uneven_64":
            a.tile = a.plan_block = 0
        t0 = time.perf_counter()
        r = run_ours(a, rank, world, local_rank, workload=wl, cpu_budget=PER_CONFIG_CPU_S)
        r["bench_wall_s"] = round(time.perf_counter() - t0, 1)
        for k in ("metric", "unit", "n_gpus", "higher_is_better", "scaling", "vs_baseline", "dtype", "data"):
            r.pop(k, None)
        res[wl] = r
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default 100; 5 for the 3D scans)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=None, choices=sorted(WORKLOADS),
                    help="one workload only (default: the fan-beam headline plus every other scan "
                         "configuration under extra.per_config)")
    ap.add_argument("--no-per-config", action="store_true", help="the headline workload only")
    ap.add_argument("--split", default=None, choices=["views"],
                    help="split one scan of --workload by views over the ranks (strong scaling, one "
                         "all-reduce of the adjoint per step) instead of one batch per rank")
    ap.add_argument("--case", default=None, help="run one profiling case (%s) and exit" % ", ".join(
        ["cone_384", "uneven_16"]))
    ap.add_argument("--adjoint", default=None, choices=["gather", "scatter"],
                    help="adjoint method (default: the gather for 2D batches and single-tilt-axis "
                         "parallel scans, the scatter elsewhere)")
    ap.add_argument("--chunk", type=int, default=0, help="images per thread of the batched path")
    ap.add_argument("--order", default="auto", choices=["auto", "view", "row", "column", "rowblock"],
                    help="ray order of the 3D single-image path")
    ap.add_argument("--block", type=int, default=128)
    ap.add_argument("--tile", type=int, default=0, help="rays per work item of the persistent batch")
    ap.add_argument("--plan-block", type=int, default=0, help="threads per CTA of the persistent batch")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-views", type=int, default=24)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    all_configs = args.workload is None and not args.no_per_config
    if args.workload is None:
        args.workload = "fan2d_512x16"
    if args.steps is None:
        args.steps = 5 if args.workload in ("par3d_256_tilt", "cone_512", "helix_512x256") else 100

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args, rank, world)), flush=True)
        return

    import torch
    if args.case:
        import __graft_entry__
        __graft_entry__.build()
        CASES[args.case]()
        return
    if world > 1:
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    import __graft_entry__
    if rank == 0:  # one process builds (or finds the build current); the others wait for it
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
    if rank != 0:
        __graft_entry__.build()  # up to date by now: only checks and imports
    if args.split == "views":
        out = run_split(args, rank, world, local_rank)
        if rank == 0:
            print(json.dumps(out), flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    out = run_ours(args, rank, world, local_rank)
    if all_configs:
        out.setdefault("extra", {})["per_config"] = per_config(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
