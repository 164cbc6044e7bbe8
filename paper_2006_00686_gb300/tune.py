"""Autotuner: chooses launch parameters by timing them on the current GPU.

* ``tune_projector`` -- for one scan and batch size: the batched path (quad planes,
  shared-memory tiles or one thread per ray), the images walked per thread, the adjoint
  method (gather or scatter) and the block size of the one-thread-per-ray kernels; the
  candidate with the least forward + adjoint time wins.
* ``tune_batch_plan`` -- for a persistent uneven batch: rays per work item and threads
  per CTA.

Results are cached in a JSON file keyed by GPU name and scan (sizes, views, detector,
batch), so a second process reuses them without timing anything.
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

from . import xray as X


def _gpu_name() -> str:
    return torch.cuda.get_device_name(torch.cuda.current_device())


def scan_key(g, batch: int) -> str:
    return (f"{_gpu_name()}|{g.kind}|{g.nx}x{g.ny}x{g.nz}|{g.dx:g},{g.dy:g},{g.dz:g}|v{g.n_views}"
            f"|d{g.n_rows}x{g.n_cols}|b{batch}")


def _load(path):
    if path and os.path.exists(path):
        try:
            with open(path) as fh:
                return json.load(fh)
        except (OSError, ValueError):
            return {}
    return {}


def _store(path, cache):
    if not path:
        return
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time(fn, reps: int, budget_s: float) -> float:
    """Median milliseconds of fn over up to `reps` runs (fewer if over the time budget)."""
    fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b))
        if sum(times) > 1e3 * budget_s:
            break
    return float(np.median(times))


def projector_candidates(g, batch: int) -> list:
    out = []
    if g.is3d:
        # the column-trace walk of cone and helical scans (scatter adjoint), the volume-copy path
        # in either ray order with either adjoint, then the caller's layout
        if g.kind in ("cone", "cone_arc", "helix", "helix_arc"):
            out.append(dict(path=X.XR_PATH_INTERLEAVED, batch_chunk=16, adjoint=X.XR_ADJ_SCATTER, block=128,
                            order=X.XR_ORDER_TRACE))
        for order in (X.XR_ORDER_VIEW, X.XR_ORDER_ROW, X.XR_ORDER_COLUMN, X.XR_ORDER_ROWBLOCK):
            for adj in (X.XR_ADJ_GATHER, X.XR_ADJ_SCATTER):
                out.append(dict(path=X.XR_PATH_INTERLEAVED, batch_chunk=16, adjoint=adj, block=128, order=order))
        out.append(dict(path=X.XR_PATH_INTERLEAVED, batch_chunk=16, adjoint=X.XR_ADJ_GATHER, block=256,
                        order=X.XR_ORDER_ROW))
        out.append(dict(path=X.XR_PATH_RAY, batch_chunk=min(16, max(1, batch)), adjoint=X.XR_ADJ_SCATTER,
                        block=128, order=X.XR_ORDER_VIEW))
        return out
    if batch >= 4:
        for chunk in (16, 8, 4):
            if chunk > 4 * ((batch + 3) // 4) and chunk != 4:
                continue
            for adj in (X.XR_ADJ_GATHER, X.XR_ADJ_SCATTER):
                out.append(dict(path=X.XR_PATH_INTERLEAVED, batch_chunk=chunk, adjoint=adj, block=128))
        out.append(dict(path=X.XR_PATH_TILED, batch_chunk=16, adjoint=X.XR_ADJ_SCATTER, block=128))
    else:
        # one image at a time through the image and its y-fastest copy
        for adj in (X.XR_ADJ_SCATTER, X.XR_ADJ_GATHER):
            out.append(dict(path=X.XR_PATH_INTERLEAVED, batch_chunk=1, adjoint=adj, block=128))
    for block in (128, 256):
        for adj in (X.XR_ADJ_SCATTER, X.XR_ADJ_GATHER):
            out.append(dict(path=X.XR_PATH_RAY, batch_chunk=1 if batch < 4 else min(16, batch), adjoint=adj,
                            block=block))
    return out


def _apply(P, c):
    P.set_tuning(block=c["block"], batch_chunk=c["batch_chunk"], adjoint=c["adjoint"], path=c["path"],
                 order=c.get("order", 0))


def tune_projector(P: "X.Projector", batch: int, cache_path: str | None = None, reps: int = 5,
                   budget_s: float = 2.0, x=None, verbose: bool = False) -> dict:
    """Choose and apply the fastest tuning for batches of `batch` images; returns it with
    the measured times."""
    g = P.geom
    key = scan_key(g, batch)
    cache = _load(cache_path)
    if key in cache:
        best = cache[key]
        _apply(P, best)
        return best
    dev = P.device
    if x is None:
        x = torch.rand(g.image_shape(batch if batch > 1 else None), device=dev)
    y = torch.empty(g.sino_shape(batch if batch > 1 else None), device=dev)
    z = torch.empty_like(x)
    P.reserve(max(batch, 1))
    results = []
    for c in projector_candidates(g, batch):
        _apply(P, c)
        f_ms = _time(lambda: P.forward(x, out=y), reps, budget_s)
        a_ms = _time(lambda: P.adjoint(y, out=z), reps, budget_s)
        results.append(dict(c, forward_ms=f_ms, adjoint_ms=a_ms))
        if verbose:
            print("tune", key, results[-1], flush=True)
    best = min(results, key=lambda r: r["forward_ms"] + r["adjoint_ms"])
    _apply(P, best)
    cache = _load(cache_path)
    cache[key] = best
    _store(cache_path, cache)
    return best


def tune_batch_plan(projectors, images, sinos, cache_path: str | None = None, reps: int = 3,
                    budget_s: float = 2.0, verbose: bool = False) -> dict:
    """Choose rays per work item and threads per CTA of a persistent uneven batch by timing
    its forward and adjoint launches (the adjoint writes scratch images, not `images`)."""
    key = _gpu_name() + "|plan|" + ";".join(scan_key(p.geom, 1) for p in projectors)
    cache = _load(cache_path)
    if key in cache:
        return cache[key]
    scratch = [torch.empty_like(x) for x in images]
    results = []
    for tile in (64, 128, 256, 512, 1024):
        for block in (128, 256):
            fwd = X.BatchPlan(projectors, images, sinos, tile=tile, block=block)
            adj = X.BatchPlan(projectors, scratch, sinos, tile=tile, block=block)
            f_ms = _time(fwd.project, reps, budget_s)
            a_ms = _time(adj.backproject, reps, budget_s)
            results.append(dict(tile=tile, block=block, forward_ms=f_ms, adjoint_ms=a_ms))
            if verbose:
                print("tune plan", results[-1], flush=True)
            fwd.close()
            adj.close()
    best = min(results, key=lambda r: r["forward_ms"] + r["adjoint_ms"])
    cache = _load(cache_path)
    cache[key] = best
    _store(cache_path, cache)
    return best
