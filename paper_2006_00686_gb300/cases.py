"""Small named cases for profiling single kernels (one warm-up pass, one timed pass).

    python -m paper_2006_00686_gb300.cases cone_384      # forward, scatter and tiled gather adjoints
    python -m paper_2006_00686_gb300.cases uneven_16     # 16 uneven fans: plain launches, then one plan

Each case is sized so that one launch of each kernel takes milliseconds and the volume is
larger than L2 (129 MB) where DRAM figures matter, as the profiling captures need.
"""
from __future__ import annotations

import math
import sys

import numpy as np
import torch

from . import inputs
from .xray import BatchPlan, Projector


def _events(n):
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def cone_384():
    """Circular cone, 384^3 voxels (226 MB) spanning the 512^3 scan's field of view, 90 views,
    512 x 384 detector of spacing 2."""
    v = np.arange(90, dtype=np.float64)
    s = 512 / 384
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


def uneven_16():
    """The first 16 of the 64 uneven fans: the plain adjoint (one launch set per problem),
    then the same adjoints as one persistent plan."""
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


CASES = {"cone_384": cone_384, "uneven_16": uneven_16}

if __name__ == "__main__":
    for name in sys.argv[1:] or list(CASES):
        CASES[name]()
