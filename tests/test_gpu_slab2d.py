"""Edge cases of the single-image 2D slab walks against the oracle.

A 2D scan with 1024 rays per SM or more takes the pair-plane forward (one ray per thread, slab
by slab) and the lockstep adjoint (32 rays per warp into padded accumulator planes); so do the
problems of a batch plan whose problems are all 2D.  Both clamp or pad the minor row instead of
testing bounds, so images one pixel wide or high, rays that miss or graze the image, unordered
ray lists (the warp's lanes then disagree on the driving axis) and views whose rays all run
parallel to an axis (every lane walks alone) are checked here: forward per ray, adjoint image
and the dot test."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2006_00686_gb300.inputs import Geometry
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu
pi = math.pi


@pytest.fixture(scope="module")
def X():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    from paper_2006_00686_gb300 import xray
    return xray


def _big_enough(g):
    assert g.n_rays >= 1024 * torch.cuda.get_device_properties(0).multi_processor_count


def _check(X, g, what, seed, near_axis=False):
    # near_axis: the scan has rays within a few thousandths of a radian of an axis on an image
    # a few units across, where the per-ray bound takes the near-axis term (tests/gpu_helpers.py)
    rng = np.random.default_rng(seed)
    f = rng.uniform(0.5, 1.5, g.image_shape()).astype(np.float32)
    f64 = f.astype(np.float64).reshape(-1)
    P = X.Projector(g)
    y = P.forward(torch.from_numpy(f).cuda()).cpu().numpy().reshape(-1)
    w_min = H.minor_slope_2d(g, range(g.n_rays)) if near_axis else None
    H.check_rays(g, y, np.asarray(O.forward(g, f64)).reshape(-1), np.asarray(O.forward(g, np.abs(f64))).reshape(-1),
                 float(np.abs(f64).max()), f"{what} forward", w_min=w_min)
    s = rng.uniform(0.0, 1.0, g.n_rays).astype(np.float32)
    s_t = torch.from_numpy(s.reshape(g.sino_shape())).cuda()
    z = P.adjoint(s_t, method=X.XR_ADJ_SCATTER).cpu().numpy().reshape(-1)
    H.check_adjoint(z, np.asarray(O.adjoint(g, s.astype(np.float64))).reshape(-1), f"{what} adjoint")
    lhs = float((torch.from_numpy(y).double() * torch.from_numpy(s).double()).sum())
    rhs = float((torch.from_numpy(f64) * torch.from_numpy(z).double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (what, lhs, rhs)
    P.close()


@pytest.mark.parametrize("kind", ["par2d", "fan2d"])
@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 7), (7, 1), (2, 3), (9, 1), (1, 9)])
def test_thin_images_on_the_slab_walks(X, kind, nx, ny):
    # 720 views x 233 bins: the single-image slab walks; the detector covers the image with
    # rays that miss it on both sides.  Some views lie 0.0013 rad from an axis
    v = np.arange(720, dtype=np.float64)
    kw = dict(dx=0.9, dy=1.1, cx=0.2, cy=-0.15, n_cols=233)
    if kind == "par2d":
        g = Geometry(kind, nx, ny, angles=pi * v / 720 + 0.0013, du=0.061, u0=0.0071, **kw)
    else:
        g = Geometry(kind, nx, ny, angles=2 * pi * v / 720 + 0.0013, du=0.093, u0=0.0083, sod=30.0, sdd=45.0, **kw)
    _big_enough(g)
    _check(X, g, f"{kind} {nx}x{ny}", seed=nx * 31 + ny, near_axis=True)


def test_unordered_ray_list_on_the_slab_walks(X):
    # random rays: the lanes of a warp share no view, so they disagree on the driving axis and
    # walk far-apart slab ranges; rays that miss the image too
    rng = np.random.default_rng(5)
    n = 170000
    half = 0.5 * math.hypot(37 * 0.9, 29 * 1.1)
    ang = np.stack([rng.uniform(-1.2 * half, 1.2 * half, n), rng.uniform(0, 2 * pi, n)], axis=1)
    g = Geometry("rays2d", 37, 29, dx=0.9, dy=1.1, cx=0.4, cy=-0.3, angles=ang)
    _big_enough(g)
    _check(X, g, "rays2d", seed=6)


def test_axis_parallel_views_on_the_slab_walks(X):
    # every ray parallel to the pixel rows or columns: no lane steps in lockstep, all walk alone;
    # the detector offset keeps every ray at least 1e-4 from a grid line (no tie to break)
    ang = np.array([0.0, pi / 2, pi, 3 * pi / 2])
    g = Geometry("par2d", 40, 30, dx=0.9, dy=1.1, cx=0.3, cy=-0.2, angles=ang, n_cols=40001, du=0.001,
                 u0=0.00037)
    u = (np.arange(g.n_cols) - (g.n_cols - 1) / 2) * 0.001 + 0.00037
    lines = np.concatenate([0.3 - 20 * 0.9 + 0.9 * np.arange(41), -0.2 - 15 * 1.1 + 1.1 * np.arange(31)])
    for s in (u, -u):
        assert np.abs(s[:, None] - lines[None, :]).min() >= 1e-4
    _big_enough(g)
    _check(X, g, "par2d axis views", seed=8)


def test_plan_of_thin_problems_and_a_ray_list(X):
    # a persistent plan of 2D problems (pair-plane forward, lockstep adjoint into each problem's
    # planes): thin images, a single pixel and a random ray list, with ragged work items
    rng = np.random.default_rng(9)
    v = np.arange(90, dtype=np.float64)
    geoms = [Geometry("fan2d", nx, ny, dx=0.9, dy=1.1, cx=0.2, cy=-0.1, angles=2 * pi * v / 90 + 0.01, n_cols=37,
                      du=0.7, u0=0.05, sod=40.0, sdd=60.0) for nx, ny in ((1, 13), (13, 1), (1, 1), (6, 5))]
    half = 0.5 * math.hypot(11 * 0.9, 7 * 1.1)
    ang = np.stack([rng.uniform(-half, half, 3001), rng.uniform(0, 2 * pi, 3001)], axis=1)
    geoms.append(Geometry("rays2d", 11, 7, dx=0.9, dy=1.1, cx=0.1, cy=0.2, angles=ang))
    Ps = [X.Projector(g) for g in geoms]
    fs = [torch.from_numpy(rng.uniform(0.5, 1.5, g.image_shape()).astype(np.float32)).cuda() for g in geoms]
    ys = [torch.empty(g.sino_shape(), device="cuda") for g in geoms]
    X.BatchPlan(Ps, fs, ys, tile=96).project()
    sv = [torch.from_numpy(rng.uniform(0.0, 1.0, g.sino_shape()).astype(np.float32)).cuda() for g in geoms]
    zs = [torch.full(g.image_shape(), float("nan"), device="cuda") for g in geoms]
    X.BatchPlan(Ps, zs, sv, tile=96).backproject()
    torch.cuda.synchronize()
    for q, g in enumerate(geoms):
        f64 = fs[q].cpu().numpy().astype(np.float64).reshape(-1)
        H.check_rays(g, ys[q].cpu().numpy().reshape(-1), np.asarray(O.forward(g, f64)).reshape(-1),
                     np.asarray(O.forward(g, np.abs(f64))).reshape(-1), float(np.abs(f64).max()), f"plan forward {q}")
        z_ref = np.asarray(O.adjoint(g, sv[q].cpu().numpy().astype(np.float64).reshape(-1))).reshape(-1)
        H.check_adjoint(zs[q].cpu().numpy().reshape(-1), z_ref, f"plan adjoint {q}")
    for P in Ps:
        P.close()
