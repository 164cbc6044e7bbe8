"""Degenerate grids on every GPU path, against the oracle: images one pixel wide or high (a
single column of pixel pairs, a lone last pixel in every row, one 8 x 8 tile), a single
pixel, and thin 3D volumes; batched (quad planes, staged gather), single-image and fused."""
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


def _g2(kind, nx, ny):
    v = np.arange(16, dtype=np.float64)
    kw = dict(dx=0.9, dy=1.1, cx=0.2, cy=-0.15, n_cols=9)
    if kind == "par2d":
        return Geometry(kind, nx, ny, angles=pi * v / 16 + 0.05, du=0.7, u0=0.13, **kw)
    return Geometry(kind, nx, ny, angles=2 * pi * v / 16 + 0.05, du=0.9, u0=0.11, sod=30.0, sdd=45.0, **kw)


def _check(X, g, batch, what, fused=True):
    rng = np.random.default_rng(batch + g.nx * 7 + g.ny)
    shape = (batch,) + g.image_shape() if batch > 1 else g.image_shape()
    f = rng.uniform(0.5, 1.5, shape).astype(np.float32)
    P = X.Projector(g)
    y = P.forward(torch.from_numpy(f).cuda()).cpu().numpy().reshape(batch, -1)
    f64 = f.astype(np.float64).reshape(batch, -1)
    y_ref = np.asarray(O.forward(g, f64)).reshape(batch, -1)
    scale = np.asarray(O.forward(g, np.abs(f64))).reshape(batch, -1)
    s = rng.uniform(0.0, 1.0, (batch, g.n_rays)).astype(np.float32)
    s_t = torch.from_numpy(s.reshape(((batch,) if batch > 1 else ()) + g.sino_shape())).cuda()
    z_ref = np.asarray(O.adjoint(g, s.astype(np.float64))).reshape(batch, -1)
    methods = [X.XR_ADJ_SCATTER] + ([] if g.is3d else [X.XR_ADJ_GATHER])
    for b in range(batch):
        H.check_rays(g, y[b], y_ref[b], scale[b], float(np.abs(f64[b]).max()), f"{what}[{b}] forward")
    for m in methods:
        z = P.adjoint(s_t, method=m).cpu().numpy().reshape(batch, -1)
        for b in range(batch):
            H.check_adjoint(z[b], z_ref[b], f"{what}[{b}] adjoint method {m}")
    if fused:
        yf, zf = P.forward_adjoint(torch.from_numpy(f).cuda())
        zf_ref = np.asarray(O.adjoint(g, yf.cpu().numpy().astype(np.float64).reshape(batch, -1))).reshape(batch, -1)
        zf = zf.cpu().numpy().reshape(batch, -1)
        for b in range(batch):
            H.check_adjoint(zf[b], zf_ref[b], f"{what}[{b}] fused")
    P.close()


@pytest.mark.parametrize("kind", ["par2d", "fan2d"])
@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 7), (7, 1), (2, 3), (3, 2), (9, 1), (1, 9)])
@pytest.mark.parametrize("batch", [1, 16])
def test_thin_2d_grids(X, kind, nx, ny, batch):
    _check(X, _g2(kind, nx, ny), batch, f"{kind} {nx}x{ny}")


@pytest.mark.parametrize("dims", [(1, 1, 1), (1, 5, 3), (5, 1, 3), (4, 3, 1)])
@pytest.mark.parametrize("kind", ["par3d", "cone", "helix"])
def test_thin_3d_grids(X, kind, dims):
    nx, ny, nz = dims
    v = np.arange(12, dtype=np.float64)
    kw = dict(dx=0.9, dy=1.1, dz=1.0, cx=0.1, cy=-0.2, cz=0.05, n_cols=7, n_rows=5)
    if kind == "par3d":
        ang = np.stack([2 * pi * v / 12 + 0.1, np.linspace(-0.6, 0.6, 12)], axis=1)
        g = Geometry(kind, nx, ny, nz, angles=ang, du=0.8, dv=0.7, u0=0.07, v0=0.05, **kw)
    else:
        src = np.linspace(-1.5, 1.5, 12) if kind == "helix" else None
        g = Geometry(kind, nx, ny, nz, angles=2 * pi * v / 12 + 0.1, du=0.9, dv=0.8, u0=0.07, v0=0.05,
                     sod=25.0, sdd=40.0, src_z=src, **kw)
    _check(X, g, 1, f"{kind} {dims}")
