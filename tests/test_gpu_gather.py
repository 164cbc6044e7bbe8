"""The gather adjoint of 2D batches (per-warp shared-memory stages of per-ray records) on the
views it stages, the views it reads from global memory, and the views with rays parallel to an
axis, against the oracle; and the way out of its bounded waits.

A warp's 8 x 8 pixel tile projects onto at most 32 bins in a staged view; detectors finer than
the pixels make some views (oblique ones first) or all views exceed that, and those are read
from the records in global memory.  Views at 0 and 90 degrees of a parallel scan hold rays on
the pixel rows and columns, whose lengths only the walk gives."""
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


def _geom(which):
    v = np.arange(24, dtype=np.float64)
    kw = dict(nx=45, ny=38, dx=1.0, dy=1.0, cx=0.6, cy=-0.3)
    if which == "par_mixed":
        # 8 (|cos| + |sin|) / 0.33 + 2 bins: 26 at 0 degrees (staged), 36 at 45 (direct)
        return Geometry("par2d", angles=pi * v / 24, n_cols=220, du=0.33, u0=0.05, **kw)
    if which == "par_direct":
        return Geometry("par2d", angles=pi * v / 24 + 0.1, n_cols=330, du=0.2, u0=0.03, **kw)
    if which == "par_axes":
        # four views on the axes (every ray parallel to the pixel rows or columns), four oblique;
        # the detector offset keeps rays 0.25 away from grid lines (no tie to break)
        ang = np.array([0.0, pi / 2, pi, 3 * pi / 2, 0.3, 1.2, 2.0, 2.8])
        return Geometry("par2d", angles=ang, n_cols=61, du=1.0, u0=0.25, **kw)
    if which == "fan_fine":
        return Geometry("fan2d", angles=2 * pi * v / 24, n_cols=400, du=0.35, u0=0.1, sod=120.0, sdd=200.0, **kw)
    return Geometry("fan2d_arc", angles=2 * pi * v / 24, n_cols=400, du=0.0022, u0=0.0005, sod=120.0, sdd=200.0,
                    **kw)


@pytest.mark.parametrize("which", ["par_mixed", "par_direct", "par_axes", "fan_fine", "arc_fine"])
@pytest.mark.parametrize("batch,chunk", [(16, 16), (5, 8), (4, 4)])
def test_gather_staged_direct_and_axis_views(X, which, batch, chunk):
    # four, two and one planes of 4 images per thread
    g = _geom(which)
    P = X.Projector(g)
    P.reserve(batch)
    P.set_tuning(batch_chunk=chunk)
    rng = np.random.default_rng(batch + len(which))
    y = torch.from_numpy(rng.uniform(-1.0, 1.0, g.sino_shape(batch)).astype(np.float32)).cuda()
    z = P.adjoint(y, method=X.XR_ADJ_GATHER).cpu().numpy().reshape(batch, -1)
    z_ref = O.adjoint(g, y.cpu().numpy().astype(np.float64).reshape(batch, -1))
    for b in range(batch):
        H.check_adjoint(z[b], z_ref[b], f"{which}[{b}] gather")
    # the exact transpose of the forward on the same scan
    f = torch.from_numpy(rng.uniform(0.0, 1.0, (batch,) + g.image_shape()).astype(np.float32)).cuda()
    Af = P.forward(f).double()
    lhs = float((Af * y.double()).sum())
    rhs = float((f.double() * torch.from_numpy(z).cuda().reshape(f.shape)).sum())
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), float((Af.abs() * y.double().abs()).sum()) * 1e-2), (lhs, rhs)
    assert P.device_error() == 0
    P.close()


def test_bounded_wait_gives_up_and_the_device_stays_usable(X):
    # nothing completes the barrier: the wait returns after its bound (about 1 ms here), the
    # warp reports it, and the next launches run normally
    assert X.wait_bound_selftest(2_000_000)
    g = _geom("par_mixed")
    P = X.Projector(g)
    y = torch.ones(g.sino_shape(4), device="cuda")
    z = P.adjoint(y, method=X.XR_ADJ_GATHER).cpu().numpy().reshape(4, -1)
    z_ref = np.asarray(O.adjoint(g, np.ones(g.n_rays))).reshape(-1)
    H.check_adjoint(z[3], z_ref, "after the self-test")
    assert P.device_error() == 0
    P.close()


@pytest.mark.parametrize("kind", ["par2d", "fan2d", "fan2d_arc"])
def test_single_image_2d_adjoint_lockstep(X, kind):
    # a single-image 2D scan large enough to fill the GPU (more than 1024 rays per SM) takes
    # the scatter with 32 neighbouring rays per warp in lockstep; odd sizes, off-centre pixels,
    # views on the axes.  The parallel detector's offset keeps every ray at least 0.05 from a
    # grid line, so the oracle and the ray setup cannot break a tie (the bigger-index rule)
    # differently through rounding
    v = np.arange(720, dtype=np.float64)
    kw = dict(nx=201, ny=187, dx=0.9, dy=1.1, cx=1.5, cy=-2.0, n_cols=251)
    if kind == "par2d":
        g = Geometry(kind, angles=pi * v / 720, du=0.8, u0=0.3, **kw)
    elif kind == "fan2d":
        g = Geometry(kind, angles=2 * pi * v / 720, du=1.3, u0=0.4, sod=400.0, sdd=600.0, **kw)
    else:
        g = Geometry(kind, angles=2 * pi * v / 720, du=0.0021, u0=0.0003, sod=400.0, sdd=600.0, **kw)
    assert g.n_rays >= 1024 * torch.cuda.get_device_properties(0).multi_processor_count
    P = X.Projector(g)
    rng = np.random.default_rng(7)
    y = torch.from_numpy(rng.uniform(0.0, 1.0, g.sino_shape()).astype(np.float32)).cuda()
    z = P.adjoint(y, method=X.XR_ADJ_SCATTER).cpu().numpy().reshape(-1)
    z_ref = np.asarray(O.adjoint(g, y.cpu().numpy().astype(np.float64).reshape(-1))).reshape(-1)
    H.check_adjoint(z, z_ref, f"{kind} single-image lockstep adjoint")
    f = torch.from_numpy(rng.uniform(0.0, 1.0, g.image_shape()).astype(np.float32)).cuda()
    Af = P.forward(f).double()
    lhs = float((Af * y.double()).sum())
    rhs = float((f.double() * torch.from_numpy(z).cuda().reshape(f.shape).double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)
    P.close()
