"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Unit sets of single rays, forward and adjoint on reduced copies of every scan
configuration, the five configurations at full size on sampled rays (forward) and on view
subsets (adjoint), the dot-product test, batching and the ambiguity rule."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2006_00686_gb300 import inputs
from paper_2006_00686_gb300.inputs import Geometry
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu
pi = math.pi


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _proj(g):
    from paper_2006_00686_gb300.xray import Projector
    return Projector(g)


def _phantom(g, seed, n_shapes=8, device="cpu"):
    return inputs.phantom(g, n_shapes, seed, device=device)


# ---------------------------------------------------------------------------------------
# Unit sets (sparse rows) of single rays
# ---------------------------------------------------------------------------------------

def _rand_geom(kind, rng):
    three = kind in inputs.KINDS_3D
    nx, ny = int(rng.integers(9, 41)), int(rng.integers(9, 41))
    nz = int(rng.integers(9, 33)) if three else 1
    kw = dict(nx=nx, ny=ny, nz=nz, dx=rng.uniform(0.6, 1.4), dy=rng.uniform(0.6, 1.4), dz=rng.uniform(0.6, 1.4),
              cx=rng.uniform(-2, 2), cy=rng.uniform(-2, 2), cz=rng.uniform(-2, 2))
    nv = 7
    if kind in ("rays2d", "rays3d"):
        # rays given by their parameters, spread over the image's bounding circle
        half = 0.5 * math.sqrt((nx * kw["dx"]) ** 2 + (ny * kw["dy"]) ** 2 + (nz * kw["dz"]) ** 2)
        n = 900
        if kind == "rays2d":
            ang = np.stack([rng.uniform(-half, half, n), rng.uniform(-pi, 3 * pi, n)], axis=1)
        else:
            ang = np.stack([rng.uniform(-half, half, n), rng.uniform(-half, half, n), rng.uniform(-pi, 3 * pi, n),
                            rng.uniform(-pi, pi, n)], axis=1)
        return Geometry(kind, angles=ang, **kw)
    if kind == "par2d":
        return Geometry(kind, angles=rng.uniform(-pi, 3 * pi, nv), n_cols=41, du=rng.uniform(0.5, 1.5), **kw)
    if kind == "fan2d":
        return Geometry(kind, angles=rng.uniform(0, 2 * pi, nv), n_cols=41, du=rng.uniform(1, 2),
                        sod=100.0, sdd=160.0, **kw)
    if kind == "fan2d_arc":
        return Geometry(kind, angles=rng.uniform(0, 2 * pi, nv), n_cols=41, du=0.012, sod=100.0, sdd=160.0, **kw)
    if kind == "par3d":
        ang = np.stack([rng.uniform(-pi, 3 * pi, nv), rng.uniform(-pi, pi, nv)], axis=1)
        return Geometry(kind, angles=ang, n_cols=21, n_rows=17, du=rng.uniform(1, 2), dv=rng.uniform(1, 2), **kw)
    src_z = rng.uniform(-5, 5, nv) if kind.startswith("helix") else None
    if kind in ("cone", "helix"):
        return Geometry(kind, angles=rng.uniform(0, 2 * pi, nv), src_z=src_z, n_cols=21, n_rows=17,
                        du=rng.uniform(2, 3), dv=rng.uniform(2, 3), sod=100.0, sdd=160.0, **kw)
    return Geometry(kind, angles=rng.uniform(0, 2 * pi, nv), src_z=src_z, n_cols=21, n_rows=17,
                    du=0.02, dv=0.02, sod=100.0, sdd=160.0, **kw)


@pytest.mark.parametrize("kind", list(inputs.KINDS))
def test_unit_sets_random_geometry(kind):
    rng = np.random.default_rng(100 + inputs.KINDS[kind])
    g = _rand_geom(kind, rng)
    rays = H.sample_rays(g, 600, seed=1)
    P = _proj(g)
    rows_gpu = P.ray_units(rays)
    rows_ref = [O.ray_units(g, int(r)) for r in rays]
    graze = H.check_unit_sets(g, rows_gpu, rows_ref)
    n_units = sum(len(r[1]) for r in rows_ref)
    assert n_units > 1000 and graze <= 0.01 * n_units


SPECIAL_3D = [(a, b) for a in (0.0, pi / 2, pi, 3 * pi / 2, 0.4, 2.2, 4.0, 5.5)
              for b in (0.0, pi / 2, -pi / 2, 0.3, -0.5, pi / 4)]


@pytest.mark.parametrize("offset", [0.0, 0.5, 0.25])
def test_unit_sets_special_rays(offset):
    # axis-parallel, in-plane and on-grid rays: closed ranges and the ambiguity rule
    g2 = Geometry("par2d", 12, 10, angles=[0.0, pi / 2, pi, 3 * pi / 2, pi / 4, 3 * pi / 4, 0.3, 2.0],
                  n_cols=31, du=0.5, u0=offset)
    g3 = Geometry("par3d", 10, 8, 6, angles=SPECIAL_3D, n_cols=19, n_rows=15, du=0.5, dv=0.5, u0=offset,
                  v0=-offset)
    for g in (g2, g3):
        P = _proj(g)
        rays = np.arange(g.n_rays)
        rows_gpu = P.ray_units(rays)
        rows_ref = [O.ray_units(g, int(r)) for r in rays]
        # rays through grid vertices touch units at a point: such zero-length touches may
        # come out as grazing lengths on one side; every other unit matches exactly
        graze = H.check_unit_sets(g, rows_gpu, rows_ref)
        assert graze <= 0.01 * sum(len(r[0]) for r in rows_ref)
        # axis-parallel rays (closed ranges + the ambiguity rule) match exactly
        dirs = np.asarray(g.angles).reshape(g.n_views, -1)
        for q, r in enumerate(rays):
            v = r // (g.n_rows * g.n_cols)
            if np.all(np.isclose(np.mod(dirs[v], pi / 2), 0.0) | np.isclose(np.mod(dirs[v], pi / 2), pi / 2)):
                np.testing.assert_array_equal(np.sort(rows_gpu[q][0]), rows_ref[q][0])


@pytest.mark.parametrize("kind", ["rays2d", "rays3d"])
def test_ray_list_forward_adjoint_dot(kind):
    # random ray lists (Section 4.3): forward and scatter adjoint vs the oracle, dot test
    rng = np.random.default_rng(31)
    if kind == "rays2d":
        g0 = Geometry("rays2d", 48, 40, dx=0.9, dy=1.1, cx=0.5, cy=-0.3, angles=np.zeros((1, 2)))
        half = 0.5 * math.hypot(48 * 0.9, 40 * 1.1)
        ang = np.stack([rng.uniform(-half, half, 20000), rng.uniform(0, 2 * pi, 20000)], axis=1)
    else:
        g0 = Geometry("rays3d", 24, 20, 16, dx=0.9, dy=1.1, dz=1.0, cx=0.5, cy=-0.3, cz=0.2, angles=np.zeros((1, 4)))
        half = 0.5 * math.sqrt((24 * 0.9) ** 2 + (20 * 1.1) ** 2 + 16 ** 2)
        ang = np.stack([rng.uniform(-half, half, 20000), rng.uniform(-half, half, 20000),
                        rng.uniform(0, 2 * pi, 20000), rng.uniform(-pi / 2, pi / 2, 20000)], axis=1)
    g = Geometry(kind, g0.nx, g0.ny, g0.nz, dx=g0.dx, dy=g0.dy, dz=g0.dz, cx=g0.cx, cy=g0.cy, cz=g0.cz, angles=ang)
    P = _proj(g)
    f = _phantom(g, 17)
    y = P.forward(f.cuda()).cpu().numpy().reshape(-1)
    f64 = f.numpy().astype(np.float64).reshape(-1)
    H.check_rays(g, y, O.forward(g, f64), O.forward(g, np.abs(f64)), float(np.abs(f64).max()), kind)
    yin = rng.random(g.n_rays).astype(np.float32)
    z = P.adjoint(torch.from_numpy(yin.reshape(g.sino_shape())).cuda()).cpu().numpy().reshape(-1)
    H.check_adjoint(z, O.adjoint(g, yin.astype(np.float64)), kind)
    with pytest.raises(Exception):
        P.adjoint(torch.from_numpy(yin.reshape(g.sino_shape())).cuda(), method=2)  # no detector to gather over
    x = torch.from_numpy(rng.random(g.image_shape(), dtype=np.float32)).cuda()
    yv = torch.from_numpy(yin.reshape(g.sino_shape())).cuda()
    lhs = float((P.forward(x).double() * yv.double()).sum())
    rhs = float((x.double() * P.adjoint(yv).double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_ray_list_of_cone_parameters_reproduces_the_cone():
    g = H.cone_small(32, 12)
    params = np.stack([O.ray_params(g, r) for r in range(g.n_rays)])
    gl = Geometry("rays3d", g.nx, g.ny, g.nz, dx=g.dx, dy=g.dy, dz=g.dz, cx=g.cx, cy=g.cy, cz=g.cz, angles=params)
    f = _phantom(g, 5).cuda()
    yc = _proj(g).forward(f).reshape(-1)
    yl = _proj(gl).forward(f).reshape(-1)
    assert float((yc - yl).abs().max()) <= 1e-5 * float(yc.abs().max())


def test_ambiguity_examples_on_gpu():
    # Section 4.1 examples through the CUDA path
    cases = [
        (Geometry("par2d", 5, 5, angles=[0.0], n_cols=1, u0=1.5), 5 + np.arange(5)),
        (Geometry("par3d", 4, 4, 4, angles=[[0.0, 0.0]], u0=1.0, v0=1.0), 20 + np.arange(4)),
        (Geometry("par3d", 3, 3, 3, angles=[[0.0, pi / 4]], u0=-0.5, v0=math.sqrt(2)), np.array([6])),
    ]
    for g, want in cases:
        (idx, ln), = _proj(g).ray_units([0])
        np.testing.assert_array_equal(np.sort(idx), want)


@pytest.mark.parametrize("name,geom", [
    ("ts1", Geometry("par2d", 3, 3, angles=[pi / 4], n_cols=1, u0=1.0)),
    ("ts2", Geometry("fan2d_arc", 4, 4, angles=[pi / 2], n_cols=1, u0=-pi / 6, sod=4.0, sdd=4.0)),
    ("ts3", Geometry("par3d", 3, 3, 3, angles=[[pi / 4, pi / 4]])),
    ("ts4", Geometry("cone_arc", 4, 4, 4, angles=[pi / 4], u0=pi / 12, v0=pi / 12, sod=4.0, sdd=4.0)),
    ("ts5", Geometry("helix_arc", 4, 4, 4, angles=[pi / 4], src_z=[0.5], u0=pi / 12, v0=pi / 12, sod=4.0,
                     sdd=4.0)),
])
def test_paper_test_suites_on_gpu(name, geom):
    (idx, ln), = _proj(geom).ray_units([0])
    o = np.argsort(idx)
    ref_i, ref_l = O.ray_units(geom, 0)
    np.testing.assert_array_equal(idx[o], ref_i)
    np.testing.assert_allclose(ln[o], ref_l, rtol=0, atol=2e-6)


# ---------------------------------------------------------------------------------------
# Forward / adjoint on reduced configurations (every ray, every unit)
# ---------------------------------------------------------------------------------------

SMALL = {
    "par2d_64": lambda: inputs.par2d_64(),
    "fan2d_128": lambda: H.fan2d_small(),
    "par3d_32_tilt": lambda: H.par3d_small(),
    "cone_64": lambda: H.cone_small(),
    "helix_64x32": lambda: H.helix_small(),
}


@pytest.mark.parametrize("name", list(SMALL))
def test_forward_small(name):
    g = SMALL[name]()
    batch = 3
    f = torch.stack([_phantom(g, 10 + b) for b in range(batch)])
    P = _proj(g)
    y = P.forward(f.cuda()).cpu().numpy().reshape(batch, -1)
    f64 = f.numpy().astype(np.float64).reshape(batch, -1)
    y_ref = O.forward(g, f64)
    scale = O.forward(g, np.abs(f64))
    for b in range(batch):
        H.check_rays(g, y[b], y_ref[b], scale[b], float(np.abs(f64[b]).max()), f"{name}[{b}]")


@pytest.mark.parametrize("name", list(SMALL))
def test_adjoint_small(name):
    g = SMALL[name]()
    f = _phantom(g, 21).numpy().astype(np.float64)
    y = O.forward(g, f).astype(np.float32)  # the same float32 sinogram feeds both sides
    P = _proj(g)
    methods = [1, 2]
    z_ref = O.adjoint(g, y.astype(np.float64))
    for m in methods:
        z = P.adjoint(torch.from_numpy(y.reshape(g.sino_shape())).cuda(), method=m).cpu().numpy()
        H.check_adjoint(z, z_ref, f"{name} method {m}")


@pytest.mark.parametrize("name", list(SMALL))
def test_dot_product(name):
    g = SMALL[name]()
    rng = np.random.default_rng(5)
    P = _proj(g)
    x = torch.from_numpy(rng.random(g.image_shape(), dtype=np.float32)).cuda()
    yv = torch.from_numpy(rng.random(g.sino_shape(), dtype=np.float32)).cuda()
    ax = P.forward(x).double()
    aty = P.adjoint(yv).double()
    lhs = float((ax * yv.double()).sum())
    rhs = float((x.double() * aty).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_batch_chunks_bitwise_identical():
    # one-thread-per-ray kernels: the chunk of images walked together changes nothing
    g = H.fan2d_small(96, 60)
    f = torch.stack([_phantom(g, 30 + b) for b in range(5)]).cuda()
    P = _proj(g)
    P.auto_reserve = False
    outs = []
    for chunk in (1, 2, 4, 8):
        P.set_tuning(batch_chunk=chunk)
        outs.append(P.forward(f).cpu())
    for o in outs[1:]:
        assert torch.equal(o, outs[0])


@pytest.mark.parametrize("path", ["tiled", "interleaved"])
@pytest.mark.parametrize("name", ["par2d_64", "fan2d_128"])
@pytest.mark.parametrize("batch", [4, 5, 16, 20])
def test_batched_fast_path(name, batch, path):
    # batched paths: shared-memory tiles, or interleaved images with 4 lanes per ray;
    # forward, scatter and gather adjoints vs the oracle
    from paper_2006_00686_gb300.xray import XR_PATH_INTERLEAVED, XR_PATH_TILED
    g = SMALL[name]()
    f = torch.stack([_phantom(g, 70 + b) for b in range(batch)])
    P = _proj(g)
    P.set_tuning(path=XR_PATH_TILED if path == "tiled" else XR_PATH_INTERLEAVED)
    P.reserve(batch)
    y = P.forward(f.cuda())
    f64 = f.numpy().astype(np.float64).reshape(batch, -1)
    y_ref = O.forward(g, f64)
    scale = O.forward(g, np.abs(f64))
    yh = y.cpu().numpy().reshape(batch, -1)
    for b in range(batch):
        H.check_rays(g, yh[b], y_ref[b], scale[b], float(np.abs(f64[b]).max()), f"{name}[{b}] fast")
    yin = torch.from_numpy(y_ref.astype(np.float32).reshape(g.sino_shape(batch))).cuda()
    z_ref = O.adjoint(g, y_ref.astype(np.float32).astype(np.float64))
    for method, what in ((2, "gather"), (1, "scatter")):
        z = P.adjoint(yin, method=method).cpu().numpy().reshape(batch, -1)
        for b in range(batch):
            H.check_adjoint(z[b], z_ref[b], f"{name}[{b}] fast {what}")
    # the one-thread-per-ray kernels agree with the fast path
    P.set_tuning(batch_chunk=1)
    y1 = P.forward(f.cuda())
    assert float((y1 - y).abs().max()) <= 1e-5 * float(y.abs().max())


@pytest.mark.parametrize("name,order", [("par3d_32_tilt", 0), ("cone_64", 0), ("helix_64x32", 0),
                                        ("cone_64", 3), ("helix_64x32", 3), ("cone_64", 4), ("helix_64x32", 4)])
def test_fast3d_matches_ray_path(name, order):
    # the 3D fast path (reads a y-fastest copy for x-leaning rays) and the one-thread-per-ray
    # kernels on the caller's layout walk the same voxels in the same order: bitwise equal
    # forwards, adjoints equal up to the order of the atomic additions; a forward after an
    # adjoint (both use the workspace) is unchanged
    from paper_2006_00686_gb300.xray import XR_PATH_RAY
    # order 3 (XR_ORDER_COLUMN): threads over (view, col, row) on a z-fastest copy; order 4
    # (XR_ORDER_ROWBLOCK): the same in blocks of 32 rows (helix_64x32 has 16 rows: a partial
    # block)
    g = SMALL[name]()
    x = torch.stack([_phantom(g, 40 + b) for b in range(2)]).cuda()
    Pf, Pr = _proj(g), _proj(g)
    Pf.set_tuning(order=order)
    Pr.set_tuning(path=XR_PATH_RAY)
    yf, yr = Pf.forward(x), Pr.forward(x)
    if Pf.column_batch or (order == 0 and Pf.trace_walk):
        # the single-tilt-axis scan runs as 2D column problems, and the automatic order takes
        # the column-trace walk of cone and helical scans: the same lengths by other
        # arithmetic (the slab walk; lengths in horizontal distance times sec)
        assert Pf.reserved >= 1 and float((yf - yr).abs().max()) <= 1e-5 * float(yr.abs().max())
    else:
        assert Pf.reserved >= 1 and torch.equal(yf, yr)
    zf, zr = Pf.adjoint(yf, method=1), Pr.adjoint(yf, method=1)
    assert float((zf - zr).abs().max()) <= 1e-5 * float(zr.abs().max())
    # the tile-driven gather sums the same (ray, voxel) lengths
    zg = Pf.adjoint(yf, method=2)
    assert float((zg - zr).abs().max()) <= 1e-5 * float(zr.abs().max())
    assert torch.equal(Pf.forward(x), yf)


def _tilt_geoms():
    # the reduced single-tilt-axis scan; anisotropic off-centre voxels seen from phi_1 = pi
    # with fewer, wider columns than slices (some slices get no column), a detector offset
    # and one row in the middle of a slab
    g1 = H.par3d_small(32)
    v = np.arange(24, dtype=np.float64)
    ang = np.stack([np.full(24, pi), np.radians(-60.0 + 5.0 * v)], axis=1)
    g2 = Geometry("par3d", 26, 24, 20, dx=0.9, dy=1.1, dz=1.2, cx=1.5, cy=-0.7, cz=0.4, angles=ang,
                  n_cols=18, n_rows=21, du=1.3, dv=1.1, u0=0.37, v0=0.2)
    return g1, g2


@pytest.mark.parametrize("which", [0, 1])
def test_column_batch_matches_3d_walk(which):
    # a single-tilt-axis parallel scan (every ray in the y-plane of its column, Section 3.2
    # Case 2) runs as a batch of 2D column problems on the 2D kernels; forward and gather
    # adjoint against the 3D walk on the caller's layout and against the oracle, two volumes
    from paper_2006_00686_gb300.xray import XR_ADJ_GATHER, XR_ADJ_SCATTER, XR_PATH_RAY
    g = _tilt_geoms()[which]
    Pc, Pr = _proj(g), _proj(g)
    assert Pc.column_batch
    Pr.set_tuning(path=XR_PATH_RAY)
    f = torch.stack([_phantom(g, 60 + b) for b in range(2)])
    yc, yr = Pc.forward(f.cuda()), Pr.forward(f.cuda())
    assert float((yc - yr).abs().max()) <= 1e-5 * float(yr.abs().max())
    f64 = f.numpy().astype(np.float64).reshape(2, -1)
    y_ref = O.forward(g, f64)
    scale = O.forward(g, np.abs(f64))
    yh = yc.cpu().numpy().reshape(2, -1)
    for b in range(2):
        H.check_rays(g, yh[b], y_ref[b], scale[b], float(np.abs(f64[b]).max()), f"column batch [{b}]")
    rng = np.random.default_rng(which)
    y = torch.from_numpy(rng.uniform(0.0, 1.0, g.sino_shape(2)).astype(np.float32)).cuda()
    zc = Pc.adjoint(y, method=XR_ADJ_GATHER)
    zs = Pr.adjoint(y, method=XR_ADJ_SCATTER)
    assert float((zc - zs).abs().max()) <= 1e-5 * float(zs.abs().max())
    z_ref = O.adjoint(g, y.cpu().numpy().astype(np.float64).reshape(2, -1))
    zh = zc.cpu().numpy().reshape(2, -1)
    for b in range(2):
        H.check_adjoint(zh[b], z_ref[b], f"column batch adjoint [{b}]")
    # the automatic adjoint of the column batch is the gather: the same sums
    assert torch.equal(Pc.adjoint(y), zc)
    Pc.close()
    Pr.close()


def test_column_batch_only_for_single_tilt_axis():
    g = H.par3d_small(32)
    ang = np.array(g.angles, copy=True)
    ang[3, 0] = 0.2  # one view off the tilt axis: the rays leave their column planes
    assert not _proj(Geometry("par3d", 32, 32, 32, angles=ang, n_cols=32, n_rows=32)).column_batch
    # columns half a slice apart: two columns share a slice
    assert not _proj(Geometry("par3d", 32, 32, 32, angles=g.angles, n_cols=64, n_rows=32, du=0.5)).column_batch
    # columns on slice boundaries (integer y): a tie the kernels would have to break alike
    assert not _proj(Geometry("par3d", 32, 32, 32, angles=g.angles, n_cols=31, n_rows=32)).column_batch
    assert _proj(g).column_batch


def test_gather_matches_scatter_2d():
    for g in (inputs.par2d_64(), H.fan2d_small(128, 90)):
        P = _proj(g)
        y = P.forward(_phantom(g, 3).cuda())
        zs = P.adjoint(y, method=1).cpu().numpy().astype(np.float64)
        zg = P.adjoint(y, method=2).cpu().numpy().astype(np.float64)
        assert np.abs(zs - zg).max() <= 1e-5 * np.abs(zs).max()


def _odd_geom(kind, views=48):
    # an odd number of columns (the last pixel of each row alone in its thread), anisotropic
    # off-centre pixels, a detector offset.  The parallel scan has axis-parallel views; its
    # offset keeps every ray at least 0.04 from a grid line, so the oracle and the kernel
    # cannot break a tie (the bigger-index rule) differently through rounding.
    v = np.arange(views, dtype=np.float64)
    kw = dict(nx=101, ny=75, dx=0.9, dy=1.1, cx=3.0, cy=-2.0)
    if kind == "par2d":
        return Geometry(kind, angles=pi * v / 48, n_cols=170, du=0.8, u0=0.31, **kw)
    if kind == "fan2d":
        return Geometry(kind, angles=2 * pi * v / 48, n_cols=200, du=1.0, u0=0.7, sod=200.0, sdd=320.0, **kw)
    return Geometry(kind, angles=2 * pi * v / 48, n_cols=200, du=0.0032, u0=0.001, sod=200.0, sdd=320.0, **kw)


@pytest.mark.parametrize("kind,batch,views", [(k, b, 48) for k in ("par2d", "fan2d", "fan2d_arc")
                                               for b in (4, 8, 13)] + [("fan2d", 16, v) for v in (1, 2, 3)])
def test_gather_odd_width_against_oracle(kind, batch, views):
    # the 2D gather (two pixels per thread, one, two or four planes of images; the views split
    # into 8 chunks per CTA here, fewer for scans of 1-3 views) on an image of odd width,
    # against the oracle's adjoint and the scatter
    from paper_2006_00686_gb300.xray import XR_ADJ_GATHER, XR_ADJ_SCATTER
    g = _odd_geom(kind, views)
    P = _proj(g)
    P.reserve(batch)
    P.set_tuning(batch_chunk=16 if batch > 8 else batch)
    rng = np.random.default_rng(batch)
    y = torch.from_numpy(rng.uniform(0.0, 1.0, g.sino_shape(batch)).astype(np.float32)).cuda()
    zg = P.adjoint(y, method=XR_ADJ_GATHER)
    zs = P.adjoint(y, method=XR_ADJ_SCATTER)
    z_ref = O.adjoint(g, y.cpu().numpy().astype(np.float64).reshape(batch, -1))
    zh, zsh = zg.cpu().numpy().reshape(batch, -1), zs.cpu().numpy().reshape(batch, -1)
    for b in range(batch):
        H.check_adjoint(zh[b], z_ref[b], f"{kind}[{b}] gather")
        H.check_adjoint(zsh[b], z_ref[b], f"{kind}[{b}] scatter")
    P.close()


def test_rays_that_miss_the_image_are_zero():
    g = Geometry("par2d", 16, 16, angles=[0.0, 0.7], n_cols=64, du=1.0)  # s up to +-31.5
    P = _proj(g)
    y = P.forward(torch.ones(g.image_shape()).cuda()).cpu().numpy()
    s = (np.arange(64) - 31.5)
    assert np.all(y[0][np.abs(s) > 8] == 0.0)
    assert np.all(y[1][np.abs(s) > 8 * math.sqrt(2)] == 0.0)


def test_status_codes_on_gpu():
    from paper_2006_00686_gb300.xray import XRayError
    g = inputs.par2d_64()
    P = _proj(g)
    x = torch.zeros(g.image_shape(), device="cuda")
    with pytest.raises(XRayError, match="aligned"):
        buf = torch.zeros(g.n_units + 1, device="cuda")
        P.forward(buf[1:].view(g.image_shape()))
    with pytest.raises(XRayError):
        P.forward(x.double())
    from paper_2006_00686_gb300 import xray as X
    import ctypes
    assert X.lib().xr_project(P.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), 0,
                              None) == 8


# ---------------------------------------------------------------------------------------
# The five configurations at full size
# ---------------------------------------------------------------------------------------

FULL = {
    "par2d_64": (inputs.par2d_64, 1, 10, 1),
    "fan2d_512x16": (inputs.fan2d_512, inputs.FAN2D_BATCH, 10, 2),
    "par3d_256_tilt": (inputs.par3d_256_tilt, 1, 30, 3),
    "cone_512": (inputs.cone_512, 1, 30, 4),
    "helix_512x256": (inputs.helix_512x256, 1, 30, 5),
}


@pytest.mark.parametrize("name", list(FULL))
def test_full_size_forward_sampled(name):
    make, batch, n_shapes, seed = FULL[name]
    g = make()
    f = torch.stack([inputs.phantom(g, n_shapes, seed * 100 + b, device="cuda") for b in range(batch)])
    P = _proj(g)
    y = P.forward(f if batch > 1 else f[0])
    rays = H.sample_rays(g, 400 if g.is3d else 1500, seed=seed)
    y_s = y.reshape(batch, -1)[:, torch.from_numpy(rays).cuda()].cpu().numpy()
    f64 = f.cpu().numpy().astype(np.float64).reshape(batch, -1)
    del y
    for b in range(batch):
        y_ref = O.forward(g, f64[b], rays=rays)
        scale = O.forward(g, np.abs(f64[b]), rays=rays)
        H.check_rays(g, y_s[b], y_ref, scale, float(np.abs(f64[b]).max()), f"{name}[{b}]")
    P.close()


VIEW_SUBSET = {"par2d_64": 90, "fan2d_512x16": 8, "par3d_256_tilt": 6, "cone_512": 2, "helix_512x256": 6}


@pytest.mark.parametrize("name", list(FULL))
def test_full_size_adjoint_view_subset(name):
    make, _, n_shapes, seed = FULL[name]
    g0 = make()
    views = np.linspace(0, g0.n_views - 1, VIEW_SUBSET[name]).round().astype(np.int64)
    g = g0.subset_views(views)
    rng = np.random.default_rng(seed)
    y = rng.random(g.sino_shape(), dtype=np.float32)
    P = _proj(g)
    z = P.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    z_ref = O.adjoint(g, y.astype(np.float64).reshape(-1))
    H.check_adjoint(z, z_ref, name)
    for m in (1, 2):
        z2 = P.adjoint(torch.from_numpy(y).cuda(), method=m).cpu().numpy()
        H.check_adjoint(z2, z_ref, f"{name} method {m}")
    P.close()


def test_bench_configuration_full_size_fan_x16():
    # the benchmark's own launch configuration (16 images, quad planes, gather adjoint) at
    # full size, every ray and every pixel against the oracle
    g = inputs.fan2d_512()
    P = _proj(g)
    f = inputs.phantom_batch(g, 16, 10, 200)
    y = P.forward(f.cuda())
    z = P.adjoint(y)
    assert P.tuning()["path"] == 2 and P.reserved >= 16
    f64 = f.numpy().astype(np.float64).reshape(16, -1)
    y_ref = O.forward(g, f64)
    scale = O.forward(g, np.abs(f64))
    yh = y.cpu().numpy().reshape(16, -1)
    for b in range(16):
        H.check_rays(g, yh[b], y_ref[b], scale[b], float(np.abs(f64[b]).max()), f"fan x16 [{b}]")
    z_ref = O.adjoint(g, yh.astype(np.float64))
    zh = z.cpu().numpy().reshape(16, -1)
    for b in range(16):
        H.check_adjoint(zh[b], z_ref[b], f"fan x16 adjoint [{b}]")
    P.close()


@pytest.mark.parametrize("path", ["tiled", "interleaved"])
def test_calls_do_not_interfere(path):
    # a forward after an adjoint (which shares the handle's workspace) gives the same result
    from paper_2006_00686_gb300.xray import XR_PATH_INTERLEAVED, XR_PATH_TILED
    g = H.fan2d_small(128, 90)
    P = _proj(g)
    P.set_tuning(path=XR_PATH_TILED if path == "tiled" else XR_PATH_INTERLEAVED)
    x = torch.stack([_phantom(g, 90 + b) for b in range(16)]).cuda()
    y1 = P.forward(x)
    for method in (1, 2):
        P.adjoint(y1, method=method)
        y2 = P.forward(x)
        assert float((y2 - y1).abs().max()) <= 1e-6 * float(y1.abs().max())
