"""The system matrix as the timed kernels see it, against the oracle's rows.

For a small scan, the forward of the one-hot image e_I is column I of the projection matrix,
and the adjoint of the one-hot sinogram e_r is row r.  Both are rebuilt here through the same
launch configurations the benchmark times -- the quad-plane forward and the pair gather of 2D
batches (16 images per call), the column-trace walk of cone and helical scans, the row-blocked
crossing-order walk, and the column batch of single-tilt-axis scans -- and every ray's row is
compared with the oracle's unit list (eq. conditions_2D_1 / conditions_3D_1 and the ambiguity
rule of Section 4.1): the set of units longer than the grazing threshold delta matches
exactly, matched lengths agree to delta, and a unit on one side only is at most delta long.
The grids have odd sizes, off-centre anisotropic units, axis-parallel views, a detector row
on the central plane and a central column through the rotation axis."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2006_00686_gb300.inputs import Geometry
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu
pi = math.pi

# views on the axes (traces along grid planes) and oblique ones
ANGLES = np.array([0.0, pi / 2, pi, 3 * pi / 2, 0.37, 1.91, 2.66, 4.4, 5.3])


@pytest.fixture(scope="module")
def X():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    from paper_2006_00686_gb300 import xray
    return xray


def _oracle_rows(g):
    return [O.ray_units(g, r) for r in range(g.n_rays)]


def _rows_from_dense(M):
    """M[r, I] -> [(nonzero I, values)] per ray."""
    out = []
    for r in range(M.shape[0]):
        nz = np.nonzero(M[r])[0]
        out.append((nz, M[r, nz]))
    return out


def _matrix_by_forward(P, g, batch):
    M = np.zeros((g.n_rays, g.n_units), dtype=np.float64)
    for I0 in range(0, g.n_units, batch):
        b = min(batch, g.n_units - I0)
        B = max(b, 4) if not g.is3d else b  # 2D: keep the batched quad-plane path
        E = torch.zeros((B, g.n_units), device="cuda")
        E[torch.arange(b), torch.arange(I0, I0 + b)] = 1.0
        y = P.forward(E.reshape((B,) + g.image_shape())).reshape(B, -1)
        M[:, I0:I0 + b] = y[:b].double().cpu().numpy().T
    return M


def _matrix_by_adjoint(P, g, batch, method=0):
    M = np.zeros((g.n_rays, g.n_units), dtype=np.float64)
    for r0 in range(0, g.n_rays, batch):
        b = min(batch, g.n_rays - r0)
        B = max(b, 4) if not g.is3d else b
        E = torch.zeros((B, g.n_rays), device="cuda")
        E[torch.arange(b), torch.arange(r0, r0 + b)] = 1.0
        z = P.adjoint(E.reshape((B,) + g.sino_shape()), method=method).reshape(B, -1)
        M[r0:r0 + b] = z[:b].double().cpu().numpy()
    return M


def _check(g, M, ref, what):
    graze = H.check_unit_sets(g, _rows_from_dense(M), ref)
    n = sum(len(r[0]) for r in ref)
    assert n > 200, what
    # grazing-only units: those with a length below delta on both sides, a handful at most
    assert graze <= max(4, n // 500), f"{what}: {graze} grazing differences of {n}"


def _geom2d(kind):
    kw = dict(dx=0.9, dy=1.1, cx=0.7, cy=-0.4, angles=ANGLES)
    if kind == "par2d":
        return Geometry("par2d", 23, 19, n_cols=33, du=0.8, **kw)
    if kind == "fan2d":
        return Geometry("fan2d", 23, 19, n_cols=33, du=1.3, sod=60.0, sdd=90.0, **kw)
    return Geometry("fan2d_arc", 23, 19, n_cols=33, du=0.018, sod=60.0, sdd=90.0, **kw)


@pytest.mark.parametrize("kind", ["par2d", "fan2d", "fan2d_arc"])
def test_2d_batched_forward_and_gather_rows(X, kind):
    # 16 images per call: the quad-plane forward (fwd_plane_kernel<4>) and the pair gather
    g = _geom2d(kind)
    ref = _oracle_rows(g)
    P = X.Projector(g)
    _check(g, _matrix_by_forward(P, g, 16), ref, f"{kind} forward")
    _check(g, _matrix_by_adjoint(P, g, 16, method=X.XR_ADJ_GATHER), ref, f"{kind} gather")
    _check(g, _matrix_by_adjoint(P, g, 16, method=X.XR_ADJ_SCATTER), ref, f"{kind} scatter")
    P.close()


@pytest.mark.parametrize("kind", ["par2d", "fan2d", "fan2d_arc"])
def test_single_image_2d_pair_walk_rows(X, kind):
    # one image per call on a 2D scan with 1024 rays per SM or more: the lockstep slab walk
    # on pair planes (forward and adjoint), the configuration of the plain single-image
    # launches.  The forward of every one-hot image gives the matrix's columns, kept at a
    # sample of rays (every ray of the four axis views, 1200 others); the adjoint of one-hot
    # sinograms gives the rows of 300 sampled rays
    v = np.arange(720, dtype=np.float64)
    kw = dict(dx=0.9, dy=1.1, cx=0.7, cy=-0.4, n_cols=241)
    if kind == "par2d":
        # u0: every ray of the axis views at least 0.005 from a grid line (no tie to break)
        g = Geometry(kind, 23, 19, angles=2 * pi * v / 720, du=0.13, u0=0.025, **kw)
    elif kind == "fan2d":
        g = Geometry(kind, 23, 19, angles=2 * pi * v / 720, du=0.3, sod=60.0, sdd=90.0, **kw)
    else:
        g = Geometry(kind, 23, 19, angles=2 * pi * v / 720, du=0.0035, sod=60.0, sdd=90.0, **kw)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert g.n_rays >= 1024 * sms
    rng = np.random.default_rng(11)
    axis = np.concatenate([np.arange(241) + 241 * k for k in (0, 180, 360, 540)])
    rays = np.unique(np.concatenate([axis, rng.choice(g.n_rays, 1200, replace=False)]))
    P = X.Projector(g)
    Mf = np.zeros((len(rays), g.n_units))
    rt = torch.from_numpy(rays).cuda()
    for I in range(g.n_units):
        e = torch.zeros(g.n_units, device="cuda")
        e[I] = 1.0
        Mf[:, I] = P.forward(e.reshape(g.image_shape())).reshape(-1)[rt].double().cpu().numpy()
    ref_all = {int(r): O.ray_units(g, int(r)) for r in rays}
    graze = H.check_unit_sets(g, _rows_from_dense(Mf), [ref_all[int(r)] for r in rays])
    assert graze <= max(4, sum(len(ref_all[int(r)][0]) for r in rays) // 500), graze
    sample = rng.choice(rays, 300, replace=False)
    Ma = np.zeros((len(sample), g.n_units))
    for q, r in enumerate(sample):
        y = torch.zeros(g.n_rays, device="cuda")
        y[int(r)] = 1.0
        Ma[q] = P.adjoint(y.reshape(g.sino_shape()), method=X.XR_ADJ_SCATTER).reshape(-1).double().cpu().numpy()
    graze = H.check_unit_sets(g, _rows_from_dense(Ma), [ref_all[int(r)] for r in sample])
    assert graze <= max(4, sum(len(ref_all[int(r)][0]) for r in sample) // 500), graze
    P.close()


def _geom3d(kind):
    kw = dict(dx=0.9, dy=1.1, dz=0.8, cx=0.6, cy=-0.5, cz=0.3, angles=ANGLES, n_cols=21, n_rows=15,
              sod=50.0, sdd=80.0)
    if kind in ("cone", "helix"):
        kw.update(du=1.4, dv=1.3)
    else:
        kw.update(du=0.02, dv=0.02)
    if kind.startswith("helix"):
        kw["src_z"] = np.linspace(-3.0, 3.0, len(ANGLES))
    return Geometry(kind, 17, 15, 13, **kw)


@pytest.mark.parametrize("kind", ["cone", "cone_arc", "helix", "helix_arc"])
@pytest.mark.parametrize("order", ["trace", "rowblock"])
def test_3d_cone_forward_and_scatter_rows(X, kind, order):
    g = _geom3d(kind)
    ref = _oracle_rows(g)
    P = X.Projector(g)
    P.set_tuning(order=X.XR_ORDER_TRACE if order == "trace" else X.XR_ORDER_ROWBLOCK)
    _check(g, _matrix_by_forward(P, g, 64), ref, f"{kind} {order} forward")
    _check(g, _matrix_by_adjoint(P, g, 64, method=X.XR_ADJ_SCATTER), ref, f"{kind} {order} scatter")
    P.close()


def test_single_tilt_axis_column_batch_rows(X):
    # phi_1 = 0: the scan runs as 2D column problems (quad-plane forward, pair gather)
    phi2 = np.deg2rad(np.array([-60.0, -30.0, 0.0, 20.0, 45.0, 60.0]))
    g = Geometry("par3d", 15, 13, 11, dx=0.9, dy=1.1, dz=0.8, cx=0.3, cy=-0.2, cz=0.1,
                 angles=np.stack([np.zeros_like(phi2), phi2], axis=1), n_cols=13, n_rows=17, du=1.1, dv=0.9)
    ref = _oracle_rows(g)
    P = X.Projector(g)
    _matrix_by_forward(P, g, 1)  # reserves the workspace
    assert P.column_batch
    _check(g, _matrix_by_forward(P, g, 64), ref, "column batch forward")
    _check(g, _matrix_by_adjoint(P, g, 64, method=X.XR_ADJ_GATHER), ref, "column batch gather")
    P.close()


def test_uneven_2d_batch_plan_rows(X):
    # a persistent plan of three fans of different sizes (the lockstep slab walk of 2D work
    # lists): column I of every problem's matrix from one-hot images, row r from one-hot
    # sinograms, all problems in one launch per basis vector
    geoms = [Geometry("fan2d", n, n + 2, dx=0.9, dy=1.1, cx=0.3, cy=-0.2, angles=ANGLES, n_cols=c, du=1.2,
                      sod=60.0, sdd=90.0) for n, c in ((13, 21), (19, 29), (9, 17))]
    Ps = [X.Projector(g) for g in geoms]
    imgs = [torch.zeros(g.image_shape(), device="cuda") for g in geoms]
    sinos = [torch.zeros(g.sino_shape(), device="cuda") for g in geoms]
    fwd, adj = X.BatchPlan(Ps, imgs, sinos, tile=64), X.BatchPlan(Ps, imgs, sinos, tile=64)
    Mf = [np.zeros((g.n_rays, g.n_units)) for g in geoms]
    Ma = [np.zeros((g.n_rays, g.n_units)) for g in geoms]
    for I in range(max(g.n_units for g in geoms)):
        for g, x in zip(geoms, imgs):
            x.zero_()
            if I < g.n_units:
                x.view(-1)[I] = 1.0
        fwd.project()
        for q, (g, y) in enumerate(zip(geoms, sinos)):
            if I < g.n_units:
                Mf[q][:, I] = y.double().cpu().numpy().reshape(-1)
    for r in range(max(g.n_rays for g in geoms)):
        for g, y in zip(geoms, sinos):
            y.zero_()
            if r < g.n_rays:
                y.view(-1)[r] = 1.0
        adj.backproject()
        for q, (g, x) in enumerate(zip(geoms, imgs)):
            if r < g.n_rays:
                Ma[q][r] = x.double().cpu().numpy().reshape(-1)
    for q, g in enumerate(geoms):
        ref = _oracle_rows(g)
        _check(g, Mf[q], ref, f"plan forward {q}")
        _check(g, Ma[q], ref, f"plan adjoint {q}")
    for P in Ps:
        P.close()


@pytest.mark.parametrize("kind", ["cone", "helix"])
def test_trace_walk_rays_on_grid_planes(X, kind):
    # even grids centred at the origin and an odd detector: at the axis-parallel views the
    # central column's vertical plane is a grid plane (x = 0 or y = 0), and the central row is
    # horizontal at a z plane (z = 0, helix: the source heights are whole voxels).  Those rays lie
    # on planes: the ambiguity rule of Section 4.1 gives them the units with the bigger index, at
    # full lengths, so the unit sets must match the oracle exactly there
    ang = np.array([0.0, pi / 2, pi, 3 * pi / 2, pi / 4, 0.9])
    kw = dict(angles=ang, n_cols=21, n_rows=15, du=1.0, dv=1.0, sod=40.0, sdd=64.0)
    if kind == "helix":
        kw["src_z"] = np.array([0.0, 1.0, -1.0, 2.0, 0.0, -2.0])
    g = Geometry(kind, 16, 16, 12, **kw)
    ref = _oracle_rows(g)
    P = X.Projector(g)
    assert P.trace_walk
    P.set_tuning(order=X.XR_ORDER_TRACE)
    Mf = _matrix_by_forward(P, g, 64)
    Ma = _matrix_by_adjoint(P, g, 64, method=X.XR_ADJ_SCATTER)
    # every unit longer than delta matches exactly; with integer detector offsets many rays also
    # pass through grid edges and vertices, whose zero-length touches may show on one side as
    # lengths below delta (so no cap on their number here)
    H.check_unit_sets(g, _rows_from_dense(Mf), ref)
    H.check_unit_sets(g, _rows_from_dense(Ma), ref)
    # the central column at the axis-parallel views (traces on a grid plane), every row, and the
    # central row there (on a z plane too): the oracle's units, none missing, full lengths
    delta = H.grazing_delta(g)
    views = g.n_rows * g.n_cols
    for v in range(4):
        for row in range(g.n_rows):
            r = v * views + row * g.n_cols + g.n_cols // 2
            i_ref, l_ref = ref[r]
            assert len(i_ref) > 0
            for M in (Mf, Ma):
                np.testing.assert_array_equal(np.nonzero(M[r] > delta)[0], i_ref[l_ref > delta])
    r_axis = g.n_rows // 2 * g.n_cols + g.n_cols // 2  # view 0, central row and column
    assert np.allclose(ref[r_axis][1], 1.0)  # on two planes: a run of whole voxels
    P.close()
