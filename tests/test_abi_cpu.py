"""The C-ABI library loads and exports every function include/xray.h declares; host-side
validation returns the documented status codes.  No compute call needs a GPU here."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "xray.h")


@pytest.fixture(scope="module")
def X():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2006_00686_gb300 import xray
    return xray


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(xr_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_api():
    names = declared_functions()
    for must in ("xr_geometry_create", "xr_project", "xr_backproject", "xr_ray_units", "xr_batch_project"):
        assert must in names


def test_library_exports_every_declared_symbol(X):
    L = X.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_header(X):
    assert sorted(X.SIGNATURES) == declared_functions()


def test_status_strings(X):
    for code in range(0, 12):
        s = X.lib().xr_status_string(code).decode()
        assert s and s != "unknown status"
    assert X.lib().xr_status_string(99).decode() == "unknown status"
    assert X.lib().xr_version() >= 1


def _desc(X, **kw):
    ang = np.linspace(0, math.pi, 4, endpoint=False)
    base = dict(kind=0, nx=8, ny=8, nz=1, dx=1.0, dy=1.0, dz=1.0, cx=0.0, cy=0.0, cz=0.0, n_views=4,
                n_rows=1, n_cols=9, du=1.0, dv=1.0, u0=0.0, v0=0.0, sod=0.0, sdd=0.0)
    base.update(kw)
    d = X._Desc()
    for k, v in base.items():
        setattr(d, k, v)
    keep = np.ascontiguousarray(ang)
    d.angles = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return d, keep


@pytest.mark.parametrize("kw,code", [
    (dict(kind=10), 3),                     # XR_ERR_KIND
    (dict(kind=-1), 3),
    (dict(kind=8, n_cols=9), 2),            # a ray list has one sample per "view"
    (dict(kind=9, nz=4, n_rows=2, n_cols=1), 2),
    (dict(nx=0), 2),                        # XR_ERR_SIZE
    (dict(n_cols=0), 2),
    (dict(nx=20000), 2),
    (dict(dx=0.0), 4),                      # XR_ERR_GEOMETRY
    (dict(du=-1.0), 4),
    (dict(kind=1, sod=3.0, sdd=10.0), 4),   # source inside the image
    (dict(kind=1, sod=100.0, sdd=0.0), 4),  # flat detector without distance
    (dict(kind=6, nz=4, n_rows=2, sod=100.0, sdd=150.0), 1),  # helix without source heights
])
def test_invalid_descriptions(X, kw, code):
    d, keep = _desc(X, **kw)
    h = ctypes.c_void_p(123)
    assert X.lib().xr_geometry_create(ctypes.byref(d), ctypes.byref(h)) == code
    assert not h.value


def test_null_arguments(X):
    L = X.lib()
    h = ctypes.c_void_p()
    assert L.xr_geometry_create(None, ctypes.byref(h)) == 1
    assert L.xr_project(None, None, None, 1, None) == 1
    assert L.xr_backproject(None, None, None, 1, None) == 1
    assert L.xr_ray_units(None, None, 1, 1, None, None, None, None) == 1
    assert L.xr_system_rows_count(None, 0, 1, None, None) == 1
    assert L.xr_system_rows_fill(None, 0, 1, None, None, None, None) == 1
    assert L.xr_batch_project(None, None) == 1
    assert L.xr_batch_ray_setup(None, None) == 1
    assert L.xr_wait_bound_selftest(1000, None) == 1
    assert L.xr_project_backproject(None, None, None, None, 1, None) == 1
    out = ctypes.c_int32(-1)
    assert L.xr_wait_bound_selftest(0, ctypes.byref(out)) == L.xr_wait_bound_selftest(-5, ctypes.byref(out)) != 0
    assert out.value == -1
    assert L.xr_batch_create(None, 1, 0, 0, ctypes.byref(h)) == 1
    L.xr_geometry_destroy(None)
    L.xr_batch_destroy(None)


def test_product_path_fails_loudly_without_gpu(X):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2006_00686_gb300.inputs import par2d_64
    with pytest.raises(X.XRayError):
        X.Projector(par2d_64())


# ---------------------------------------------------------------------------------------
# Column batch of single-tilt-axis parallel scans: the host-side plan (no GPU needed)
# ---------------------------------------------------------------------------------------

def _tilt(nx=8, ny=6, nz=5, phi1=0.0, **kw):
    from paper_2006_00686_gb300.inputs import Geometry
    phi2 = np.radians([-50.0, -10.0, 30.0, 70.0])
    ang = np.stack([np.full(4, phi1), phi2], axis=1)
    base = dict(dx=0.9, dy=1.1, dz=1.2, cx=0.3, cy=-0.2, cz=0.1, n_cols=6, n_rows=5, du=1.1, dv=0.9, u0=0.05,
                v0=0.1)
    base.update(kw)
    return Geometry("par3d", nx, ny, nz, angles=ang, **base)


def _oracle_slices(g):
    # the slice of every unit the oracle gives the central-row rays of each column (Section 3.2
    # Case 2: a ray of the column meets only the slice holding its plane); -1: no unit
    from oracle import oracle as O
    out = []
    for c in range(g.n_cols):
        js = set()
        for v in range(g.n_views):
            idx, _ = O.ray_units(g, (v * g.n_rows + g.n_rows // 2) * g.n_cols + c)
            js |= {int(I) // g.nx % g.ny for I in np.asarray(idx)}
        assert len(js) <= 1, f"column {c} meets slices {js}"
        out.append(js.pop() if js else -1)
    return np.array(out)


@pytest.mark.parametrize("phi1", [0.0, math.pi])
def test_column_batch_plan_matches_the_oracle(X, phi1):
    g = _tilt(phi1=phi1)
    ok, slice_of = X.column_batch_plan(g)
    assert ok
    np.testing.assert_array_equal(slice_of, _oracle_slices(g))
    assert len(set(slice_of[slice_of >= 0].tolist())) == (slice_of >= 0).sum()


def test_column_batch_plan_columns_outside_the_volume(X):
    g = _tilt(n_cols=9, du=1.4)  # the outer columns' planes miss the 6.6-wide volume
    ok, slice_of = X.column_batch_plan(g)
    assert ok and (slice_of == -1).any() and (slice_of >= 0).any()
    np.testing.assert_array_equal(slice_of, _oracle_slices(g))


@pytest.mark.parametrize("kw", [
    dict(du=0.5),                 # two columns per slice
    dict(du=1.1, u0=0.0, cy=0.0, ny=6, dy=1.1, n_cols=5),  # a column plane on a slice boundary (y = 0)
])
def test_column_batch_plan_refuses(X, kw):
    ok, slice_of = X.column_batch_plan(_tilt(**kw))
    assert not ok and (slice_of == -1).all()


def test_column_batch_plan_needs_one_tilt_axis(X):
    from paper_2006_00686_gb300.inputs import Geometry
    g = _tilt()
    ang = np.array(g.angles, copy=True)
    ang[2, 0] = 0.3
    assert not X.column_batch_plan(Geometry("par3d", g.nx, g.ny, g.nz, angles=ang, n_cols=6, n_rows=5))[0]
    ang[:, 0] = [0.0, math.pi, 0.0, 0.0]  # both signs of cos(phi_1): the columns swap planes
    assert not X.column_batch_plan(Geometry("par3d", g.nx, g.ny, g.nz, angles=ang, n_cols=6, n_rows=5))[0]
    cone = Geometry("cone", 8, 6, 5, angles=[0.1, 0.7], n_cols=6, n_rows=5, sod=40.0, sdd=60.0)
    assert not X.column_batch_plan(cone)[0]


def test_column_batch_plan_rejects_invalid_descriptions(X):
    from paper_2006_00686_gb300.inputs import Geometry
    with pytest.raises(X.XRayError):
        X.column_batch_plan(Geometry("par3d", 8, 6, 5, dx=0.0, angles=[[0.0, 0.2]], n_cols=6, n_rows=5))
    assert X.lib().xr_column_batch_plan(None, None, None) == 1
