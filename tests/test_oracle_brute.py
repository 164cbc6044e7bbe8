"""Pins of the oracle against an independent brute force (per-unit slab clipping of a ray
built from the physical scan layout), closed forms and invariants.  CPU only."""
import math

import numpy as np
import pytest

from oracle import brute as B
from oracle import oracle as O
from paper_2006_00686_gb300.inputs import Geometry

pi = math.pi
LEN_TOL = 1e-9  # both sides are float64; lengths agree to rounding


def _dense(g, ray):
    idx, ln = O.ray_units(g, ray)
    out = np.zeros(g.n_units)
    out[idx] = ln
    assert np.all(np.diff(idx) > 0), "oracle rows must be sorted and unique"
    return out


def _check_ray(g, ray):
    p, d = B.ray_of(g, ray)
    want = B.lengths(g, p, d).reshape(-1)
    got = _dense(g, ray)
    np.testing.assert_allclose(got, want, rtol=0, atol=LEN_TOL)
    # the set of units with non-vanishing length is the same
    np.testing.assert_array_equal(got > LEN_TOL, want > LEN_TOL)
    # closed form: the lengths add up to the chord through the image box
    assert got.sum() == pytest.approx(B.box_chord(g, p, d), abs=1e-9)


def _rand_geom(kind, rng):
    three = kind in ("par3d", "cone", "cone_arc", "helix", "helix_arc")
    nx, ny = int(rng.integers(2, 9)), int(rng.integers(2, 9))
    nz = int(rng.integers(2, 7)) if three else 1
    dx, dy, dz = rng.uniform(0.5, 1.5, 3)
    cx, cy, cz = rng.uniform(-1.0, 1.0, 3)
    nv = 6
    kw = dict(nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz, cx=cx, cy=cy, cz=cz)
    if kind == "par2d":
        return Geometry(kind, angles=rng.uniform(-2 * pi, 4 * pi, nv), n_cols=9, du=rng.uniform(0.3, 1.2),
                        u0=rng.uniform(-1, 1), **kw)
    if kind == "fan2d":
        return Geometry(kind, angles=rng.uniform(0, 2 * pi, nv), n_cols=9, du=rng.uniform(0.5, 2.0),
                        u0=rng.uniform(-1, 1), sod=rng.uniform(10, 20), sdd=rng.uniform(25, 35), **kw)
    if kind == "fan2d_arc":
        return Geometry(kind, angles=rng.uniform(0, 2 * pi, nv), n_cols=9, du=rng.uniform(0.02, 0.08),
                        u0=rng.uniform(-0.05, 0.05), sod=rng.uniform(10, 20), sdd=30.0, **kw)
    if kind == "par3d":
        ang = np.stack([rng.uniform(-pi, 3 * pi, nv), rng.uniform(-pi, pi, nv)], axis=1)
        return Geometry(kind, angles=ang, n_cols=5, n_rows=4, du=rng.uniform(0.3, 1.2), dv=rng.uniform(0.3, 1.2),
                        u0=rng.uniform(-1, 1), v0=rng.uniform(-1, 1), **kw)
    helical = kind.startswith("helix")
    src_z = rng.uniform(-2, 2, nv) if helical else None
    if kind in ("cone", "helix"):
        return Geometry(kind, angles=rng.uniform(0, 2 * pi, nv), src_z=src_z, n_cols=5, n_rows=4,
                        du=rng.uniform(0.5, 2.0), dv=rng.uniform(0.5, 2.0), u0=rng.uniform(-1, 1),
                        v0=rng.uniform(-1, 1), sod=rng.uniform(10, 20), sdd=rng.uniform(25, 35), **kw)
    return Geometry(kind, angles=rng.uniform(0, 2 * pi, nv), src_z=src_z, n_cols=5, n_rows=4,
                    du=rng.uniform(0.02, 0.08), dv=rng.uniform(0.02, 0.08), u0=rng.uniform(-0.05, 0.05),
                    v0=rng.uniform(-0.05, 0.05), sod=rng.uniform(10, 20), sdd=30.0, **kw)


KINDS = ["par2d", "fan2d", "fan2d_arc", "par3d", "cone", "cone_arc", "helix", "helix_arc"]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_rays_vs_brute_force(kind, seed):
    rng = np.random.default_rng(1000 * seed + KINDS.index(kind))
    g = _rand_geom(kind, rng)
    for ray in range(g.n_rays):
        _check_ray(g, ray)


# Rays in every special position: axis-parallel (2D Case 2 and its Remark; 3D Cases 3, 4),
# in a coordinate plane (3D Case 2 and its Remark; horizontal oblique), on grid lines and
# planes (the ambiguity rule), and in every quadrant of the direction.
SPECIAL_2D = [0.0, pi / 2, pi, 3 * pi / 2, pi / 4, 3 * pi / 4, 5 * pi / 4, 0.3, 2.0, -0.7]
SPECIAL_3D = [(a, b) for a in (0.0, pi / 2, pi, 3 * pi / 2, 0.4, 2.2, 4.0, 5.5) for b in
              (0.0, pi / 2, -pi / 2, 0.3, -0.5, pi / 4)]


@pytest.mark.parametrize("offset", [0.0, 0.5, 0.37])
def test_special_rays_2d(offset):
    g = Geometry("par2d", 6, 5, dx=1.0, dy=1.0, angles=SPECIAL_2D, n_cols=15, du=0.5, u0=offset)
    for ray in range(g.n_rays):
        _check_ray(g, ray)


@pytest.mark.parametrize("offset", [0.0, 0.5, 0.23])
def test_special_rays_3d(offset):
    g = Geometry("par3d", 5, 4, 3, angles=SPECIAL_3D, n_cols=9, n_rows=7, du=0.5, dv=0.5, u0=offset,
                 v0=-offset)
    for ray in range(g.n_rays):
        _check_ray(g, ray)


def test_anisotropic_offset_special_3d():
    # dyadic spacings and offsets: on-grid rays sit exactly on the grid planes on both sides
    g = Geometry("par3d", 4, 5, 3, dx=0.75, dy=1.25, dz=0.5, cx=0.25, cy=-0.75, cz=0.25, angles=SPECIAL_3D,
                 n_cols=7, n_rows=5, du=0.625, dv=0.25, u0=0.25, v0=0.125)
    for ray in range(g.n_rays):
        _check_ray(g, ray)


def test_dense_sampling_sanity():
    rng = np.random.default_rng(7)
    for kind in ("fan2d", "cone"):
        g = _rand_geom(kind, rng)
        for ray in range(0, g.n_rays, 7):
            p, d = B.ray_of(g, ray)
            est = B.sampled_lengths(g, p, d, h=1e-3).reshape(-1)
            np.testing.assert_allclose(_dense(g, ray), est, rtol=0, atol=2.5e-3)


def test_axis_aligned_and_diagonal_closed_forms():
    n = 8
    # axis-parallel ray: every unit along the row has length d, total n*d
    g = Geometry("par2d", n, n, dx=0.7, dy=0.7, angles=[0.0, pi / 2], n_cols=1, u0=0.3)
    for ray in range(2):
        idx, ln = O.ray_units(g, ray)
        np.testing.assert_allclose(ln, 0.7)
        assert ln.sum() == pytest.approx(n * 0.7)
    # main diagonal of a square: total n*sqrt(2)*d, the n diagonal pixels have sqrt(2)*d
    g = Geometry("par2d", n, n, angles=[pi / 4], n_cols=1, u0=0.0)
    idx, ln = O.ray_units(g, 0)
    assert ln.sum() == pytest.approx(n * math.sqrt(2))
    diag = [j * n + (n - 1 - j) for j in range(n)]
    np.testing.assert_allclose(np.array(ln)[np.isin(idx, diag)], math.sqrt(2))


def test_forward_adjoint_dot_product():
    rng = np.random.default_rng(3)
    for kind in ("par2d", "fan2d", "par3d", "cone", "helix"):
        g = _rand_geom(kind, rng)
        x = rng.standard_normal(g.n_units)
        y = rng.standard_normal(g.n_rays)
        lhs = float(np.dot(O.forward(g, x, threads=2), y))
        rhs = float(np.dot(x, O.adjoint(g, y, threads=2)))
        assert lhs == pytest.approx(rhs, rel=1e-12)


def test_adjoint_matches_explicit_matrix():
    rng = np.random.default_rng(4)
    g = _rand_geom("cone", rng)
    A = np.stack([_dense(g, r) for r in range(g.n_rays)])
    y = rng.standard_normal((2, g.n_rays))
    np.testing.assert_allclose(O.adjoint(g, y, threads=2), y @ A, rtol=1e-12, atol=1e-12)
    x = rng.standard_normal((2, g.n_units))
    np.testing.assert_allclose(O.forward(g, x, threads=2), x @ A.T, rtol=1e-12, atol=1e-12)


def test_ray_subset_forward_and_adjoint():
    rng = np.random.default_rng(5)
    g = _rand_geom("fan2d", rng)
    rays = np.array([3, 0, 17, 40])
    x = rng.standard_normal(g.n_units)
    np.testing.assert_allclose(O.forward(g, x, rays=rays), O.forward(g, x)[rays], rtol=1e-15)
    y = rng.standard_normal(rays.size)
    full = np.zeros(g.n_rays)
    full[rays] = y
    np.testing.assert_allclose(O.adjoint(g, y, rays=rays), O.adjoint(g, full), rtol=1e-12, atol=1e-14)


def test_symmetry_2d_reversal():
    # Section 2.2.1: the ray (s, phi + pi) is the ray (-s, phi)
    ang = [0.3, 0.3 + pi, 1.9, 1.9 + pi, 2 * pi + 0.3]
    g = Geometry("par2d", 7, 7, angles=ang, n_cols=3, du=1.3, u0=0.0)
    x = np.random.default_rng(0).random(g.n_units)
    y = O.forward(g, x).reshape(len(ang), 3)
    np.testing.assert_allclose(y[1], y[0][::-1], rtol=1e-13)
    np.testing.assert_allclose(y[3], y[2][::-1], rtol=1e-13)
    np.testing.assert_allclose(y[4], y[0], rtol=1e-13)


def test_symmetry_3d_reversal():
    # Section 3.2.1: (-s1, s2, phi1 + pi, -phi2) == (s1, s2, phi1, phi2)
    ang = [[0.4, 0.7], [0.4 + pi, -0.7], [2.1, -0.3], [2.1 + pi, 0.3]]
    g = Geometry("par3d", 5, 4, 6, angles=ang, n_cols=5, n_rows=3, du=0.9, dv=0.8)
    x = np.random.default_rng(1).random(g.n_units)
    y = O.forward(g, x).reshape(4, 3, 5)
    np.testing.assert_allclose(y[1], y[0][:, ::-1], rtol=1e-13)
    np.testing.assert_allclose(y[3], y[2][:, ::-1], rtol=1e-13)


def test_rotation_by_quarter_turn():
    # A square image rotated by 90 degrees seen at phi + pi/2 gives the same projection
    ang = np.array([0.0, 0.2, 0.9, pi / 4])
    n = 9
    g1 = Geometry("par2d", n, n, angles=ang, n_cols=13, du=0.8)
    g2 = Geometry("par2d", n, n, angles=ang + pi / 2, n_cols=13, du=0.8)
    f = np.random.default_rng(2).random((n, n))
    np.testing.assert_allclose(O.forward(g2, np.rot90(f).copy()), O.forward(g1, f), rtol=1e-12, atol=1e-12)


def test_fan_equals_parallel_after_transform():
    # Section 2.2.2: a fan ray equals the parallel ray (s, phi) it maps to
    g = Geometry("fan2d", 10, 10, angles=[0.7, 2.9], n_cols=5, du=1.7, sod=12.0, sdd=20.0)
    x = np.random.default_rng(3).random(g.n_units)
    yf = O.forward(g, x)
    for ray in range(g.n_rays):
        s, phi = O.ray_params(g, ray)
        gp = Geometry("par2d", 10, 10, angles=[phi], n_cols=1, u0=s)
        assert O.forward(gp, x)[0] == pytest.approx(yf[ray], rel=1e-12)


def test_uniform_disc_converges_to_chord():
    # Not a parity pin: the point-sampled disc's projection tends to 2 sqrt(R^2 - s^2) as O(d)
    n, R = 200, 80.0
    c = np.arange(n) - (n - 1) / 2
    f = ((c[None, :] ** 2 + c[:, None] ** 2) <= R * R).astype(np.float64)
    s = np.array([0.0, 20.3, 50.7])
    g = Geometry("par2d", n, n, angles=[0.37], n_cols=3, du=1.0, u0=0.0)
    g.u0, g.du = 0.0, 1.0
    got = np.array([O.forward(Geometry("par2d", n, n, angles=[0.37], n_cols=1, u0=v), f)[0] for v in s])
    np.testing.assert_allclose(got, 2 * np.sqrt(R * R - s * s), atol=3.0)


def test_uniform_ball_converges_to_chord():
    # Not a parity pin either: the 3D analogue of the disc.  A point-sampled ball of radius R
    # projects, along a ray at distance rho from its centre, to 2 sqrt(R^2 - rho^2) as O(d);
    # oblique directions (phi1, phi2) and both detector offsets exercise the 3D parameters
    n, R = 72, 28.0
    c = np.arange(n) - (n - 1) / 2
    f = ((c[:, None, None] ** 2 + c[None, :, None] ** 2 + c[None, None, :] ** 2) <= R * R).astype(np.float64)
    f = f.reshape(-1)
    for phi1, phi2, s1, s2 in ((0.31, 0.47, 0.0, 0.0), (1.13, -0.62, 9.4, -7.1), (2.71, 0.05, -17.3, 12.2),
                               (0.0, 0.0, 21.6, 3.3)):
        g = Geometry("par3d", n, n, n, angles=np.array([[phi1, phi2]]), n_cols=1, n_rows=1, u0=s1, v0=s2)
        rho2 = s1 * s1 + s2 * s2
        assert O.forward(g, f)[0] == pytest.approx(2 * math.sqrt(R * R - rho2), abs=3.0)


# ---------------------------------------------------------------------------------------
# Ray lists: rays given by their own parameters (Section 4.3)
# ---------------------------------------------------------------------------------------

def _ray_list(kind, rng, n=40):
    nx, ny = int(rng.integers(2, 9)), int(rng.integers(2, 9))
    kw = dict(nx=nx, ny=ny, dx=rng.uniform(0.5, 1.5), dy=rng.uniform(0.5, 1.5), cx=rng.uniform(-1, 1),
              cy=rng.uniform(-1, 1))
    half = 0.5 * math.hypot(nx * kw["dx"], ny * kw["dy"])
    if kind == "rays2d":
        ang = np.stack([rng.uniform(-half - 1, half + 1, n), rng.uniform(-3 * pi, 3 * pi, n)], axis=1)
        return Geometry(kind, angles=ang, **kw)
    nz = int(rng.integers(2, 7))
    kw.update(nz=nz, dz=rng.uniform(0.5, 1.5), cz=rng.uniform(-1, 1))
    ang = np.stack([rng.uniform(-half - 1, half + 1, n), rng.uniform(-half - 1, half + 1, n),
                    rng.uniform(-3 * pi, 3 * pi, n), rng.uniform(-2 * pi, 2 * pi, n)], axis=1)
    return Geometry(kind, angles=ang, **kw)


@pytest.mark.parametrize("kind", ["rays2d", "rays3d"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ray_lists_vs_brute_force(kind, seed):
    g = _ray_list(kind, np.random.default_rng(100 + seed))
    for r in range(g.n_rays):
        _check_ray(g, r)


def test_ray_lists_special_rays():
    # on grid lines, axis-parallel, diagonal, every quadrant: the ambiguity rule applies
    ang2 = [[1.0, 0.0], [0.0, pi / 2], [3.0, 0.0], [-3.0, pi / 2], [0.5, pi / 4], [2.0, pi], [-1.0, 3 * pi / 2],
            [0.0, 0.0], [1.5, -pi / 2]]
    g = Geometry("rays2d", 6, 6, angles=ang2)
    for r in range(g.n_rays):
        _check_ray(g, r)
    ang3 = [[1.0, 1.0, 0.0, 0.0], [0.0, 0.0, pi / 2, 0.0], [-0.5, math.sqrt(2), 0.0, pi / 4],
            [1.0, -1.0, pi / 2, pi / 2], [0.3, 0.2, pi / 4, pi / 4], [2.0, 0.0, pi, -pi / 2]]
    g3 = Geometry("rays3d", 4, 4, 4, angles=ang3)
    for r in range(g3.n_rays):
        _check_ray(g3, r)


@pytest.mark.parametrize("scan", ["fan2d", "cone"])
def test_ray_list_of_a_scans_parameters_is_that_scan(scan):
    # the parameters of a scan's own rays, given as a list, reproduce the scan exactly
    rng = np.random.default_rng(7)
    g = _rand_geom(scan, rng)
    params = np.stack([O.ray_params(g, r) for r in range(g.n_rays)])
    gl = Geometry("rays2d" if scan == "fan2d" else "rays3d", g.nx, g.ny, g.nz, dx=g.dx, dy=g.dy, dz=g.dz,
                  cx=g.cx, cy=g.cy, cz=g.cz, angles=params)
    f = rng.random(g.n_units)
    np.testing.assert_array_equal(O.forward(gl, f), O.forward(g, f))
