"""Pins of the oracle to what the paper prints: the five test-suite tables, the hand-computed
intermediates, the closed-form lengths, the ambiguity examples and the stated identities."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2006_00686_gb300.inputs import Geometry

pi = math.pi
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
r2, r3 = math.sqrt(2.0), math.sqrt(3.0)
tan12, sin12, cos12 = math.tan(pi / 12), math.sin(pi / 12), math.cos(pi / 12)


def _table(name):
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, name)) if ln.strip() and not ln.startswith("#")]
    return np.array([int(r[0]) for r in rows]), np.array([float(r[1]) for r in rows])


# The paper prints float output to six significant digits (Section 5, first paragraph).
PRINT_TOL = 5e-6

TS1 = Geometry("par2d", 3, 3, angles=[pi / 4], n_cols=1, u0=1.0)
TS2 = Geometry("fan2d_arc", 4, 4, angles=[pi / 2], n_cols=1, u0=-pi / 6, sod=4.0, sdd=4.0)
TS3 = Geometry("par3d", 3, 3, 3, angles=[[pi / 4, pi / 4]])
TS4 = Geometry("cone_arc", 4, 4, 4, angles=[pi / 4], u0=pi / 12, v0=pi / 12, sod=4.0, sdd=4.0)
TS5 = Geometry("helix_arc", 4, 4, 4, angles=[pi / 4], src_z=[0.5], u0=pi / 12, v0=pi / 12, sod=4.0, sdd=4.0)


@pytest.mark.parametrize("geom,table", [
    (TS1, "ts1_par2d.txt"),
    (TS2, "ts2_fan_equiangular.txt"),
    (TS3, "ts3_par3d.txt"),
    (TS4, "ts4_cone_equiangular.txt"),
    (TS5, "ts5_helix_equiangular.txt"),
])
def test_paper_tables(geom, table):
    want_i, want_l = _table(table)
    idx, ln = O.ray_units(geom, 0)
    np.testing.assert_array_equal(idx, want_i)
    np.testing.assert_allclose(ln, want_l, rtol=0, atol=PRINT_TOL)


def test_ts1_geometric_lengths():
    # Section 5.1: lengths 2 - sqrt2, 2sqrt2 - 2, 2sqrt2 - 2 for pixels (0,0), (0,1), (1,0)
    idx, ln = O.ray_units(TS1, 0)
    np.testing.assert_allclose(ln, [2 - r2, 2 * r2 - 2, 2 * r2 - 2], rtol=1e-14)


def test_ts2_params_and_lengths():
    # Section 5.2: (s, phi) = (-2, -pi/6), i.e. the ray (2, 5pi/6); lengths 2sqrt3/3, 4 - 2sqrt3
    s, phi = O.ray_params(TS2, 0)
    assert s == pytest.approx(2.0, abs=1e-14) and phi == pytest.approx(5 * pi / 6, abs=1e-14)
    idx, ln = O.ray_units(TS2, 0)
    np.testing.assert_allclose(ln, [2 * r3 / 3, 4 - 2 * r3], rtol=1e-14)


def test_ts3_geometric_lengths():
    idx, ln = O.ray_units(TS3, 0)
    np.testing.assert_allclose(ln, [1.5 * r2 - 1, 1 - r2 / 2, r2, 1 - r2 / 2, 1.5 * r2 - 1], rtol=1e-14)


def test_ts4_params_and_closed_forms():
    # Section 5.4: phi1 = pi/3, phi2 = pi/12, s1 = 4 sin(pi/12), s2 = 4 sin(pi/12) cos(pi/12)
    s1, s2, p1, p2 = O.ray_params(TS4, 0)
    np.testing.assert_allclose([s1, s2, p1, p2], [4 * sin12, 4 * sin12 * cos12, pi / 3, pi / 12], rtol=1e-14)
    q = (4 - r2) * tan12 * math.sin(5 * pi / 12) / math.sin(pi / 3)
    closed = {
        28: 2 * (1 - q) / cos12,  # voxel (1,3,0)
        24: 2 * r3 / (3 * cos12),  # voxel (1,2,0)
        20: 2 * (q - r3 / 3) / cos12,  # voxel (1,1,0)
        1: 2 * r3 / (3 * cos12),  # voxel (0,0,1)
        21: (1 - (4 * r2 - 2) * tan12) / sin12,  # voxel (1,1,1)
        5: (((4 - r2) * (r2 - 2 * tan12 * math.sin(5 * pi / 12) / math.sin(pi / 3)) + 4 * r3 / 3) * tan12 - 1)
        / sin12,  # voxel (0,1,1)
    }
    idx, ln = O.ray_units(TS4, 0)
    got = dict(zip(idx.tolist(), ln.tolist()))
    assert set(got) == set(closed)
    for k, v in closed.items():
        assert got[k] == pytest.approx(v, rel=1e-12), k


def test_ts5_params_and_closed_forms():
    # Section 5.5: s2 = 4 cos(pi/12) sin(pi/12) + cos(pi/12)/2.  The printed closed forms for
    # voxels (0,3,0) and (1,3,0) are attached to the opposite voxels in the table; the table
    # (and the brute force) puts A at voxel (1,3,0) = index 28 and B at (0,3,0) = index 12.
    s1, s2, p1, p2 = O.ray_params(TS5, 0)
    np.testing.assert_allclose([s1, s2], [4 * sin12, 4 * cos12 * sin12 + cos12 / 2], rtol=1e-14)
    q = (4 - r2) * tan12 * math.sin(5 * pi / 12) / math.sin(pi / 3)
    A = (0.5 - (4 * r2 - 4) * tan12) / sin12
    B = 2 * (1 - q) / cos12 - A
    closed = {
        8: 2 * r3 / (3 * cos12),  # (0,2,0)
        4: 2 * (q - r3 / 3) / cos12,  # (0,1,0)
        1: 2 * r3 / (3 * cos12),  # (0,0,1)
        5: (2 - (8 - 2 * r2) * tan12 * math.sin(5 * pi / 12)) / (math.cos(pi / 6) * cos12),  # (0,1,1)
        28: A,
        12: B,
    }
    idx, ln = O.ray_units(TS5, 0)
    got = dict(zip(idx.tolist(), ln.tolist()))
    assert set(got) == set(closed)
    for k, v in closed.items():
        assert got[k] == pytest.approx(v, rel=1e-12), k


def test_helix_h0_equals_circular_cone():
    # Section 5.5: with H = 0 the helical output equals the circular cone output
    g = Geometry("helix_arc", 4, 4, 4, angles=[pi / 4], src_z=[0.0], u0=pi / 12, v0=pi / 12, sod=4.0, sdd=4.0)
    a, b = O.ray_units(g, 0), O.ray_units(TS4, 0)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_in_plane_case2_reduces_to_2d():
    # Section 3.2, Case 2 (eq. condition_nonzero_t_case2_3D_1): with phi_1 = 0 a 3D parallel
    # ray lies in the plane y = s_1 and meets only the voxels of the slice holding that plane,
    # under the 2D condition in (x, z).  So the 3D transform restricted to one detector column
    # (s_1 = u) is the 2D parallel transform of that column's y-slice, with s = s_2 the row
    # coordinate and phi = phi_2; the adjoint likewise.  The oracle computes the two through
    # its separate 3D and 2D derivations.  phi_2 = 0 and pi/2 give axis-parallel rays (the
    # closed ranges of Cases 3/4 against 2D Case 2); no column or row lies on a grid plane.
    rng = np.random.default_rng(21)
    nx, ny, nz = 7, 6, 5
    dx, dy, dz, cx, cy, cz = 0.9, 1.1, 1.2, 0.4, -0.3, 0.2
    phi2 = np.radians([-57.0, -20.0, 0.0, 33.0, 61.0, 90.0])
    n_cols, n_rows, du, dv, u0, v0 = 5, 9, 1.3, 0.8, 0.21, 0.13
    g3 = Geometry("par3d", nx, ny, nz, dx=dx, dy=dy, dz=dz, cx=cx, cy=cy, cz=cz,
                  angles=np.stack([np.zeros_like(phi2), phi2], axis=1), n_cols=n_cols, n_rows=n_rows,
                  du=du, dv=dv, u0=u0, v0=v0)
    g2 = Geometry("par2d", nx, nz, dx=dx, dy=dz, cx=cx, cy=cz, angles=phi2, n_cols=n_rows, du=dv, u0=v0)
    f = rng.uniform(0.0, 1.0, (nz, ny, nx))
    sino = rng.uniform(0.0, 1.0, (len(phi2), n_rows, n_cols))
    y3 = O.forward(g3, f.reshape(-1)).reshape(len(phi2), n_rows, n_cols)
    z3 = O.adjoint(g3, sino.reshape(-1)).reshape(nz, ny, nx)
    z_expect = np.zeros((nz, ny, nx))
    for c in range(n_cols):
        y = (c - 0.5 * (n_cols - 1)) * du + u0          # the column's plane y = s_1 = u
        jh = (cy + 0.5 * ny * dy - y) / dy               # its slice coordinate (j counts down)
        assert 0.0 < jh < ny and abs(jh - round(jh)) > 0.05
        j = int(math.floor(jh))
        y2 = O.forward(g2, f[:, j, :].reshape(-1)).reshape(len(phi2), n_rows)
        np.testing.assert_allclose(y3[:, :, c], y2, rtol=1e-12, atol=1e-12)
        z_expect[:, j, :] += O.adjoint(g2, sino[:, :, c].reshape(-1)).reshape(nz, nx)
    np.testing.assert_allclose(z3, z_expect, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("cone,fan,du,u0", [("cone", "fan2d", 1.1, 0.3), ("cone_arc", "fan2d_arc", 0.02, 0.004)])
def test_cone_central_row_reduces_to_fan(cone, fan, du, u0):
    # The central row of a flat cone detector (h = 0, so beta = 0 and s_2 = 0 in eq.
    # equispaced_cone_beam) holds horizontal rays in the source plane z = 0: they meet only the
    # slice holding that plane, as the fan beam of eq. 2Dparalleltofan_2 does on the slice's
    # image.  The cone's view angle phi'_1 (source at -D(cos phi'_1, sin phi'_1, 0)) is the fan's
    # alpha - pi/2 (source at D(-sin alpha, cos alpha)); both detectors run along
    # (-sin phi'_1, cos phi'_1).  Flat (eq. equispaced_cone_beam vs 2Dparalleltofan_2) and
    # equiangular (eq. equiangular_cone_beam vs 2Dparalleltofan, du in radians) detectors;
    # forward and adjoint, through the oracle's separate 3D and 2D formulas, with anisotropic
    # off-centre voxels.
    rng = np.random.default_rng(5)
    nx, ny, nz = 9, 8, 5
    dx, dy, dz, cx, cy, cz = 0.9, 1.1, 1.3, 0.4, -0.3, 0.45
    phi = np.radians([0.0, 17.0, 100.0, 200.0, 290.0])
    sod, sdd, n_cols = 30.0, 50.0, 15
    gc = Geometry(cone, nx, ny, nz, dx=dx, dy=dy, dz=dz, cx=cx, cy=cy, cz=cz, angles=phi, n_cols=n_cols,
                  n_rows=3, du=du, dv=0.7 * du, u0=u0, v0=0.0, sod=sod, sdd=sdd)
    gf = Geometry(fan, nx, ny, dx=dx, dy=dy, cx=cx, cy=cy, angles=phi + pi / 2, n_cols=n_cols, du=du, u0=u0,
                  sod=sod, sdd=sdd)
    kh = (cz + 0.5 * nz * dz) / dz  # slice coordinate of z = 0 (k counts down)
    assert abs(kh - round(kh)) > 0.1
    k = int(math.floor(kh))
    f = rng.uniform(0.0, 1.0, (nz, ny, nx))
    yc = O.forward(gc, f.reshape(-1)).reshape(len(phi), 3, n_cols)[:, 1, :]
    yf = O.forward(gf, f[k].reshape(-1)).reshape(len(phi), n_cols)
    np.testing.assert_allclose(yc, yf, rtol=1e-12, atol=1e-12)
    sino = np.zeros((len(phi), 3, n_cols))
    sino[:, 1, :] = rng.uniform(0.0, 1.0, (len(phi), n_cols))
    zc = O.adjoint(gc, sino.reshape(-1)).reshape(nz, ny, nx)
    z_expect = np.zeros((nz, ny, nx))
    z_expect[k] = O.adjoint(gf, sino[:, 1, :].reshape(-1)).reshape(ny, nx)
    np.testing.assert_allclose(zc, z_expect, rtol=1e-12, atol=1e-12)


def test_par3d_horizontal_views_reduce_to_2d_rows():
    # Reading R5 (phi_2 = 0 with any phi_1, not listed among the paper's cases): the foot point
    # s_1 theta_1 + s_2 theta_2 becomes (-s_1 sin phi_1, s_1 cos phi_1, s_2) and theta is
    # horizontal, so every detector row (s_2 = w) holds rays in the plane z = w that meet only
    # the slice holding it, as the 2D parallel beam with phi = phi_1 and s = s_1 = u does on the
    # slice's image.  phi_1 = 0 and pi/2 are axis-parallel views.
    rng = np.random.default_rng(6)
    nx, ny, nz = 9, 8, 5
    dx, dy, dz, cx, cy, cz = 0.9, 1.1, 1.3, 0.4, -0.3, 0.45
    phi1 = np.radians([-30.0, 0.0, 25.0, 90.0, 140.0])
    n_rows, n_cols, du, dv, u0, v0 = 5, 11, 0.9, 1.1, 0.17, 0.23
    g3 = Geometry("par3d", nx, ny, nz, dx=dx, dy=dy, dz=dz, cx=cx, cy=cy, cz=cz,
                  angles=np.stack([phi1, np.zeros_like(phi1)], axis=1), n_cols=n_cols, n_rows=n_rows, du=du,
                  dv=dv, u0=u0, v0=v0)
    g2 = Geometry("par2d", nx, ny, dx=dx, dy=dy, cx=cx, cy=cy, angles=phi1, n_cols=n_cols, du=du, u0=u0)
    f = rng.uniform(0.0, 1.0, (nz, ny, nx))
    sino = rng.uniform(0.0, 1.0, (len(phi1), n_rows, n_cols))
    y3 = O.forward(g3, f.reshape(-1)).reshape(len(phi1), n_rows, n_cols)
    z3 = O.adjoint(g3, sino.reshape(-1)).reshape(nz, ny, nx)
    z_expect = np.zeros((nz, ny, nx))
    for r in range(n_rows):
        z = (r - 0.5 * (n_rows - 1)) * dv + v0
        kh = (cz + 0.5 * nz * dz - z) / dz  # the row's slice coordinate (k counts down)
        assert 0.0 < kh < nz and abs(kh - round(kh)) > 0.01  # no row on a slice boundary
        k = int(math.floor(kh))
        y2 = O.forward(g2, f[k].reshape(-1)).reshape(len(phi1), n_cols)
        np.testing.assert_allclose(y3[:, r, :], y2, rtol=1e-12, atol=1e-12)
        z_expect[k] += O.adjoint(g2, sino[:, r, :].reshape(-1)).reshape(ny, nx)
    np.testing.assert_allclose(z3, z_expect, rtol=1e-12, atol=1e-12)


def _steps(trace, kind):
    return [r for r in trace if r[0] == kind]


def test_ts1_hand_intermediates():
    # Section 5.1 (i)-(iii)
    _, _, tr = O.ray_units(TS1, 0, trace=True)
    drive = _steps(tr, 0)
    cand = _steps(tr, 1)
    assert drive[0][2] == pytest.approx(1 - 3 * r2 / 2) and drive[0][3] == pytest.approx(3 - r2)
    # (ii) prints C_1 = 5/2 - 3sqrt2/2 for i = 1; eq. restriction_j with the printed
    # C_x = 1 - sqrt2/2 gives 2 - sqrt2 (C_1 falls by tan(phi) = 1 per step of i).  Both leave
    # the single valid j = 0 that the paper states; the consistent value is pinned.
    assert drive[1][2] == pytest.approx(1 - r2 / 2) and drive[1][3] == pytest.approx(2 - r2)
    assert drive[0][3] - drive[1][3] == pytest.approx(1.0)
    valid = {(int(r[1]), int(r[2])): r for r in cand}
    assert sorted(valid) == [(0, 0), (0, 1), (1, 0)]  # (i, j); i = 2 has no valid j
    assert valid[(0, 0)][3] == pytest.approx(1.5 * r2 - 1)
    assert valid[(0, 1)][3] == pytest.approx(r2 / 2 - 1)
    assert valid[(1, 0)][3] == pytest.approx(1.5 * r2 - 1)


def test_ts2_hand_intermediates():
    # Section 5.2 (i)-(iii): phi = 5pi/6 lies outside Case 1; the open j-range is the one
    # the paper computes by hand.
    _, _, tr = O.ray_units(TS2, 0, trace=True)
    drive = _steps(tr, 0)
    assert drive[0][2] == pytest.approx(2 * r3 / 3)
    assert (drive[0][4], drive[0][5]) == pytest.approx((1 + 2 * r3 / 3, 2 + r3))
    assert drive[1][2] == pytest.approx(0.0, abs=1e-12)
    assert (drive[1][4], drive[1][5]) == pytest.approx((1 + r3, 2 + 4 * r3 / 3))
    cand = _steps(tr, 1)
    assert [(int(r[1]), int(r[2])) for r in cand] == [(0, 3), (1, 3)]
    assert cand[0][3] == pytest.approx(2 * r3 - 2) and cand[1][3] == pytest.approx(2 * r3 - 2)


def test_ts3_hand_intermediates():
    # Section 5.3 (i)-(iii): C_x, the j-range, C_y and the k-range for each i
    _, _, tr = O.ray_units(TS3, 0, trace=True)
    drive = _steps(tr, 0)
    assert [d[2] for d in drive] == pytest.approx([-3.0, -1.0, 1.0])
    assert [(d[4], d[5]) for d in drive] == [pytest.approx((1, 3)), pytest.approx((0, 2)), pytest.approx((-1, 1))]
    cand = _steps(tr, 1)
    assert [(int(r[1]), int(r[2])) for r in cand] == [(0, 2), (1, 1), (2, 0)]
    assert [r[3] for r in cand] == pytest.approx([-1.0, 1.0, 3.0])
    want_k = [((1 + r2) / 2, (3 + 3 * r2) / 2), ((1 - r2) / 2, (3 + r2) / 2), ((1 - 3 * r2) / 2, (3 - r2) / 2)]
    for r, (lo, hi) in zip(cand, want_k):
        assert (r[4], r[5]) == pytest.approx((lo, hi))


def test_ambiguity_2d_grid_line():
    # Section 4.1, first example: 5x5, ray (1.5, 0) lies on a grid line -> pixel (1, i)
    g = Geometry("par2d", 5, 5, angles=[0.0], n_cols=1, u0=1.5)
    idx, ln = O.ray_units(g, 0)
    np.testing.assert_array_equal(idx, 5 + np.arange(5))
    np.testing.assert_allclose(ln, 1.0)


def test_ambiguity_3d_grid_edge():
    # Section 4.1, second example: 4x4x4, ray (1, 1, 0, 0) on a grid edge -> voxels (1, 1, i)
    g = Geometry("par3d", 4, 4, 4, angles=[[0.0, 0.0]], u0=1.0, v0=1.0)
    idx, ln = O.ray_units(g, 0)
    np.testing.assert_array_equal(idx, (1 * 4 + 1) * 4 + np.arange(4))
    np.testing.assert_allclose(ln, 1.0)


def test_ambiguity_3d_grid_plane():
    # Section 4.1, third example: 3x3x3, ray (-0.5, sqrt2, 0, pi/4) in a grid plane: only
    # i = 0 with k = 0 and length sqrt2, voxels (0,1,0) and (0,2,0) -> (0,2,0), index 6
    g = Geometry("par3d", 3, 3, 3, angles=[[0.0, pi / 4]], u0=-0.5, v0=r2)
    idx, ln = O.ray_units(g, 0)
    np.testing.assert_array_equal(idx, [6])
    np.testing.assert_allclose(ln, [r2], rtol=1e-12)


def test_edge_rays_keep_edge_units():
    # A ray on the outer boundary of the image still crosses the edge row / column
    for s, want_j in ((2.5, 0), (-2.5, 4)):
        g = Geometry("par2d", 5, 5, angles=[0.0], n_cols=1, u0=s)
        idx, ln = O.ray_units(g, 0)
        np.testing.assert_array_equal(idx, want_j * 5 + np.arange(5))
    g = Geometry("par2d", 5, 5, angles=[pi / 2], n_cols=1, u0=2.5)  # x = -2.5: left edge
    idx, _ = O.ray_units(g, 0)
    np.testing.assert_array_equal(idx, np.arange(5) * 5 + 0)
    g = Geometry("par2d", 5, 5, angles=[0.0], n_cols=1, u0=2.5000001)  # just outside
    assert O.ray_units(g, 0)[0].size == 0
