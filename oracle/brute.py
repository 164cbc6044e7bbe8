"""Independent brute force for tiny grids (TEST INFRASTRUCTURE ONLY).

Shares nothing with ``xray_oracle.c``: the ray is built directly from the scan's physical
layout (source position, detector point) instead of the paper's transformation formulas,
and every unit's intersection length is obtained by clipping the line against the unit's
box (slab method), with no use of the non-vanishing-intersectability condition.

* ``ray_of(g, r)`` -> point, unit direction in world coordinates.
* ``lengths(g, point, direction)`` -> dense array of exact lengths for every unit.
* ``sampled_lengths(...)`` -> lengths estimated by dense midpoint sampling (error <= 2h).
* ``box_chord(...)`` -> length of the line inside the whole image box.

For a direction component that is exactly zero (|component| < 1e-12), the line lies in a
family of grid planes; the unit along that axis is the one whose index-space interval
[n, n+1) holds the line, and the far edge belongs to the last unit.  This is the paper's
ambiguity rule of Section 4.1 (bigger index) restated as "floor of the index coordinate".
"""
from __future__ import annotations

import math

import numpy as np

_EPS = 1e-12


def _cs(a):
    """cos, sin of an angle; an angle within rounding of a multiple of pi/2 gives exact 0/+-1."""
    c, s = math.cos(a), math.sin(a)
    if abs(c) < _EPS:
        return 0.0, math.copysign(1.0, s)
    if abs(s) < _EPS:
        return math.copysign(1.0, c), 0.0
    return c, s


def _det(g, r, c):
    u = (c - 0.5 * (g.n_cols - 1)) * g.du + g.u0
    v = (r - 0.5 * (g.n_rows - 1)) * g.dv + g.v0
    return u, v


def ray_of(g, ray: int):
    """World-space point on the ray and unit direction, from the scan layout."""
    nc, nr = int(g.n_cols), int(g.n_rows)
    c, r, v = ray % nc, (ray // nc) % nr, ray // (nc * nr)
    u, w = _det(g, r, c)
    ang = np.asarray(g.angles)
    k = g.kind
    if k == "par2d":
        c, s = _cs(float(ang[v]))
        p = np.array([-u * s, u * c, 0.0])
        d = np.array([c, s, 0.0])
    elif k in ("fan2d", "fan2d_arc"):
        a = float(ang[v])
        S = g.sod * np.array([-math.sin(a), math.cos(a), 0.0])  # source, angle a from +y
        e_c = np.array([math.sin(a), -math.cos(a), 0.0])  # source -> origin
        e_t = np.array([math.cos(a), math.sin(a), 0.0])  # along the detector
        if k == "fan2d":
            d = g.sdd * e_c + u * e_t  # flat detector at distance sdd
        else:
            d = math.cos(u) * e_c + math.sin(u) * e_t  # u is the fan angle
        p = S
    elif k == "rays2d":
        # the ray with normal distance s and direction (cos phi, sin phi) (eq. direction_normal)
        sv, phi = float(ang[v][0]), float(ang[v][1])
        c, s = _cs(phi)
        p = np.array([-sv * s, sv * c, 0.0])
        d = np.array([c, s, 0.0])
    elif k == "rays3d":
        # p = s1 theta_1 + s2 theta_2, direction theta (eq. 3Dparallel_direction, theta_1, theta_2)
        s1v, s2v, f1, f2 = (float(x) for x in ang[v])
        c1, s1 = _cs(f1)
        c2, s2 = _cs(f2)
        d = np.array([c2 * c1, c2 * s1, s2])
        p = s1v * np.array([-s1, c1, 0.0]) + s2v * np.array([-s2 * c1, -s2 * s1, c2])
    elif k == "par3d":
        c1, s1 = _cs(float(ang[v][0]))
        c2, s2 = _cs(float(ang[v][1]))
        d = np.array([c2 * c1, c2 * s1, s2])
        t1 = np.array([-s1, c1, 0.0])
        t2 = np.array([-s2 * c1, -s2 * s1, c2])
        p = u * t1 + w * t2
    else:
        a = float(ang[v])
        H = float(g.src_z[v]) if k in ("helix", "helix_arc") else 0.0
        e_c = np.array([math.cos(a), math.sin(a), 0.0])  # source -> rotation axis
        e_u = np.array([-math.sin(a), math.cos(a), 0.0])
        e_v = np.array([0.0, 0.0, 1.0])
        S = -g.sod * e_c + H * e_v
        if k in ("cone", "helix"):
            d = g.sdd * e_c + u * e_u + w * e_v  # flat detector at distance sdd
        else:
            d = math.cos(w) * (math.cos(u) * e_c + math.sin(u) * e_u) + math.sin(w) * e_v
        p = S
    d = d / np.linalg.norm(d)
    d = np.where(np.abs(d) < _EPS, 0.0, d)
    return p, d


def _bounds(g):
    """Plane coordinates per axis in index order: x grows with i, y and z fall with j, k."""
    bx = g.cx + (np.arange(g.nx + 1) - g.nx / 2.0) * g.dx
    by = g.cy + (g.ny / 2.0 - np.arange(g.ny + 1)) * g.dy
    bz = g.cz + (g.nz / 2.0 - np.arange(g.nz + 1)) * g.dz
    return bx, by, bz


def _axis_intervals(b, p, d, n, lower_first):
    """Per unit along one axis: (t_lo, t_hi) of the slab, or a membership mask when d == 0."""
    if d != 0.0:
        t = (b - p) / d
        t0, t1 = t[:-1], t[1:]
        return np.minimum(t0, t1), np.maximum(t0, t1), None
    # index coordinate of the point, unit = floor, far edge to the last unit
    h = (b[1] - b[0])
    uc = (p - b[0]) / h
    mask = np.zeros(n, dtype=bool)
    if 0.0 <= uc <= n:
        mask[min(int(math.floor(uc)), n - 1)] = True
    return np.full(n, -np.inf), np.full(n, np.inf), mask


def lengths(g, p, d) -> np.ndarray:
    """Exact intersection length with every unit, shape image_shape (2D: [ny, nx])."""
    bx, by, bz = _bounds(g)
    three = g.kind in ("par3d", "cone", "cone_arc", "helix", "helix_arc", "rays3d")
    lx0, lx1, mx = _axis_intervals(bx, p[0], d[0], g.nx, True)
    ly0, ly1, my = _axis_intervals(by, p[1], d[1], g.ny, False)
    if three:
        lz0, lz1, mz = _axis_intervals(bz, p[2], d[2], g.nz, False)
        lo = np.maximum(np.maximum(lz0[:, None, None], ly0[None, :, None]), lx0[None, None, :])
        hi = np.minimum(np.minimum(lz1[:, None, None], ly1[None, :, None]), lx1[None, None, :])
        L = np.maximum(hi - lo, 0.0)
        L[~np.isfinite(L)] = 0.0
        if mx is not None:
            L = L * mx[None, None, :]
        if my is not None:
            L = L * my[None, :, None]
        if mz is not None:
            L = L * mz[:, None, None]
        return L
    lo = np.maximum(ly0[:, None], lx0[None, :])
    hi = np.minimum(ly1[:, None], lx1[None, :])
    L = np.maximum(hi - lo, 0.0)
    L[~np.isfinite(L)] = 0.0
    if mx is not None:
        L = L * mx[None, :]
    if my is not None:
        L = L * my[:, None]
    return L


def box_chord(g, p, d) -> float:
    """Length of the line inside the image box (slab method on one box)."""
    lo = np.array([g.cx - g.nx * g.dx / 2, g.cy - g.ny * g.dy / 2, g.cz - g.nz * g.dz / 2])
    hi = np.array([g.cx + g.nx * g.dx / 2, g.cy + g.ny * g.dy / 2, g.cz + g.nz * g.dz / 2])
    three = g.kind in ("par3d", "cone", "cone_arc", "helix", "helix_arc", "rays3d")
    t0, t1 = -np.inf, np.inf
    for a in range(3 if three else 2):
        if d[a] == 0.0:
            if not (lo[a] <= p[a] <= hi[a]):
                return 0.0
            continue
        ta, tb = (lo[a] - p[a]) / d[a], (hi[a] - p[a]) / d[a]
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    return max(0.0, t1 - t0)


def sampled_lengths(g, p, d, h: float = 1e-3) -> np.ndarray:
    """Midpoint sampling of the line at spacing h inside the box; per-unit error <= 2h."""
    three = g.kind in ("par3d", "cone", "cone_arc", "helix", "helix_arc", "rays3d")
    lo = np.array([g.cx - g.nx * g.dx / 2, g.cy - g.ny * g.dy / 2, g.cz - g.nz * g.dz / 2])
    hi = np.array([g.cx + g.nx * g.dx / 2, g.cy + g.ny * g.dy / 2, g.cz + g.nz * g.dz / 2])
    R = float(np.linalg.norm(hi - lo)) + float(np.linalg.norm(p - 0.5 * (lo + hi)))
    t = np.arange(-R, R, h) + 0.5 * h
    pts = p[None, :] + t[:, None] * d[None, :]
    ii = np.floor((pts[:, 0] - lo[0]) / g.dx).astype(np.int64)
    jj = np.floor((hi[1] - pts[:, 1]) / g.dy).astype(np.int64)
    kk = np.floor((hi[2] - pts[:, 2]) / g.dz).astype(np.int64) if three else np.zeros_like(ii)
    ok = (ii >= 0) & (ii < g.nx) & (jj >= 0) & (jj < g.ny) & (kk >= 0) & (kk < g.nz)
    flat = ((kk * g.ny + jj) * g.nx + ii)[ok]
    L = np.bincount(flat, minlength=g.nx * g.ny * g.nz).astype(np.float64) * h
    return L.reshape((g.nz, g.ny, g.nx) if three else (g.ny, g.nx))
