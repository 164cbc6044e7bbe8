"""Seeded synthetic inputs for the X-ray transform: scan descriptions and phantoms.

This module is shared by the CUDA path's tests and benchmark and by the oracle's tests.
It holds none of the transform's arithmetic (no ray parameters, no intersection
lengths): only the description of a scan (image grid, view angles, detector sampling,
source distances) and point-sampled ellipse / ellipsoid phantoms.

Conventions (Section 2.1 and Section 3.1 of the paper, "imaging coordinate system" and
"pixel/voxel indexes"):

* image array ``[nz][ny][nx]`` (2D: ``[ny][nx]``), ``i`` along +x, ``j`` counting rows
  from the top (y decreasing), ``k`` counting slices from the top (z decreasing);
  1D index ``I = (k*ny + j)*nx + i``;
* unit ``(k, j, i)`` is centred at ``(cx + (i-(nx-1)/2)dx, cy + ((ny-1)/2-j)dy,
  cz + ((nz-1)/2-k)dz)``;
* sinogram array ``[n_views][n_rows][n_cols]`` (2D: ``n_rows == 1``), detector sample
  coordinates ``u_c = (c-(n_cols-1)/2)du + u0`` and ``v_r = (r-(n_rows-1)/2)dv + v0``.

Scan kinds (name -> C enum value used by both the library and the oracle):

``par2d``     parallel beam, ``angles[v]`` = phi, ``u`` = s (Section 2.2.1)
``fan2d``     equispaced fan, ``angles[v]`` = alpha, flat detector at ``sdd`` (eq. 2Dparalleltofan_2)
``fan2d_arc`` equiangular fan, ``angles[v]`` = alpha, ``u`` is the angle gamma (eq. 2Dparalleltofan)
``par3d``     parallel beam, ``angles[v]`` = (phi1, phi2), ``u`` = s1, ``v`` = s2 (Section 3.2.1)
``cone``      equispaced circular cone, ``angles[v]`` = phi'_1, flat detector (eq. equispaced_cone_beam)
``cone_arc``  equiangular circular cone, ``u``, ``v`` are the angles alpha, beta (eq. equiangular_cone_beam)
``helix``     equispaced helical cone, ``src_z[v]`` = H (eq. Helical_cone_beam_equispaced)
``helix_arc`` equiangular helical cone (eq. Helical_cone_beam_equiangular)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import numpy as np

KINDS = {
    "par2d": 0,
    "fan2d": 1,
    "fan2d_arc": 2,
    "par3d": 3,
    "cone": 4,
    "cone_arc": 5,
    "helix": 6,
    "helix_arc": 7,
    "rays2d": 8,  # a list of rays, each given by its parameters (s, phi)
    "rays3d": 9,  # a list of rays, each given by its parameters (s1, s2, phi1, phi2)
}
KINDS_3D = ("par3d", "cone", "cone_arc", "helix", "helix_arc", "rays3d")
RAY_LISTS = {"rays2d": 2, "rays3d": 4}  # parameters per ray


@dataclass
class Geometry:
    """One scan: image grid + rays. Plain numbers only; both code paths read it."""

    kind: str
    nx: int
    ny: int
    nz: int = 1
    dx: float = 1.0
    dy: float = 1.0
    dz: float = 1.0
    cx: float = 0.0
    cy: float = 0.0
    cz: float = 0.0
    angles: np.ndarray = None  # float64 [n_views] (par3d: [n_views, 2]; ray lists: [n_rays, 2 or 4])
    src_z: np.ndarray = None  # float64 [n_views], helical kinds only
    n_cols: int = 1
    n_rows: int = 1
    du: float = 1.0
    dv: float = 1.0
    u0: float = 0.0
    v0: float = 0.0
    sod: float = 0.0
    sdd: float = 0.0

    def __post_init__(self):
        if self.kind not in KINDS:
            raise ValueError(f"unknown scan kind {self.kind!r}")
        self.angles = np.ascontiguousarray(np.asarray(self.angles, dtype=np.float64))
        if self.src_z is not None:
            self.src_z = np.ascontiguousarray(np.asarray(self.src_z, dtype=np.float64))
        if not self.is3d:
            self.nz, self.n_rows = 1, 1
        if self.kind in RAY_LISTS:
            # one "view" per ray, one detector sample each
            self.angles = self.angles.reshape(-1, RAY_LISTS[self.kind])
            self.n_rows, self.n_cols = 1, 1

    @property
    def kind_id(self) -> int:
        return KINDS[self.kind]

    @property
    def is3d(self) -> bool:
        return self.kind in KINDS_3D

    @property
    def n_views(self) -> int:
        return int(self.angles.shape[0])

    @property
    def n_rays(self) -> int:
        return self.n_views * self.n_rows * self.n_cols

    @property
    def n_units(self) -> int:
        return self.nx * self.ny * self.nz

    def image_shape(self, batch: int | None = None) -> tuple:
        s = (self.nz, self.ny, self.nx) if self.is3d else (self.ny, self.nx)
        return s if batch is None else (batch,) + s

    def sino_shape(self, batch: int | None = None) -> tuple:
        s = (self.n_views, self.n_rows, self.n_cols) if self.is3d else (self.n_views, self.n_cols)
        return s if batch is None else (batch,) + s

    def subset_views(self, idx) -> "Geometry":
        idx = np.asarray(idx, dtype=np.int64)
        return replace(
            self,
            angles=self.angles[idx].copy(),
            src_z=None if self.src_z is None else self.src_z[idx].copy(),
        )


# --------------------------------------------------------------------------------------
# Workloads: the five scan configurations and the uneven fan batch
# --------------------------------------------------------------------------------------


def par2d_64() -> Geometry:
    """2D parallel beam: 64x64 unit pixels centred at the origin, 90 views phi=v*pi/90,
    95 bins of spacing 1 (s = c - 47)."""
    v = np.arange(90, dtype=np.float64)
    return Geometry("par2d", 64, 64, angles=v * math.pi / 90.0, n_cols=95, du=1.0)


def fan2d_512(n_views: int = 720) -> Geometry:
    """2D equispaced fan beam: 512x512 pixels of 1.0, 720 views over 2*pi, 768 bins of
    1.2 on a flat detector 1500 from the source, source 1000 from the origin."""
    v = np.arange(n_views, dtype=np.float64)
    return Geometry("fan2d", 512, 512, angles=2.0 * math.pi * v / n_views, n_cols=768, du=1.2,
                    sod=1000.0, sdd=1500.0)


FAN2D_BATCH = 16


def par3d_256_tilt() -> Geometry:
    """3D parallel beam with a single tilt axis (y): 256^3 voxels, phi1=0,
    181 tilts phi2 = -60 deg .. 60 deg, 256x256 detector of spacing 1."""
    v = np.arange(181, dtype=np.float64)
    phi2 = np.deg2rad(-60.0 + v * (120.0 / 180.0))
    ang = np.stack([np.zeros_like(phi2), phi2], axis=1)
    return Geometry("par3d", 256, 256, 256, angles=ang, n_cols=256, n_rows=256)


def cone_512() -> Geometry:
    """3D circular equispaced cone beam: 512^3 voxels of 0.8x0.8x1.0 centred at
    (10,-5,3), 720 views over 2*pi, 1024x768 flat detector of spacing 1.0,
    source-origin 1000, source-detector 1500."""
    v = np.arange(720, dtype=np.float64)
    return Geometry("cone", 512, 512, 512, dx=0.8, dy=0.8, dz=1.0, cx=10.0, cy=-5.0, cz=3.0,
                    angles=2.0 * math.pi * v / 720.0, n_cols=1024, n_rows=768,
                    sod=1000.0, sdd=1500.0)


def helix_512x256() -> Geometry:
    """3D helical equispaced cone beam: 512x512x256 voxels of 1.0, 4 turns of 720 views,
    pitch 1.0, 736x64 flat detector of spacing 1.0, source-origin 600,
    source-detector 1100.  The table feed per turn is pitch * (detector height scaled to
    the rotation axis) = 64 * 600/1100; the source height runs from -2 turns to +2 turns
    of feed across the scan."""
    views_per_turn, turns, pitch = 720, 4, 1.0
    n_rows, dv, sod, sdd = 64, 1.0, 600.0, 1100.0
    feed = pitch * n_rows * dv * sod / sdd
    v = np.arange(views_per_turn * turns, dtype=np.float64)
    h = -feed * turns / 2.0 + feed * v / views_per_turn
    return Geometry("helix", 512, 512, 256, angles=2.0 * math.pi * v / views_per_turn, src_z=h,
                    n_cols=736, n_rows=n_rows, dv=dv, sod=sod, sdd=sdd)


def fans_uneven(n: int = 64, seed: int = 5, n_views: int = 720) -> list:
    """Uneven batch of 2D equispaced fans: image sides drawn in [128, 1024], pixel 1.0,
    720 views over 2*pi, bins = 1.5*side rounded up to a multiple of 8, spacing 1.2,
    source-origin 1000, source-detector 1500."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(128, 1025, size=n)
    v = np.arange(n_views, dtype=np.float64)
    out = []
    for side in sides:
        side = int(side)
        bins = int(math.ceil(1.5 * side / 8.0) * 8)
        out.append(Geometry("fan2d", side, side, angles=2.0 * math.pi * v / n_views, n_cols=bins,
                            du=1.2, sod=1000.0, sdd=1500.0))
    return out


WORKLOADS = {
    "par2d_64": par2d_64,
    "fan2d_512x16": fan2d_512,
    "par3d_256_tilt": par3d_256_tilt,
    "cone_512": cone_512,
    "helix_512x256": helix_512x256,
}

# --------------------------------------------------------------------------------------
# Phantoms: additive ellipses / ellipsoids, point-sampled at unit centres
# --------------------------------------------------------------------------------------


def _half_extent(g: Geometry) -> np.ndarray:
    return 0.5 * np.array([g.nx * g.dx, g.ny * g.dy, g.nz * g.dz], dtype=np.float64)


def ellipse_params(g: Geometry, n: int, seed: int) -> np.ndarray:
    """[n, 6] rows (x0, y0, a, b, angle, density): centres uniform in the disc of 0.8 times
    the inscribed radius, semi-axes U[0.05, 0.4] * side, angle U[0, pi), density U[0, 1]."""
    rng = np.random.default_rng(seed)
    he = _half_extent(g)
    r_in = float(min(he[0], he[1]))
    side = 2.0 * r_in
    rad = 0.8 * r_in * np.sqrt(rng.random(n))
    ang = 2.0 * math.pi * rng.random(n)
    x0 = g.cx + rad * np.cos(ang)
    y0 = g.cy + rad * np.sin(ang)
    a = side * rng.uniform(0.05, 0.4, n)
    b = side * rng.uniform(0.05, 0.4, n)
    rot = math.pi * rng.random(n)
    dens = rng.random(n)
    return np.stack([x0, y0, a, b, rot, dens], axis=1)


def ellipsoid_params(g: Geometry, n: int, seed: int) -> np.ndarray:
    """[n, 10] rows (x0, y0, z0, a, b, c, e1, e2, e3, density): centres uniform in the ball
    of 0.8 times the inscribed radius, semi-axes U[0.05, 0.4] * smallest side, three Euler
    angles U[0, pi), density U[0, 1]."""
    rng = np.random.default_rng(seed)
    he = _half_extent(g)
    r_in = float(he.min())
    side = 2.0 * r_in
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rad = 0.8 * r_in * np.cbrt(rng.random(n))
    c0 = np.array([g.cx, g.cy, g.cz]) + d * rad[:, None]
    axes = side * rng.uniform(0.05, 0.4, (n, 3))
    eul = math.pi * rng.random((n, 3))
    dens = rng.random(n)
    return np.concatenate([c0, axes, eul, dens[:, None]], axis=1)


def _rot_zyz(e1, e2, e3):
    c1, s1, c2, s2, c3, s3 = math.cos(e1), math.sin(e1), math.cos(e2), math.sin(e2), math.cos(e3), math.sin(e3)
    rz1 = np.array([[c1, s1, 0], [-s1, c1, 0], [0, 0, 1]])
    ry = np.array([[c2, 0, s2], [0, 1, 0], [-s2, 0, c2]])
    rz3 = np.array([[c3, s3, 0], [-s3, c3, 0], [0, 0, 1]])
    return rz3 @ ry @ rz1


def phantom(g: Geometry, n_shapes: int, seed: int, device: str = "cpu", dtype=None):
    """Point-sampled phantom as a torch tensor of shape ``g.image_shape()`` (float32 by
    default).  Evaluated in float64 on ``device``; values are sums of densities of the
    shapes whose interior (closed) contains the unit centre."""
    import torch

    dtype = torch.float32 if dtype is None else dtype
    dev = torch.device(device)
    f64 = torch.float64
    xs = g.cx + (torch.arange(g.nx, device=dev, dtype=f64) - (g.nx - 1) / 2.0) * g.dx
    ys = g.cy + ((g.ny - 1) / 2.0 - torch.arange(g.ny, device=dev, dtype=f64)) * g.dy
    if not g.is3d:
        P = ellipse_params(g, n_shapes, seed)
        img = torch.zeros((g.ny, g.nx), device=dev, dtype=f64)
        Y, X = ys[:, None], xs[None, :]
        for x0, y0, a, b, rot, dens in P:
            c, s = math.cos(rot), math.sin(rot)
            xr = (X - x0) * c + (Y - y0) * s
            yr = -(X - x0) * s + (Y - y0) * c
            img += dens * (((xr / a) ** 2 + (yr / b) ** 2) <= 1.0).to(f64)
        return img.to(dtype)
    zs = g.cz + ((g.nz - 1) / 2.0 - torch.arange(g.nz, device=dev, dtype=f64)) * g.dz
    P = ellipsoid_params(g, n_shapes, seed)
    img = torch.zeros((g.nz, g.ny, g.nx), device=dev, dtype=f64)
    for row in P:
        x0, y0, z0, a, b, c = row[:6]
        R = _rot_zyz(*row[6:9])
        dens = row[9]
        # Bounding box of the ellipsoid: half-widths sqrt(sum_k (R[k, a] * axis_k)^2).
        hw = np.sqrt(((R * np.array([a, b, c])[:, None]) ** 2).sum(axis=0))
        sel = []
        for coord, ctr, h in ((xs, x0, hw[0]), (ys, y0, hw[1]), (zs, z0, hw[2])):
            m = ((coord >= ctr - h) & (coord <= ctr + h)).nonzero().flatten()
            sel.append(m)
        if any(m.numel() == 0 for m in sel):
            continue
        ix, iy, iz = sel
        X = xs[ix][None, None, :] - x0
        Y = ys[iy][None, :, None] - y0
        Z = zs[iz][:, None, None] - z0
        q = 0.0
        for kk, ax in enumerate((a, b, c)):
            comp = R[kk, 0] * X + R[kk, 1] * Y + R[kk, 2] * Z
            q = q + (comp / ax) ** 2
        blk = img[iz[0]:iz[-1] + 1, iy[0]:iy[-1] + 1, ix[0]:ix[-1] + 1]
        blk += dens * (q <= 1.0).to(f64)
    return img.to(dtype)


def phantom_batch(g: Geometry, batch: int, n_shapes: int, seed0: int, device: str = "cpu"):
    """Batch of phantoms with seeds ``seed0 + b``."""
    import torch

    return torch.stack([phantom(g, n_shapes, seed0 + b, device=device) for b in range(batch)])
