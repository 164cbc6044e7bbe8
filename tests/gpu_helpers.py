"""Shared pieces of the GPU parity tests: reduced copies of the five scan configurations,
and the tolerances.

Tolerances (FP32 kernel vs FP64 oracle):
* per ray sum:  |y - y_ref| <= 1e-5 * S + eps_ray, S = sum_I |f_I| l_I (oracle).  The floor
  eps_ray = 32 * 2^-24 * T * max|f| covers rays whose sum is tiny next to their scale: the
  kernel's plane crossings are floats measured from the ray's foot point, |t| <= T (the
  image half-diagonal), so every length carries an absolute error of a few ulp(T).
  Rays nearly parallel to an axis add a term: a plane of the minor axis B is crossed at
  t = fma(q, 1/w_B, -f_B/w_B), and rounding the constant -f_B/w_B (f_B < 1) alone moves it
  by up to 2^-24 / |w_B|, so a crossing carries an absolute error of about
  2^-24 (2|t| + 1/|w_B|).  Each B crossing moves length between two units
  (|v_a - v_b| <= max|f|), and the box's entry and exit on B faces move the chord's ends:
  eps_cond = 4 * 2^-24 / |w_B| * max|f| where the caller passes the rays' minor index slopes
  (check_rays(..., w_min=...)); it exceeds eps_ray only on images a few units across.
* adjoint image: max |z - z_ref| <= 1e-4 * max |z_ref|.
* dot product:   |<Ax, y> - <x, A^T y>| <= 1e-5 * |<Ax, y>| (both reductions in float64).
* unit sets:     bit-exact for units whose length exceeds delta = 16 * 2^-24 * T on both
  sides ("grazing" units below it may appear on one side only); matched lengths agree to
  delta.
"""
from __future__ import annotations

import math

import numpy as np

from paper_2006_00686_gb300 import inputs
from paper_2006_00686_gb300.inputs import Geometry

U32 = 2.0 ** -24


def half_diag(g: Geometry) -> float:
    return 0.5 * math.sqrt((g.nx * g.dx) ** 2 + (g.ny * g.dy) ** 2 + ((g.nz * g.dz) ** 2 if g.is3d else 0.0))


def ray_tol(g: Geometry, scale: np.ndarray, fmax: float) -> np.ndarray:
    return 1e-5 * np.abs(scale) + 32.0 * U32 * half_diag(g) * fmax


def grazing_delta(g: Geometry) -> float:
    return 16.0 * U32 * half_diag(g)


def minor_slope_2d(g: Geometry, rays) -> np.ndarray:
    """Smallest index-space slope |w| of each listed 2D ray (its direction's smaller component
    over the larger unit side; 0 for rays parallel to an axis), from the oracle's (s, phi)."""
    from oracle import oracle as O
    phi = np.array([O.ray_params(g, int(r))[1] for r in rays])
    return np.minimum(np.abs(np.sin(phi)), np.abs(np.cos(phi))) / max(g.dx, g.dy)


def check_rays(g, y_gpu, y_ref, scale, fmax, what="", w_min=None):
    """Assert the per-ray bound; return the worst error in units of the tolerance.  w_min: the
    rays' minor index slopes (minor_slope_2d), for the near-axis term."""
    tol = ray_tol(g, scale, fmax)
    if w_min is not None:
        w = np.asarray(w_min, np.float64)
        tol = tol + np.where(w > 1e-9, 4.0 * U32 * fmax / np.maximum(w, 1e-9), 0.0)
    err = np.abs(np.asarray(y_gpu, np.float64) - y_ref)
    ratio = err / tol
    worst = int(np.argmax(ratio))
    assert ratio[worst] <= 1.0, (f"{what}: ray {worst} err {err[worst]:.3g} tol {tol[worst]:.3g} "
                                 f"gpu {y_gpu[worst]:.7g} ref {y_ref[worst]:.7g}; "
                                 f"{int((ratio > 1).sum())} rays over")
    return float(ratio[worst])


def check_adjoint(z_gpu, z_ref, what=""):
    z_gpu = np.asarray(z_gpu, np.float64).reshape(z_ref.shape)
    scale = float(np.abs(z_ref).max())
    err = float(np.abs(z_gpu - z_ref).max())
    assert err <= 1e-4 * scale, f"{what}: adjoint max err {err:.3g} vs scale {scale:.3g}"
    return err / scale


def check_unit_sets(g, rows_gpu, rows_ref):
    """rows_*: list of (idx, len) per ray.  Returns the number of grazing-only differences."""
    delta = grazing_delta(g)
    graze = 0
    for q, ((ig, lg), (io, lo)) in enumerate(zip(rows_gpu, rows_ref)):
        dg = dict(zip(np.asarray(ig).tolist(), np.asarray(lg, np.float64).tolist()))
        do = dict(zip(np.asarray(io).tolist(), np.asarray(lo, np.float64).tolist()))
        assert len(dg) == len(ig), f"ray {q}: a unit visited twice"
        for k in set(dg) | set(do):
            a, b = dg.get(k, 0.0), do.get(k, 0.0)
            if k in dg and k in do:
                assert abs(a - b) <= delta, f"ray {q} unit {k}: length {a} vs {b}"
            else:
                assert max(a, b) <= delta, f"ray {q} unit {k}: only one side has it (gpu {a}, oracle {b})"
                graze += 1
    return graze


# ---------------------------------------------------------------------------------------
# Reduced configurations: same scan kinds, angle sets and proportions, smaller grids
# ---------------------------------------------------------------------------------------


def fan2d_small(n=128, views=180):
    s = n / 512.0
    v = np.arange(views, dtype=np.float64)
    return Geometry("fan2d", n, n, angles=2 * math.pi * v / views, n_cols=int(768 * s), du=1.2,
                    sod=1000.0 * s, sdd=1500.0 * s)


def par3d_small(n=32):
    g = inputs.par3d_256_tilt()
    return Geometry("par3d", n, n, n, angles=g.angles, n_cols=n, n_rows=n)


def cone_small(n=64, views=90):
    s = n / 512.0
    v = np.arange(views, dtype=np.float64)
    return Geometry("cone", n, n, n, dx=0.8, dy=0.8, dz=1.0, cx=10.0 * s, cy=-5.0 * s, cz=3.0 * s,
                    angles=2 * math.pi * v / views, n_cols=int(1024 * s), n_rows=int(768 * s),
                    sod=1000.0 * s, sdd=1500.0 * s)


def helix_small(n=64, nz=32, views_per_turn=90, turns=2):
    s = n / 512.0
    n_rows = 16
    sod, sdd = 600.0 * s, 1100.0 * s
    feed = 1.0 * n_rows * 1.0 * sod / sdd
    v = np.arange(views_per_turn * turns, dtype=np.float64)
    h = -feed * turns / 2.0 + feed * v / views_per_turn
    return Geometry("helix", n, n, nz, angles=2 * math.pi * v / views_per_turn, src_z=h,
                    n_cols=int(736 * s), n_rows=n_rows, sod=sod, sdd=sdd)


def sample_rays(g: Geometry, n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(g.n_rays, size=min(n, g.n_rays), replace=False))
