"""ctypes binding of the double-precision CPU oracle (``oracle/xray_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg.  It never imports the CUDA package; scans are
passed as any object with the attributes of ``paper_2006_00686_gb300.inputs.Geometry``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "xray_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

KIND_IDS = {"par2d": 0, "fan2d": 1, "fan2d_arc": 2, "par3d": 3, "cone": 4, "cone_arc": 5,
            "helix": 6, "helix_arc": 7, "rays2d": 8, "rays3d": 9}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP when available, no FMA contraction)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", SRC, "-o", LIB, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    return LIB


class _Geom(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("cx", ctypes.c_double), ("cy", ctypes.c_double), ("cz", ctypes.c_double),
        ("n_views", ctypes.c_int), ("n_rows", ctypes.c_int), ("n_cols", ctypes.c_int),
        ("angles", ctypes.POINTER(ctypes.c_double)),
        ("src_z", ctypes.POINTER(ctypes.c_double)),
        ("du", ctypes.c_double), ("dv", ctypes.c_double), ("u0", ctypes.c_double), ("v0", ctypes.c_double),
        ("sod", ctypes.c_double), ("sdd", ctypes.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        c_long_p = P(ctypes.c_long)
        c_double_p = P(ctypes.c_double)
        _lib.orc_ray_params.argtypes = [P(_Geom), ctypes.c_long, c_double_p]
        _lib.orc_ray_units.argtypes = [P(_Geom), ctypes.c_long, c_long_p, c_double_p, ctypes.c_int,
                                       c_double_p, ctypes.c_int, P(ctypes.c_int)]
        _lib.orc_ray_units.restype = ctypes.c_int
        _lib.orc_forward.argtypes = [P(_Geom), c_double_p, c_double_p, c_long_p, ctypes.c_long,
                                     ctypes.c_int, ctypes.c_int]
        _lib.orc_adjoint.argtypes = [P(_Geom), c_double_p, c_double_p, c_long_p, ctypes.c_long,
                                     ctypes.c_int, ctypes.c_int]
        for name in ("orc_forward_attenuated", "orc_adjoint_attenuated"):
            fn = getattr(_lib, name)
            fn.argtypes = [P(_Geom), c_double_p, c_double_p, c_double_p, c_long_p, ctypes.c_long, ctypes.c_int,
                           ctypes.c_int]
            fn.restype = ctypes.c_int
        _lib.orc_max_threads.restype = ctypes.c_int
    return _lib


def max_threads() -> int:
    return int(lib().orc_max_threads())


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _geom(g):
    """(struct, keep-alive arrays) for a scan description."""
    ang = np.ascontiguousarray(np.asarray(g.angles, dtype=np.float64).reshape(-1))
    sz = None if g.src_z is None else np.ascontiguousarray(np.asarray(g.src_z, dtype=np.float64))
    n_views = int(np.asarray(g.angles).shape[0])
    s = _Geom(KIND_IDS[g.kind], int(g.nx), int(g.ny), int(g.nz), float(g.dx), float(g.dy), float(g.dz),
              float(g.cx), float(g.cy), float(g.cz), n_views, int(g.n_rows), int(g.n_cols),
              _dptr(ang), None if sz is None else _dptr(sz),
              float(g.du), float(g.dv), float(g.u0), float(g.v0), float(g.sod), float(g.sdd))
    return s, (ang, sz)


def n_rays(g) -> int:
    return int(np.asarray(g.angles).shape[0]) * int(g.n_rows) * int(g.n_cols)


def n_units(g) -> int:
    return int(g.nx) * int(g.ny) * int(g.nz)


def ray_params(g, ray: int) -> np.ndarray:
    """Canonical ray parameters: (s, phi) in 2D, (s1, s2, phi1, phi2) in 3D."""
    s, keep = _geom(g)
    out = np.zeros(4)
    lib().orc_ray_params(ctypes.byref(s), int(ray), _dptr(out))
    return out[:4 if g.kind in ("par3d", "cone", "cone_arc", "helix", "helix_arc") else 2]


def ray_units(g, ray: int, trace: bool = False):
    """(indices int64 ascending, lengths float64) of the units ray ``ray`` crosses with positive
    length; with ``trace`` also the list of intermediate records (see the C source)."""
    s, keep = _geom(g)
    cap = 4 * (int(g.nx) + int(g.ny) + int(g.nz)) + 16
    idx = np.zeros(cap, dtype=np.int64)
    ln = np.zeros(cap, dtype=np.float64)
    cap_tr = 64 * cap if trace else 0
    tr = np.zeros((max(cap_tr, 1), 8))
    ntr = ctypes.c_int(0)
    n = lib().orc_ray_units(ctypes.byref(s), int(ray), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                            _dptr(ln), cap, _dptr(tr) if trace else None, cap_tr, ctypes.byref(ntr))
    if n < 0:
        raise RuntimeError("oracle unit list overflow")
    if trace:
        return idx[:n].copy(), ln[:n].copy(), tr[:ntr.value].copy()
    return idx[:n].copy(), ln[:n].copy()


def _rays_arg(rays):
    if rays is None:
        return None, None
    r = np.ascontiguousarray(np.asarray(rays, dtype=np.int64))
    return r, r.ctypes.data_as(ctypes.POINTER(ctypes.c_long))


def forward(g, img, rays=None, threads: int | None = None) -> np.ndarray:
    """Forward projection in float64.  ``img``: [units] or [batch, units...]; returns
    [n_rays] or [batch, n_rays] (sinogram order: view, row, column)."""
    s, keep = _geom(g)
    f = np.asarray(img, dtype=np.float64)
    single = f.size == n_units(g)
    f = np.ascontiguousarray(f.reshape(-1 if single else f.shape[0], n_units(g)) if not single
                             else f.reshape(1, -1))
    batch = f.shape[0]
    r, rp = _rays_arg(rays)
    nr = n_rays(g) if r is None else r.size
    out = np.zeros((batch, nr))
    rc = lib().orc_forward(ctypes.byref(s), _dptr(f), _dptr(out), rp, nr, batch,
                           threads or max_threads())
    if rc != 0:
        raise RuntimeError("oracle unit list overflow")
    return out[0] if single else out


def adjoint(g, sino, rays=None, threads: int | None = None) -> np.ndarray:
    """Adjoint in float64.  ``sino``: [n] or [batch, n] values of the rays ``rays`` (all rays
    when None); returns [units] or [batch, units]."""
    s, keep = _geom(g)
    r, rp = _rays_arg(rays)
    nr = n_rays(g) if r is None else r.size
    y = np.asarray(sino, dtype=np.float64)
    single = y.size == nr
    y = np.ascontiguousarray(y.reshape(1 if single else y.shape[0], nr))
    batch = y.shape[0]
    out = np.zeros((batch, n_units(g)))
    rc = lib().orc_adjoint(ctypes.byref(s), _dptr(y), _dptr(out), rp, nr, batch, threads or max_threads())
    if rc != 0:
        raise RuntimeError("oracle unit list overflow")
    return out[0] if single else out


def forward_attenuated(g, mu, img, rays=None, threads: int | None = None) -> np.ndarray:
    """Attenuated forward projection in float64 (exponential weight of the attenuation map
    ``mu`` along each ray, integrated towards +theta)."""
    s, keep = _geom(g)
    m = np.ascontiguousarray(np.asarray(mu, dtype=np.float64).reshape(-1))
    f = np.asarray(img, dtype=np.float64)
    single = f.size == n_units(g)
    f = np.ascontiguousarray(f.reshape(1, -1) if single else f.reshape(f.shape[0], n_units(g)))
    batch = f.shape[0]
    r, rp = _rays_arg(rays)
    nr = n_rays(g) if r is None else r.size
    out = np.zeros((batch, nr))
    rc = lib().orc_forward_attenuated(ctypes.byref(s), _dptr(m), _dptr(f), _dptr(out), rp, nr, batch,
                                      threads or max_threads())
    if rc != 0:
        raise RuntimeError("oracle unit list overflow")
    return out[0] if single else out


def adjoint_attenuated(g, mu, sino, rays=None, threads: int | None = None) -> np.ndarray:
    """Adjoint of forward_attenuated in float64."""
    s, keep = _geom(g)
    m = np.ascontiguousarray(np.asarray(mu, dtype=np.float64).reshape(-1))
    r, rp = _rays_arg(rays)
    nr = n_rays(g) if r is None else r.size
    y = np.asarray(sino, dtype=np.float64)
    single = y.size == nr
    y = np.ascontiguousarray(y.reshape(1 if single else y.shape[0], nr))
    batch = y.shape[0]
    out = np.zeros((batch, n_units(g)))
    rc = lib().orc_adjoint_attenuated(ctypes.byref(s), _dptr(m), _dptr(y), _dptr(out), rp, nr, batch,
                                      threads or max_threads())
    if rc != 0:
        raise RuntimeError("oracle unit list overflow")
    return out[0] if single else out

