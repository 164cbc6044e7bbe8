"""Thin Python binding of libxray.so (include/xray.h): argument marshalling only.

Every step of the transform runs in the CUDA library; torch provides device memory and
the current stream.  There is no CPU fallback: if the library is not built, or no CUDA
device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from .inputs import KINDS, KINDS_3D, Geometry

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libxray.so")

XR_ADJ_AUTO, XR_ADJ_SCATTER, XR_ADJ_GATHER = 0, 1, 2
XR_ORDER_AUTO, XR_ORDER_VIEW, XR_ORDER_ROW, XR_ORDER_COLUMN, XR_ORDER_ROWBLOCK, XR_ORDER_TRACE = 0, 1, 2, 3, 4, 5
XR_PATH_AUTO, XR_PATH_TILED, XR_PATH_INTERLEAVED, XR_PATH_RAY = 0, 1, 2, 3


class XRayError(RuntimeError):
    pass


class _Desc(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("cx", ctypes.c_double), ("cy", ctypes.c_double), ("cz", ctypes.c_double),
        ("n_views", ctypes.c_int32), ("n_rows", ctypes.c_int32), ("n_cols", ctypes.c_int32),
        ("angles", ctypes.POINTER(ctypes.c_double)),
        ("src_z", ctypes.POINTER(ctypes.c_double)),
        ("du", ctypes.c_double), ("dv", ctypes.c_double), ("u0", ctypes.c_double), ("v0", ctypes.c_double),
        ("sod", ctypes.c_double), ("sdd", ctypes.c_double),
    ]


class _Info(ctypes.Structure):
    _fields_ = [("n_rays", ctypes.c_int64), ("n_units", ctypes.c_int64), ("table_bytes", ctypes.c_int64),
                ("is3d", ctypes.c_int32), ("device", ctypes.c_int32), ("column_batch", ctypes.c_int32),
                ("trace_walk", ctypes.c_int32)]


class _Tuning(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("batch_chunk", ctypes.c_int32), ("adjoint", ctypes.c_int32),
                ("path", ctypes.c_int32), ("order", ctypes.c_int32)]


class _Problem(ctypes.Structure):
    _fields_ = [("geom", ctypes.c_void_p), ("img", ctypes.c_void_p), ("sino", ctypes.c_void_p)]


# name -> (restype, argtypes); every name here is declared in include/xray.h
_VP, _I32, _I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
SIGNATURES = {
    "xr_geometry_create": (_I32, [ctypes.POINTER(_Desc), ctypes.POINTER(_VP)]),
    "xr_geometry_destroy": (None, [_VP]),
    "xr_ray_setup": (_I32, [_VP, _VP]),
    "xr_geometry_get_info": (_I32, [_VP, ctypes.POINTER(_Info)]),
    "xr_column_batch_plan": (_I32, [ctypes.POINTER(_Desc), ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_int32)]),
    "xr_reserve": (_I32, [_VP, _I32]),
    "xr_set_tuning": (_I32, [_VP, ctypes.POINTER(_Tuning)]),
    "xr_get_tuning": (_I32, [_VP, ctypes.POINTER(_Tuning)]),
    "xr_project": (_I32, [_VP, _VP, _VP, _I32, _VP]),
    "xr_backproject": (_I32, [_VP, _VP, _VP, _I32, _VP]),
    "xr_backproject_method": (_I32, [_VP, _VP, _VP, _I32, _I32, _VP]),
    "xr_project_backproject": (_I32, [_VP, _VP, _VP, _VP, _I32, _VP]),
    "xr_ray_units": (_I32, [_VP, _VP, _I32, _I32, _VP, _VP, _VP, _VP]),
    "xr_system_rows_count": (_I32, [_VP, _I64, _I32, _VP, _VP]),
    "xr_system_rows_fill": (_I32, [_VP, _I64, _I32, _VP, _VP, _VP, _VP]),
    "xr_batch_create": (_I32, [ctypes.POINTER(_Problem), _I32, _I32, _I32, ctypes.POINTER(_VP)]),
    "xr_batch_destroy": (None, [_VP]),
    "xr_batch_project": (_I32, [_VP, _VP]),
    "xr_batch_ray_setup": (_I32, [_VP, _VP]),
    "xr_batch_backproject": (_I32, [_VP, _VP]),
    "xr_project_batched_noalloc": (_I32, [ctypes.POINTER(_Problem), _I32, _I32, _VP]),
    "xr_read_probe": (_I32, [_VP, ctypes.c_int64, _I32, _VP, _I32, _VP]),
    "xr_fma_probe": (_I32, [_I32, _VP, _I32, ctypes.POINTER(ctypes.c_int64), _VP]),
    "xr_project_batched": (_I32, [ctypes.POINTER(_Problem), _I32, _VP]),
    "xr_backproject_batched": (_I32, [ctypes.POINTER(_Problem), _I32, _VP]),
    "xr_tune": (_I32, [_VP, ctypes.c_char_p]),
    "xr_get_device_error": (_I32, [_VP, ctypes.POINTER(_I32)]),
    "xr_wait_bound_selftest": (_I32, [ctypes.c_int64, ctypes.POINTER(_I32)]),
    "xr_project_attenuated": (_I32, [_VP, _VP, _VP, _VP, _I32, _VP]),
    "xr_backproject_attenuated": (_I32, [_VP, _VP, _VP, _VP, _I32, _VP]),
    "xr_status_string": (ctypes.c_char_p, [_I32]),
    "xr_last_cuda_error": (_I32, []),
    "xr_version": (_I32, []),
}

_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise XRayError(f"{LIB_PATH} is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int, what: str):
    if status != 0:
        msg = lib().xr_status_string(status).decode()
        if status == 6:
            msg += f" (cudaError {lib().xr_last_cuda_error()})"
        raise XRayError(f"{what}: {msg}")


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def _need_cuda(t: torch.Tensor, name: str):
    if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise XRayError(f"{name} must be a contiguous float32 CUDA tensor")


def _need_out(t: torch.Tensor, shape: tuple, name: str):
    """An output buffer: a contiguous float32 CUDA tensor holding exactly prod(shape) floats
    (the kernels write that many)."""
    _need_cuda(t, name)
    if t.numel() != int(np.prod(shape)):
        raise XRayError(f"{name} has {t.numel()} elements, expected {int(np.prod(shape))} (shape {tuple(shape)})")


def _desc(geom: Geometry):
    """The C description of a scan and the arrays it points into (keep them alive)."""
    angles = np.ascontiguousarray(np.asarray(geom.angles, dtype=np.float64).reshape(-1))
    src_z = None if geom.src_z is None else np.ascontiguousarray(geom.src_z, dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    d = _Desc(KINDS[geom.kind], geom.nx, geom.ny, geom.nz, geom.dx, geom.dy, geom.dz, geom.cx, geom.cy,
              geom.cz, geom.n_views, geom.n_rows, geom.n_cols, angles.ctypes.data_as(dp),
              None if src_z is None else src_z.ctypes.data_as(dp),
              geom.du, geom.dv, geom.u0, geom.v0, geom.sod, geom.sdd)
    return d, angles, src_z


def column_batch_plan(geom: Geometry):
    """(eligible, slice_of): whether the library runs this scan as 2D column problems, and the
    y-slice of each detector column (-1 outside the volume).  Host only: needs no GPU."""
    d, _angles, _src_z = _desc(geom)
    out = np.full(max(geom.n_cols, 1), -1, dtype=np.int32)
    ok = ctypes.c_int32(0)
    _check(lib().xr_column_batch_plan(ctypes.byref(d), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                      ctypes.byref(ok)), "xr_column_batch_plan")
    return bool(ok.value), out[:geom.n_cols]


class Projector:
    """X-ray transform and adjoint of one scan on the current CUDA device."""

    def __init__(self, geom: Geometry):
        if not torch.cuda.is_available():
            raise XRayError("no CUDA device: the X-ray transform runs only on the GPU")
        self.geom = geom
        d, self._angles, self._src_z = _desc(geom)
        h = ctypes.c_void_p()
        torch.cuda.current_device()  # make sure the CUDA context exists
        _check(lib().xr_geometry_create(ctypes.byref(d), ctypes.byref(h)), "xr_geometry_create")
        self._h = h
        info = _Info()
        _check(lib().xr_geometry_get_info(h, ctypes.byref(info)), "xr_geometry_get_info")
        self.n_rays, self.n_units = int(info.n_rays), int(info.n_units)
        self.table_bytes = int(info.table_bytes)
        self.column_batch = bool(info.column_batch)  # single-tilt-axis scan run as 2D column problems
        self.trace_walk = bool(info.trace_walk)  # cone / helical scan the column-trace walk applies to
        self.device = torch.device("cuda", int(info.device))
        self.reserved = 0
        self.auto_reserve = True

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().xr_geometry_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- tuning ---------------------------------------------------------------------------
    def set_tuning(self, block: int = 0, batch_chunk: int = 0, adjoint: int = 0, path: int = 0, order: int = 0):
        t = _Tuning(block, batch_chunk, adjoint, path, order)
        _check(lib().xr_set_tuning(self._h, ctypes.byref(t)), "xr_set_tuning")

    def tuning(self) -> dict:
        t = _Tuning()
        _check(lib().xr_get_tuning(self._h, ctypes.byref(t)), "xr_get_tuning")
        return {"block": t.block, "batch_chunk": t.batch_chunk, "adjoint": t.adjoint, "path": t.path,
                "order": t.order}

    def tune(self, cache_path: str | None = None) -> dict:
        """Time the candidate tunings in the library (xr_tune) for the reserved batch size and
        keep the fastest; cache_path: a text cache shared across processes."""
        _check(lib().xr_tune(self._h, None if cache_path is None else os.fsencode(cache_path)), "xr_tune")
        return self.tuning()

    def device_error(self) -> int:
        """The handle's device error word since the last call (0: none), then cleared."""
        code = ctypes.c_int32(0)
        _check(lib().xr_get_device_error(self._h, ctypes.byref(code)), "xr_get_device_error")
        return int(code.value)

    def reserve(self, max_batch: int):
        """Reserve the batched fast path's workspace (allocates; not during graph capture)."""
        _check(lib().xr_reserve(self._h, int(max_batch)), "xr_reserve")
        self.reserved = int(max_batch)

    def ray_setup(self, stream=None):
        _check(lib().xr_ray_setup(self._h, _stream(stream)), "xr_ray_setup")

    # -- operators ------------------------------------------------------------------------
    def _here(self, *named):
        """Every (tensor, name) pair lives on the projector's device (kernels run there)."""
        for t, name in named:
            if t.device != self.device:
                raise XRayError(f"{name} is on {t.device}, the projector on {self.device}")

    def _batch_of(self, t: torch.Tensor, unit_shape: tuple, name: str) -> int:
        """0 for one unbatched image or sinogram, else the batch size (an empty batch raises)."""
        if tuple(t.shape) == unit_shape:
            return 0
        if t.dim() == len(unit_shape) + 1 and tuple(t.shape[1:]) == unit_shape:
            if t.shape[0] < 1:
                raise XRayError(f"{name} is an empty batch")
            return int(t.shape[0])
        raise XRayError(f"{name} has shape {tuple(t.shape)}, expected {unit_shape} or (B,)+{unit_shape}")

    def _maybe_reserve(self, b: int):
        if not self.auto_reserve or torch.cuda.is_current_stream_capturing():
            return
        if self.geom.is3d or b < 4:
            if self.reserved < 1:  # one image copy: the single-image path
                self.reserve(1)
        elif b > self.reserved:
            self.reserve(b)

    def forward(self, img: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        _need_cuda(img, "img")
        b = self._batch_of(img, self.geom.image_shape(), "img")
        self._maybe_reserve(b)
        shape = self.geom.sino_shape(b if b else None)
        if out is None:
            out = torch.empty(shape, device=img.device, dtype=torch.float32)
        _need_out(out, shape, "out")
        self._here((img, "img"), (out, "out"))
        _check(lib().xr_project(self._h, _ptr(img), _ptr(out), max(b, 1), _stream(stream)), "xr_project")
        return out

    def adjoint(self, sino: torch.Tensor, out: torch.Tensor | None = None, method: int = XR_ADJ_AUTO,
                stream=None) -> torch.Tensor:
        _need_cuda(sino, "sino")
        b = self._batch_of(sino, self.geom.sino_shape(), "sino")
        self._maybe_reserve(b)
        shape = self.geom.image_shape(b if b else None)
        if out is None:
            out = torch.empty(shape, device=sino.device, dtype=torch.float32)
        _need_out(out, shape, "out")
        self._here((sino, "sino"), (out, "out"))
        _check(lib().xr_backproject_method(self._h, _ptr(sino), _ptr(out), max(b, 1), int(method),
                                           _stream(stream)), "xr_backproject")
        return out

    def forward_adjoint(self, img: torch.Tensor, sino_out: torch.Tensor | None = None,
                        img_out: torch.Tensor | None = None, stream=None):
        """Both operators in one launch (xr_project_backproject): returns (sino, img_out) with
        sino = A img and img_out = A^T sino, for problems too small to fill the GPU."""
        _need_cuda(img, "img")
        b = self._batch_of(img, self.geom.image_shape(), "img")
        if sino_out is None:
            sino_out = torch.empty(self.geom.sino_shape(b if b else None), device=img.device, dtype=torch.float32)
        if img_out is None:
            img_out = torch.empty(self.geom.image_shape(b if b else None), device=img.device, dtype=torch.float32)
        _need_out(sino_out, self.geom.sino_shape(b if b else None), "sino_out")
        _need_out(img_out, self.geom.image_shape(b if b else None), "img_out")
        self._here((img, "img"), (sino_out, "sino_out"), (img_out, "img_out"))
        _check(lib().xr_project_backproject(self._h, _ptr(img), _ptr(sino_out), _ptr(img_out), max(b, 1),
                                            _stream(stream)), "xr_project_backproject")
        return sino_out, img_out

    __call__ = forward

    def forward_attenuated(self, img: torch.Tensor, mu: torch.Tensor, out: torch.Tensor | None = None,
                           stream=None) -> torch.Tensor:
        """Attenuated transform (exponential attenuation of the map ``mu`` towards each ray's
        far end) of one image or a batch."""
        _need_cuda(img, "img")
        _need_cuda(mu, "mu")
        if tuple(mu.shape) != self.geom.image_shape():
            raise XRayError(f"mu has shape {tuple(mu.shape)}, expected {self.geom.image_shape()}")
        b = self._batch_of(img, self.geom.image_shape(), "img")
        self._maybe_reserve(b)
        shape = self.geom.sino_shape(b if b else None)
        if out is None:
            out = torch.empty(shape, device=img.device, dtype=torch.float32)
        _need_out(out, shape, "out")
        self._here((img, "img"), (mu, "mu"), (out, "out"))
        _check(lib().xr_project_attenuated(self._h, _ptr(mu), _ptr(img), _ptr(out), max(b, 1), _stream(stream)),
               "xr_project_attenuated")
        return out

    def adjoint_attenuated(self, sino: torch.Tensor, mu: torch.Tensor, out: torch.Tensor | None = None,
                           stream=None) -> torch.Tensor:
        """The exact transpose of forward_attenuated."""
        _need_cuda(sino, "sino")
        _need_cuda(mu, "mu")
        if tuple(mu.shape) != self.geom.image_shape():
            raise XRayError(f"mu has shape {tuple(mu.shape)}, expected {self.geom.image_shape()}")
        b = self._batch_of(sino, self.geom.sino_shape(), "sino")
        self._maybe_reserve(b)
        shape = self.geom.image_shape(b if b else None)
        if out is None:
            out = torch.empty(shape, device=sino.device, dtype=torch.float32)
        _need_out(out, shape, "out")
        self._here((sino, "sino"), (mu, "mu"), (out, "out"))
        _check(lib().xr_backproject_attenuated(self._h, _ptr(mu), _ptr(sino), _ptr(out), max(b, 1),
                                               _stream(stream)), "xr_backproject_attenuated")
        return out

    def ray_units(self, rays, cap: int | None = None):
        """Sparse rows for the given ray ids: list of (unit indices int64, lengths float32)
        per ray, in visiting order."""
        rays_t = torch.as_tensor(np.asarray(rays, dtype=np.int64), device=self.device)
        n = int(rays_t.numel())
        cap = cap or (self.geom.nx + self.geom.ny + self.geom.nz) * 3 + 8
        idx = torch.empty((n, cap), dtype=torch.int64, device=self.device)
        ln = torch.empty((n, cap), dtype=torch.float32, device=self.device)
        cnt = torch.empty((n,), dtype=torch.int32, device=self.device)
        _check(lib().xr_ray_units(self._h, _ptr(rays_t), n, cap, _ptr(idx), _ptr(ln), _ptr(cnt), _stream()),
               "xr_ray_units")
        cnt_h, idx_h, ln_h = cnt.cpu().numpy(), idx.cpu().numpy(), ln.cpu().numpy()
        if (cnt_h < 0).any():
            raise XRayError("ray_units: ray id outside the scan")
        if (cnt_h > cap).any():
            raise XRayError("ray_units: cap too small")
        return [(idx_h[q, :cnt_h[q]], ln_h[q, :cnt_h[q]]) for q in range(n)]


    def system_rows(self, ray0: int = 0, n: int | None = None, stream=None):
        """CSR rows of the projection matrix for rays [ray0, ray0 + n): (row_ptr int64 [n + 1],
        col int64 [nnz] (1D unit index), val float32 [nnz] (length)), device tensors; each row in
        the order the ray crosses its units.  Synchronises once to size the outputs."""
        n = self.n_rays - ray0 if n is None else int(n)
        ptr = torch.empty((n + 1,), dtype=torch.int64, device=self.device)
        _check(lib().xr_system_rows_count(self._h, int(ray0), n, _ptr(ptr), _stream(stream)),
               "xr_system_rows_count")
        nnz = int(ptr[-1].item())
        col = torch.empty((max(nnz, 1),), dtype=torch.int64, device=self.device)
        val = torch.empty((max(nnz, 1),), dtype=torch.float32, device=self.device)
        _check(lib().xr_system_rows_fill(self._h, int(ray0), n, _ptr(ptr), _ptr(col), _ptr(val), _stream(stream)),
               "xr_system_rows_fill")
        return ptr, col[:nnz], val[:nnz]


class XRayFunction(torch.autograd.Function):
    """y = A x with dA^T: backward is the adjoint kernel on the incoming gradient; nothing
    is saved for backward beyond the projector (lengths are recomputed)."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, proj: Projector):
        ctx.proj = proj
        return proj.forward(x.contiguous())

    @staticmethod
    def backward(ctx, gy: torch.Tensor):
        return ctx.proj.adjoint(gy.contiguous()), None


def project(x: torch.Tensor, proj: Projector) -> torch.Tensor:
    """Differentiable forward projection."""
    return XRayFunction.apply(x, proj)


class AttenuatedXRayFunction(torch.autograd.Function):
    """y = A_mu x (the attenuated transform for a fixed attenuation map mu); backward is its
    transpose on the incoming gradient."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, mu: torch.Tensor, proj: Projector):
        ctx.proj, ctx.mu = proj, mu
        return proj.forward_attenuated(x.contiguous(), mu)

    @staticmethod
    def backward(ctx, gy: torch.Tensor):
        return ctx.proj.adjoint_attenuated(gy.contiguous(), ctx.mu), None, None


def project_attenuated(x: torch.Tensor, mu: torch.Tensor, proj: Projector) -> torch.Tensor:
    """Differentiable attenuated forward projection (gradient with respect to x)."""
    return AttenuatedXRayFunction.apply(x, mu, proj)


class BatchPlan:
    """One persistent launch over many independent (uneven) problems."""

    def __init__(self, projectors, images, sinos, tile: int = 0, block: int = 0):
        n = len(projectors)
        if not (len(images) == len(sinos) == n) or n == 0:
            raise XRayError("BatchPlan needs one image and one sinogram per projector")
        arr = (_Problem * n)()
        for q, (p, x, y) in enumerate(zip(projectors, images, sinos)):
            _need_cuda(x, "img")
            _need_cuda(y, "sino")
            if x.numel() != p.n_units or y.numel() != p.n_rays:
                raise XRayError(f"problem {q}: buffer sizes do not match its geometry")
            p._here((x, f"problem {q} img"), (y, f"problem {q} sino"))
            arr[q] = _Problem(p.handle.value, x.data_ptr(), y.data_ptr())
        self._keep = (list(projectors), list(images), list(sinos))
        h = ctypes.c_void_p()
        _check(lib().xr_batch_create(arr, n, int(tile), int(block), ctypes.byref(h)), "xr_batch_create")
        self._h = h

    def ray_setup(self, stream=None):
        """Every problem's ray setup (detector and ray tables) in two launches."""
        _check(lib().xr_batch_ray_setup(self._h, _stream(stream)), "xr_batch_ray_setup")

    def project(self, stream=None):
        _check(lib().xr_batch_project(self._h, _stream(stream)), "xr_batch_project")

    def backproject(self, stream=None):
        _check(lib().xr_batch_backproject(self._h, _stream(stream)), "xr_batch_backproject")

    def close(self):
        if getattr(self, "_h", None):
            lib().xr_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wait_bound_selftest(cycles: int = 2_000_000) -> bool:
    """True when the library's bounded wait on an mbarrier that nothing completes gave up
    after `cycles` SM clock cycles (xr_wait_bound_selftest)."""
    out = _I32(-1)
    _check(lib().xr_wait_bound_selftest(int(cycles), ctypes.byref(out)), "xr_wait_bound_selftest")
    return out.value == 1


def read_bandwidth(n_bytes: int = 64 << 20, reps: int = 20, trials: int = 5) -> float:
    """Measured read bandwidth (GB/s) of a device buffer of n_bytes read `reps` times per
    launch (the L2 read bandwidth when the buffer fits L2): best of `trials` event-timed
    launches after one warm-up."""
    n = (n_bytes // 16) * 4
    buf = torch.ones(n, device="cuda")
    sink = torch.empty(1 << 22, device="cuda")
    stream = torch.cuda.current_stream()

    def launch():
        _check(lib().xr_read_probe(_ptr(buf), n, reps, _ptr(sink), sink.numel(), _stream(stream)), "xr_read_probe")

    launch()
    best = 0.0
    for _ in range(trials):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        launch()
        b.record(stream)
        b.synchronize()
        best = max(best, 4.0 * n * reps / (a.elapsed_time(b) * 1e-3) / 1e9)
    return best


def fma_throughput(iters: int = 20000, trials: int = 5) -> float:
    """Measured FP32 FMA throughput (TFLOP/s, 2 FLOP per FMA): best of `trials` event-timed
    launches of xr_fma_probe after one warm-up."""
    sink = torch.empty(1 << 22, device="cuda")
    stream = torch.cuda.current_stream()
    flop = ctypes.c_int64(0)

    def launch():
        _check(lib().xr_fma_probe(iters, _ptr(sink), sink.numel(), ctypes.byref(flop), _stream(stream)),
               "xr_fma_probe")

    launch()
    best = 0.0
    for _ in range(trials):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        launch()
        b.record(stream)
        b.synchronize()
        best = max(best, flop.value / (a.elapsed_time(b) * 1e-3) / 1e12)
    return best

