"""Thin ctypes binding of ``libtaylorgrid.so`` (the C ABI in include/taylorgrid.h).

Argument marshalling only: every step of the TaylorGrid path runs in the
library's CUDA kernels. Tensors are torch CUDA tensors used as device memory;
the stream is torch's current stream unless one is given. There is no CPU
fallback: without the built library or a CUDA device every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtaylorgrid.so")

TG_F32, TG_BF16, TG_F16 = 0, 1, 2
TG_ORDER_INPUT, TG_ORDER_BINNED = 0, 1
TG_DETERMINISTIC = 2
DTYPES = {"f32": TG_F32, "fp32": TG_F32, "float32": TG_F32, "bf16": TG_BF16, "bfloat16": TG_BF16,
          "f16": TG_F16, "fp16": TG_F16, "float16": TG_F16}
STATUS = {0: "TG_OK", 1: "TG_EINVAL", 2: "TG_ENOMEM", 3: "TG_EBUDGET", 4: "TG_ETIMEOUT", 5: "TG_EDEVICE",
          6: "TG_ENOTFOUND", 7: "TG_EBUSY"}

_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int


class TGError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class GridInfo(ctypes.Structure):
    _fields_ = [("dim", _int), ("res", _int), ("order", _int), ("channels", _int), ("K", _int),
                ("dtype", _int), ("n_vertices", _i64), ("n_coefs", _i64), ("bytes", ctypes.c_size_t),
                ("coefs", _vp), ("master", _vp)]


class ShapeStruct(ctypes.Structure):
    _fields_ = [("n_spheres", _int), ("n_boxes", _int), ("spheres", _vp), ("boxes", _vp), ("area_cdf", _vp)]


class FitDesc(ctypes.Structure):
    _fields_ = [("res", _int), ("order", _int), ("dtype", _int), ("seed", ctypes.c_uint64),
                ("n_spheres", _int), ("n_boxes", _int), ("spheres", _vp), ("boxes", _vp), ("area_cdf", _vp),
                ("points_per_step", _i64), ("eval_points", _i64), ("eval_every", _int), ("max_steps", _int),
                ("tol", ctypes.c_float), ("lr", ctypes.c_float), ("lambda_eik", ctypes.c_float),
                ("init_std", ctypes.c_float), ("k_weight", ctypes.c_float), ("lambda_tv", ctypes.c_float),
                ("flags", _int)]


class JobResult(ctypes.Structure):
    _fields_ = [("state", _int), ("kind", _int), ("steps", _i64), ("error", ctypes.c_float),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_done", ctypes.c_double),
                ("points", _i64), ("bytes", ctypes.c_size_t)]


class AdamParams(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("step", _i64)]


# name -> argtypes (restype is tg_status = int unless noted)
_SIGS = {
    "tg_create": [_int, _int, _int, _int, _int, ctypes.c_uint64, ctypes.c_float, ctypes.POINTER(_vp)],
    "tg_destroy": [_vp],
    "tg_get_info": [_vp, ctypes.POINTER(GridInfo)],
    "tg_set_coefs": [_vp, _vp, _vp],
    "tg_get_coefs": [_vp, _vp, _int, _vp],
    "tg_locate": [_int, _int, _vp, _i64, _vp, _vp, _vp],
    "tg_query": [_vp, _vp, _i64, _vp, _vp, _vp],
    "tg_query_backward": [_vp, _vp, _i64, _vp, _vp, _vp, _vp],
    "tg_batch_create": [_int, _int, _i64, ctypes.POINTER(_vp)],
    "tg_batch_destroy": [_vp],
    "tg_batch_bin": [_vp, _vp, _i64, _vp],
    "tg_query_binned": [_vp, _vp, _vp, _vp, _int, _vp],
    "tg_query_backward_binned": [_vp, _vp, _vp, _vp, _vp, _int, _vp],
    "tg_batch_order": [_vp, _vp, _vp],
    "tg_batch_points": [_vp, _vp, _vp],
    "tg_batch_timeouts": [_vp, ctypes.POINTER(_int)],
    "tg_grid_timeouts": [_vp, ctypes.POINTER(_int)],
    "tg_inject_alloc_failures": [_int, _int],
    "tg_measure_fp32_peak": [ctypes.POINTER(ctypes.c_double)],
    "tg_noalloc_timeouts": [ctypes.POINTER(_int)],
    "tg_batch_gather": [_vp, _vp, _int, _vp, _vp],
    "tg_batch_scatter": [_vp, _vp, _int, _vp, _vp],
    "tg_query_noalloc": [_vp, _vp, _i64, _vp, _vp, _vp],
    "tg_adam_step": [_vp, _vp, ctypes.POINTER(AdamParams), _vp],
    "tg_adam_step_lazy": [_vp, _vp, ctypes.POINTER(AdamParams), _vp],
    "tg_sdf_eval_target": [ctypes.POINTER(ShapeStruct), _vp, _i64, _vp, _vp],
    "tg_sample_sdf_points": [ctypes.POINTER(ShapeStruct), ctypes.c_uint64, _i64, _i64, ctypes.c_float, _vp, _vp],
    "tg_sdf_step": [_vp, _vp, ctypes.POINTER(ShapeStruct), _vp, _i64, ctypes.c_uint64, _i64, ctypes.c_float,
                    ctypes.c_float, _vp, _vp, _vp],
    "tg_tv_step": [_vp, ctypes.c_float, _vp, _vp, _vp],
    "tg_sdf_error": [_vp, ctypes.POINTER(ShapeStruct), _vp, _i64, _vp, _vp],
    "tg_sdf_iou": [_vp, ctypes.POINTER(ShapeStruct), _vp, _i64, _vp, _vp],
    "tg_extract_mesh": [_vp, _int, ctypes.c_float, _vp, _i64, _vp, _vp],
    "tg_sample_mesh": [_vp, _vp, _i64, _i64, ctypes.c_uint64, _vp, _vp],
    "tg_chamfer": [_vp, _i64, _vp, _i64, _vp, _vp],
    "tg_save": [_vp, ctypes.c_char_p],
    "tg_resample": [_vp, _vp, _vp],
    "tg_load": [ctypes.c_char_p, ctypes.POINTER(_vp)],
    "tg_server_create": [ctypes.c_size_t, _int, ctypes.POINTER(_vp)],
    "tg_server_destroy": [_vp],
    "tg_fit_job": [_vp, ctypes.POINTER(FitDesc), ctypes.POINTER(_i64)],
    "tg_query_job": [_vp, _i64, _vp, _i64, _vp, ctypes.POINTER(_i64)],
    "tg_server_step": [_vp, ctypes.POINTER(_int)],
    "tg_poll": [_vp, _i64, ctypes.POINTER(JobResult)],
    "tg_server_grid": [_vp, _i64, ctypes.POINTER(_vp)],
    "tg_release": [_vp, _i64],
    "tg_cancel": [_vp, _i64],
    "tg_server_set_policy": [_vp, _int],
    "tg_render_rays": [_vp, _vp, _vp, _vp, _i64, _int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_float, _vp, _vp,
                       _vp, _vp, _vp, _vp, _vp],
    "tg_render_rays_backward": [_vp, _vp, _vp, _vp, _i64, _int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_float,
                                _vp, _vp, _vp, _vp, _vp, _vp],
}


def exported_symbols() -> list[str]:
    return list(_SIGS) + ["tg_status_string", "tg_last_error", "tg_server_time"]


def load():
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = _int
        L.tg_status_string.argtypes = [_int]; L.tg_status_string.restype = ctypes.c_char_p
        L.tg_last_error.argtypes = []; L.tg_last_error.restype = ctypes.c_char_p
        L.tg_server_time.argtypes = [_vp]; L.tg_server_time.restype = ctypes.c_double
        _lib = L
        return L


def _check(status: int, where: str):
    if status != 0:
        raise TGError(status, where, (load().tg_last_error() or b"").decode())


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t, name, dtype=torch.float32, numel=None, optional=False):
    if t is None:
        if optional:
            return None
        raise ValueError(f"{name} is required")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (the TaylorGrid library has no CPU path)")
    if t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {dtype} tensor")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements, needs {numel}")
    return t.data_ptr()


class Grid:
    """Owning handle of a tg_grid (freed by close() or garbage collection)."""

    def __init__(self, handle: int):
        self._h = handle
        info = GridInfo()
        _check(load().tg_get_info(handle, ctypes.byref(info)), "tg_get_info")
        self.dim, self.res, self.order, self.channels, self.K = info.dim, info.res, info.order, info.channels, info.K
        self.dtype = info.dtype
        self.n_vertices, self.n_coefs = info.n_vertices, info.n_coefs

    @property
    def handle(self) -> int:
        if not self._h:
            raise ValueError("grid is closed")
        return self._h

    def info(self) -> GridInfo:
        info = GridInfo()
        _check(load().tg_get_info(self.handle, ctypes.byref(info)), "tg_get_info")
        return info

    def close(self):
        if getattr(self, "_h", None):
            load().tg_destroy(self._h)
            self._h = None

    __del__ = close


def tg_create(dim: int, res: int, order: int, channels: int = 1, dtype="f32", seed: int = 0,
              init_std: float = 0.0) -> Grid:
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    h = _vp()
    _check(load().tg_create(dim, res, order, channels, dt, seed, init_std, ctypes.byref(h)), "tg_create")
    return Grid(h.value)


def tg_set_coefs(grid: Grid, coefs: torch.Tensor, stream=None):
    _check(load().tg_set_coefs(grid.handle, _ptr(coefs, "coefs", numel=grid.n_coefs), _stream(stream)), "tg_set_coefs")


def tg_get_coefs(grid: Grid, out: torch.Tensor | None = None, which: int = 0, stream=None) -> torch.Tensor:
    if out is None:
        out = torch.empty(grid.n_coefs, device="cuda", dtype=torch.float32)
    _check(load().tg_get_coefs(grid.handle, _ptr(out, "out", numel=grid.n_coefs), which, _stream(stream)), "tg_get_coefs")
    return out


def tg_locate(dim: int, res: int, pts: torch.Tensor, stream=None):
    """Cells (N, dim) int32 and local coordinates (N, dim) float32 of Eq. 2."""
    N = pts.shape[0]
    cells = torch.empty((N, dim), device=pts.device, dtype=torch.int32)
    t = torch.empty((N, dim), device=pts.device, dtype=torch.float32)
    _check(load().tg_locate(dim, res, _ptr(pts, "pts", numel=N * dim), N, _ptr(cells, "cells", torch.int32),
                            _ptr(t, "t"), _stream(stream)), "tg_locate")
    return cells, t


def tg_query(grid: Grid, pts: torch.Tensor, out=None, grad_x=None, want_grad=False, stream=None):
    N = pts.shape[0]
    if out is None:
        out = torch.empty((N, grid.channels), device=pts.device, dtype=torch.float32)
    if grad_x is None and want_grad:
        grad_x = torch.empty((N, grid.channels, grid.dim), device=pts.device, dtype=torch.float32)
    _check(load().tg_query(grid.handle, _ptr(pts, "pts", numel=N * grid.dim), N,
                           _ptr(out, "out", numel=N * grid.channels),
                           _ptr(grad_x, "grad_x", numel=N * grid.channels * grid.dim, optional=True),
                           _stream(stream)), "tg_query")
    return (out, grad_x) if (want_grad or grad_x is not None) else out


def tg_query_backward(grid: Grid, pts, dL_df, coef_grad, dL_dgradx=None, stream=None):
    N = pts.shape[0]
    _check(load().tg_query_backward(grid.handle, _ptr(pts, "pts", numel=N * grid.dim), N,
                                    _ptr(dL_df, "dL_df", numel=N * grid.channels),
                                    _ptr(dL_dgradx, "dL_dgradx", numel=N * grid.channels * grid.dim, optional=True),
                                    _ptr(coef_grad, "coef_grad", numel=grid.n_coefs), _stream(stream)),
           "tg_query_backward")
    return coef_grad


class Batch:
    """Owning handle of a tg_batch (binned point batch)."""

    def __init__(self, dim: int, res: int, max_points: int):
        h = _vp()
        _check(load().tg_batch_create(dim, res, max_points, ctypes.byref(h)), "tg_batch_create")
        self._h = h.value
        self.dim, self.res, self.max_points, self.n = dim, res, max_points, 0

    @property
    def handle(self):
        if not self._h:
            raise ValueError("batch is closed")
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            load().tg_batch_destroy(self._h)
            self._h = None

    __del__ = close


def tg_batch_create(dim: int, res: int, max_points: int) -> Batch:
    return Batch(dim, res, max_points)


def tg_batch_bin(batch: Batch, pts: torch.Tensor, stream=None):
    N = pts.shape[0]
    _check(load().tg_batch_bin(batch.handle, _ptr(pts, "pts", numel=N * batch.dim), N, _stream(stream)), "tg_batch_bin")
    batch.n = N
    return batch


def tg_query_binned(grid: Grid, batch: Batch, out=None, grad_x=None, want_grad=False, binned_order=False,
                    stream=None):
    N = batch.n
    dev = torch.device("cuda")
    if out is None:
        out = torch.empty((N, grid.channels), device=dev, dtype=torch.float32)
    if grad_x is None and want_grad:
        grad_x = torch.empty((N, grid.channels, grid.dim), device=dev, dtype=torch.float32)
    _check(load().tg_query_binned(grid.handle, batch.handle, _ptr(out, "out", numel=N * grid.channels),
                                  _ptr(grad_x, "grad_x", numel=N * grid.channels * grid.dim, optional=True),
                                  TG_ORDER_BINNED if binned_order else TG_ORDER_INPUT, _stream(stream)),
           "tg_query_binned")
    return (out, grad_x) if (want_grad or grad_x is not None) else out


def tg_query_backward_binned(grid: Grid, batch: Batch, dL_df, coef_grad, dL_dgradx=None, binned_order=False,
                             deterministic=False, stream=None):
    N = batch.n
    flags = (TG_ORDER_BINNED if binned_order else TG_ORDER_INPUT) | (TG_DETERMINISTIC if deterministic else 0)
    _check(load().tg_query_backward_binned(grid.handle, batch.handle, _ptr(dL_df, "dL_df", numel=N * grid.channels),
                                           _ptr(dL_dgradx, "dL_dgradx", numel=N * grid.channels * grid.dim,
                                                optional=True),
                                           _ptr(coef_grad, "coef_grad", numel=grid.n_coefs), flags, _stream(stream)),
           "tg_query_backward_binned")
    return coef_grad


def tg_batch_order(batch: Batch, stream=None) -> torch.Tensor:
    """Original index of every binned slot (int32, N)."""
    idx = torch.empty(batch.n, device="cuda", dtype=torch.int32)
    _check(load().tg_batch_order(batch.handle, _ptr(idx, "idx", torch.int32) if batch.n else None, _stream(stream)),
           "tg_batch_order")
    return idx


def tg_batch_points(batch: Batch, stream=None) -> torch.Tensor:
    """The binned points in binned order (N, 3)."""
    pts = torch.empty((batch.n, 3), device="cuda", dtype=torch.float32)
    _check(load().tg_batch_points(batch.handle, _ptr(pts, "pts") if batch.n else None, _stream(stream)),
           "tg_batch_points")
    return pts


def _permute_rows(fn: str, batch: Batch, src: torch.Tensor, dst, stream):
    N = batch.n
    width = src.numel() // N if N else (src.shape[1] if src.dim() > 1 else 1)
    if N and src.numel() != N * width:
        raise ValueError(f"{fn}: src has {src.numel()} elements, not a multiple of N = {N}")
    if dst is None:
        dst = torch.empty_like(src)
    _check(getattr(load(), fn)(batch.handle, _ptr(src, "src", numel=N * width) if N else None, width,
                               _ptr(dst, "dst", numel=N * width) if N else None, _stream(stream)), fn)
    return dst


def tg_batch_gather(batch: Batch, src: torch.Tensor, dst=None, stream=None) -> torch.Tensor:
    """Rows of an input-order per-point array in binned order: dst[p] = src[idx[p]]."""
    return _permute_rows("tg_batch_gather", batch, src, dst, stream)


def tg_batch_scatter(batch: Batch, src: torch.Tensor, dst=None, stream=None) -> torch.Tensor:
    """Rows of a binned-order per-point array back in input order: dst[idx[p]] = src[p]."""
    return _permute_rows("tg_batch_scatter", batch, src, dst, stream)


def tg_batch_timeouts(batch: Batch) -> int:
    v = _int(0)
    _check(load().tg_batch_timeouts(batch.handle, ctypes.byref(v)), "tg_batch_timeouts")
    return v.value


def tg_measure_fp32_peak() -> float:
    """Measured FP32 FMA throughput of the current device in TFLOP/s (the ALU roofline's denominator)."""
    v = ctypes.c_double()
    _check(load().tg_measure_fp32_peak(ctypes.byref(v)), "tg_measure_fp32_peak")
    return v.value


def tg_inject_alloc_failures(pass_: int, fail: int) -> None:
    """Test hook: the next `pass_` device allocations of the library succeed, the `fail` after them report
    TG_ENOMEM (host-side; no GPU fault). fail = 0 switches injection off."""
    _check(load().tg_inject_alloc_failures(int(pass_), int(fail)), "tg_inject_alloc_failures")


def tg_grid_timeouts(grid: Grid) -> int:
    """Non-zero if a bounded TMA wait of a binned call made by tg_query / tg_query_backward gave up (clears it)."""
    v = _int(0)
    _check(load().tg_grid_timeouts(grid.handle, ctypes.byref(v)), "tg_grid_timeouts")
    return v.value


def tg_noalloc_timeouts() -> int:
    """Non-zero if a bounded TMA wait of a tg_query_noalloc call on the current device gave up (clears it)."""
    v = _int(0)
    _check(load().tg_noalloc_timeouts(ctypes.byref(v)), "tg_noalloc_timeouts")
    return v.value


def tg_query_noalloc(grid: Grid, pts: torch.Tensor, out=None, grad_x=None, want_grad=False, stream=None):
    """Binned forward query served entirely from the library's fixed scratch array (no allocation)."""
    N = pts.shape[0]
    if out is None:
        out = torch.empty((N, grid.channels), device=pts.device, dtype=torch.float32)
    if grad_x is None and want_grad:
        grad_x = torch.empty((N, grid.channels, grid.dim), device=pts.device, dtype=torch.float32)
    _check(load().tg_query_noalloc(grid.handle, _ptr(pts, "pts", numel=N * grid.dim), N,
                                   _ptr(out, "out", numel=N * grid.channels),
                                   _ptr(grad_x, "grad_x", numel=N * grid.channels * grid.dim, optional=True),
                                   _stream(stream)), "tg_query_noalloc")
    return (out, grad_x) if (want_grad or grad_x is not None) else out


def tg_adam_step(grid: Grid, coef_grad, lr: float, step: int, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    prm = AdamParams(lr, beta1, beta2, eps, step)
    _check(load().tg_adam_step(grid.handle, _ptr(coef_grad, "coef_grad", numel=grid.n_coefs), ctypes.byref(prm),
                               _stream(stream)), "tg_adam_step")


def tg_adam_step_lazy(grid: Grid, coef_grad, lr: float, step: int, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    prm = AdamParams(lr, beta1, beta2, eps, step)
    _check(load().tg_adam_step_lazy(grid.handle, _ptr(coef_grad, "coef_grad", numel=grid.n_coefs),
                                    ctypes.byref(prm), _stream(stream)), "tg_adam_step_lazy")


class DeviceShape:
    """A union of spheres (S, 4) and boxes (B, 6) in device memory, with its area CDF."""

    def __init__(self, spheres, boxes, area_cdf=None, device="cuda"):
        f = lambda a, w: torch.as_tensor(a, dtype=torch.float32).reshape(-1, w).contiguous().to(device)
        self.spheres = f(spheres, 4)
        self.boxes = f(boxes, 6)
        self.cdf = None if area_cdf is None else torch.as_tensor(area_cdf, dtype=torch.float32).contiguous().to(device)
        self.struct = ShapeStruct(self.spheres.shape[0], self.boxes.shape[0],
                                  self.spheres.data_ptr() if self.spheres.numel() else None,
                                  self.boxes.data_ptr() if self.boxes.numel() else None,
                                  None if self.cdf is None else self.cdf.data_ptr())


def tg_sdf_eval_target(shape: DeviceShape, pts, stream=None):
    d = torch.empty(pts.shape[0], device=pts.device, dtype=torch.float32)
    _check(load().tg_sdf_eval_target(ctypes.byref(shape.struct), _ptr(pts, "pts"), pts.shape[0], _ptr(d, "d"),
                                     _stream(stream)), "tg_sdf_eval_target")
    return d


def tg_sample_sdf_points(shape: DeviceShape, seed: int, step: int, n: int, jitter: float = 0.01, out=None,
                         stream=None):
    if out is None:
        out = torch.empty((n, 3), device="cuda", dtype=torch.float32)
    _check(load().tg_sample_sdf_points(ctypes.byref(shape.struct), seed, step, n, jitter, _ptr(out, "pts", numel=3 * n),
                                       _stream(stream)), "tg_sample_sdf_points")
    return out


def tg_sdf_step(grid: Grid, batch: Batch, shape: DeviceShape, coef_grad, loss_sums, pts=None, n=None, seed=0,
                step=0, lambda_eik=0.0, k_weight=0.0, stream=None):
    n = pts.shape[0] if pts is not None else n
    _check(load().tg_sdf_step(grid.handle, batch.handle, ctypes.byref(shape.struct),
                              None if pts is None else _ptr(pts, "pts", numel=3 * n), n, seed, step, lambda_eik,
                              k_weight, _ptr(coef_grad, "coef_grad", numel=grid.n_coefs),
                              _ptr(loss_sums, "loss_sums", numel=2), _stream(stream)), "tg_sdf_step")
    batch.n = n


def tg_tv_step(grid: Grid, lam: float, coef_grad, loss_sum=None, stream=None):
    """Adds lam * dL_TV/dtheta (Sec. 3.2's total variation term) into coef_grad; sum of n(v, c) into loss_sum."""
    _check(load().tg_tv_step(grid.handle, lam, _ptr(coef_grad, "coef_grad", numel=grid.n_coefs),
                             _ptr(loss_sum, "loss_sum", optional=True), _stream(stream)), "tg_tv_step")


def tg_sdf_error(grid: Grid, shape: DeviceShape, pts, err_sum=None, stream=None):
    if err_sum is None:
        err_sum = torch.zeros(1, device="cuda", dtype=torch.float32)
    _check(load().tg_sdf_error(grid.handle, ctypes.byref(shape.struct), _ptr(pts, "pts"), pts.shape[0],
                               _ptr(err_sum, "err_sum"), _stream(stream)), "tg_sdf_error")
    return err_sum


def tg_sdf_iou(grid: Grid, shape: DeviceShape, pts, stream=None) -> float:
    """Volumetric IoU of {f < 0} and {d < 0} over the points (synchronises to read the counts)."""
    counts = torch.zeros(2, device="cuda", dtype=torch.int64)
    _check(load().tg_sdf_iou(grid.handle, ctypes.byref(shape.struct), _ptr(pts, "pts"), pts.shape[0],
                             _ptr(counts, "counts", torch.int64), _stream(stream)), "tg_sdf_iou")
    inter, uni = counts.tolist()
    return inter / uni if uni else 1.0


def tg_extract_mesh(grid: Grid, M: int, iso: float = 0.0, max_tris=None, stream=None):
    """Triangles (T, 3, 3) of the level set f = iso of channel 0 on an M^3 lattice. Without max_tris a
    counting call sizes the buffer first (one read-back); with it, at most max_tris are kept and the full count
    is returned beside them: (tris, count)."""
    n = torch.zeros(1, device="cuda", dtype=torch.int64)
    if max_tris is None:
        _check(load().tg_extract_mesh(grid.handle, M, iso, None, 0, n.data_ptr(), _stream(stream)),
               "tg_extract_mesh")
        max_tris = int(n.item())
    tris = torch.empty((max(max_tris, 1), 3, 3), device="cuda")
    _check(load().tg_extract_mesh(grid.handle, M, iso, tris.data_ptr(), max_tris, n.data_ptr(), _stream(stream)),
           "tg_extract_mesh")
    count = int(n.item())
    return tris[:min(count, max_tris)], count


def tg_sample_mesh(tris, N: int, seed: int, stream=None):
    """N area-weighted points (N, 3) on the triangles (T, 3, 3)."""
    T = tris.shape[0]
    n = torch.tensor([T], device="cuda", dtype=torch.int64)
    pts = torch.empty((N, 3), device="cuda")
    _check(load().tg_sample_mesh(_ptr(tris, "tris") if T else None, n.data_ptr(), T, N, seed, pts.data_ptr(),
                                 _stream(stream)), "tg_sample_mesh")
    return pts


def tg_chamfer(A, B, stream=None):
    """(sum_a min_b |a - b|^2, sum_b min_a |a - b|^2) of two device point sets (synchronises)."""
    sums = torch.zeros(2, device="cuda", dtype=torch.float64)
    _check(load().tg_chamfer(_ptr(A, "A") if A.shape[0] else None, A.shape[0],
                             _ptr(B, "B") if B.shape[0] else None, B.shape[0],
                             _ptr(sums, "sums", torch.float64), _stream(stream)), "tg_chamfer")
    a, b = sums.tolist()
    return a, b


def tg_resample(src: Grid, dst: Grid, stream=None):
    """Re-expands src's field as dst's Taylor data (progressive resolution)."""
    _check(load().tg_resample(src.handle, dst.handle, _stream(stream)), "tg_resample")


def tg_save(grid: Grid, path: str):
    _check(load().tg_save(grid.handle, str(path).encode()), "tg_save")


def tg_load(path: str) -> Grid:
    h = _vp()
    _check(load().tg_load(str(path).encode(), ctypes.byref(h)), "tg_load")
    return Grid(h.value)


def tg_render_rays(density: Grid, color: Grid, rays_o, rays_d, S: int, seed: int = 0, ray_base: int = 0,
                   bg: float = 1.0, target=None, batch: Batch | None = None, density_grad=None, color_grad=None,
                   loss_sum=None, out=None, stream=None):
    """Eq. 10 rendering; with `target` also the Eq. 11 loss and both coefficient gradients."""
    R = rays_o.shape[0]
    if out is None:
        out = torch.empty((R, 3), device=rays_o.device, dtype=torch.float32)
    _check(load().tg_render_rays(density.handle, color.handle, _ptr(rays_o, "rays_o", numel=3 * R),
                                 _ptr(rays_d, "rays_d", numel=3 * R), R, S, seed, ray_base, bg,
                                 _ptr(out, "out", numel=3 * R), _ptr(target, "target", numel=3 * R, optional=True),
                                 None if batch is None else batch.handle,
                                 _ptr(density_grad, "density_grad", optional=True),
                                 _ptr(color_grad, "color_grad", optional=True),
                                 _ptr(loss_sum, "loss_sum", optional=True), _stream(stream)), "tg_render_rays")
    if batch is not None and target is not None:
        batch.n = R * S
    return out


def tg_render_rays_backward(density: Grid, color: Grid, rays_o, rays_d, dL_drgb, S: int, batch: Batch,
                            density_grad, color_grad, seed: int = 0, ray_base: int = 0, bg: float = 1.0, out=None,
                            stream=None):
    """Adds dL/dtheta of both grids for an upstream dL/drgb, recomputing every sample of the forward."""
    R = rays_o.shape[0]
    _check(load().tg_render_rays_backward(density.handle, color.handle, _ptr(rays_o, "rays_o", numel=3 * R),
                                          _ptr(rays_d, "rays_d", numel=3 * R), R, S, seed, ray_base, bg,
                                          _ptr(dL_drgb, "dL_drgb", numel=3 * R), batch.handle,
                                          _ptr(density_grad, "density_grad", numel=density.n_coefs),
                                          _ptr(color_grad, "color_grad", numel=color.n_coefs),
                                          _ptr(out, "out", numel=3 * R, optional=True), _stream(stream)),
           "tg_render_rays_backward")
    batch.n = R * S
    return out


JOB_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed", 4: "cancelled"}


class Server:
    """Continuous-batching fit / query server (tg_server_*)."""

    def __init__(self, budget_bytes: int, max_running: int = 64, smallest_first: bool = False):
        h = _vp()
        _check(load().tg_server_create(budget_bytes, max_running, ctypes.byref(h)), "tg_server_create")
        self._h = h.value
        self._keep = {}
        if smallest_first:
            _check(load().tg_server_set_policy(self._h, 1), "tg_server_set_policy")

    def fit_job(self, shape_spheres, shape_boxes, area_cdf, res, order=2, dtype="f32", seed=0, points_per_step=1 << 16,
                eval_points=1 << 16, eval_every=10, max_steps=1000, tol=2e-3, lr=5e-3, lambda_eik=0.0,
                init_std=1e-3, k_weight=0.0, lambda_tv=0.0, deterministic=False, lazy_adam=False) -> int:
        import numpy as np
        sph = np.ascontiguousarray(shape_spheres, np.float32).reshape(-1)
        box = np.ascontiguousarray(shape_boxes, np.float32).reshape(-1)
        cdf = np.ascontiguousarray(area_cdf, np.float32).reshape(-1)
        d = FitDesc(res, order, DTYPES[dtype] if isinstance(dtype, str) else dtype, seed, sph.size // 4, box.size // 6,
                    sph.ctypes.data if sph.size else None, box.ctypes.data if box.size else None, cdf.ctypes.data,
                    points_per_step, eval_points, eval_every, max_steps, tol, lr, lambda_eik, init_std, k_weight,
                    lambda_tv, (1 if deterministic else 0) | (2 if lazy_adam else 0))
        jid = _i64()
        _check(load().tg_fit_job(self._h, ctypes.byref(d), ctypes.byref(jid)), "tg_fit_job")
        return jid.value

    def query_job(self, grid_job: int, pts: torch.Tensor, out: torch.Tensor) -> int:
        jid = _i64()
        _check(load().tg_query_job(self._h, grid_job, _ptr(pts, "pts"), pts.shape[0], _ptr(out, "out"),
                                   ctypes.byref(jid)), "tg_query_job")
        self._keep[jid.value] = (pts, out)
        return jid.value

    def step(self) -> int:
        p = _int()
        _check(load().tg_server_step(self._h, ctypes.byref(p)), "tg_server_step")
        return p.value

    def poll(self, jid: int) -> dict:
        r = JobResult()
        _check(load().tg_poll(self._h, jid, ctypes.byref(r)), "tg_poll")
        return {"state": JOB_STATES.get(r.state, r.state), "kind": "fit" if r.kind == 0 else "query",
                "steps": r.steps, "error": r.error, "t_submit": r.t_submit, "t_start": r.t_start,
                "t_done": r.t_done, "points": r.points, "bytes": r.bytes}

    def grid_coefs(self, jid: int, which: int = 1) -> torch.Tensor:
        h = _vp()
        _check(load().tg_server_grid(self._h, jid, ctypes.byref(h)), "tg_server_grid")
        info = GridInfo()
        _check(load().tg_get_info(h.value, ctypes.byref(info)), "tg_get_info")
        out = torch.empty(info.n_coefs, device="cuda", dtype=torch.float32)
        _check(load().tg_get_coefs(h.value, out.data_ptr(), which, _stream(None)), "tg_get_coefs")
        return out

    def release(self, jid: int):
        _check(load().tg_release(self._h, jid), "tg_release")
        self._keep.pop(jid, None)

    def cancel(self, jid: int):
        """Cancels a queued job at once, a running fit job at its next step boundary."""
        _check(load().tg_cancel(self._h, jid), "tg_cancel")

    def time(self) -> float:
        return load().tg_server_time(self._h)

    def run_until_idle(self, timeout_s: float = 600.0, sleep_s: float = 0.0):
        import time
        t0 = time.time()
        while self.step() > 0:
            if time.time() - t0 > timeout_s:
                raise TimeoutError("server did not drain")
            if sleep_s:
                time.sleep(sleep_s)

    def close(self):
        if getattr(self, "_h", None):
            load().tg_server_destroy(self._h)
            self._h = None

    __del__ = close
