"""Thin ctypes binding of libmls (include/mls.h), same names as the C ABI.

Argument marshalling only: torch tensors are checked for device, dtype and
layout, their device pointers and the current CUDA stream are passed through,
and negative status codes become MLSError.  Every computation runs in the
CUDA kernels of libmls; there is no CPU fallback, and loading fails loudly
when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import torch

from .build import library_path

__all__ = [
    "MLSError", "Grid", "lib", "mls_build_grid", "mls_grid_destroy", "mls_grid_size", "mls_grid_order",
    "mls_knn", "mls_knn_sorted", "mls_knn_deferred", "mls_points_in_boxes", "mls_project_sorted", "mls_knn_project", "mls_knn_project_sorted", "mls_project_backward_sorted", "mls_project", "mls_project_levin", "mls_project_backward", "mls_radius_neighbors",
    "mls_project_rows", "mls_compact", "mls_mean_knn_dist", "mls_status_str", "mls_last_error", "mls_kernel_launches", "mls_release_scratch",
    "Batch", "mls_batch_create", "mls_batch_destroy", "mls_batch_set_shape", "mls_batch_get_shape",
    "mls_project_batched", "mls_batch_capture", "mls_batch_replay", "mls_batch_autotune", "mls_batch_tune_results",
    "PRECISION", "MLS_MAX_K", "FIT_STATE_FLOATS", "MLS_PT_OK", "MLS_PT_PLANE_DEGENERATE", "MLS_PT_POLY_SINGULAR",
    "MLS_PT_FP64_USED", "EXPORTED_SYMBOLS",
]

MLS_MAX_K = 64
FIT_STATE_FLOATS = 29       # MLS_FIT_STATE_FLOATS: floats of fit state per point
MLS_NOALLOC_MAX_POINTS = 262144
PRECISION = {"fp32": 0, "mixed": 1, "fp64": 2}
MLS_PT_OK, MLS_PT_PLANE_DEGENERATE, MLS_PT_POLY_SINGULAR, MLS_PT_FP64_USED = 0, 1, 2, 4
MLS_PT_NOT_CONVERGED = 8
MLS_PT_OUTLIER = 16
MLS_MAX_RADIUS_NB = 128

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int
_flt = ctypes.c_float

# (name, restype, argtypes) of every entry point declared in include/mls.h
_SIGNATURES = [
    ("mls_build_grid", _int, [_vp, _i64, _flt, _int, _vp, ctypes.POINTER(_vp)]),
    ("mls_grid_destroy", None, [_vp]),
    ("mls_grid_size", _i64, [_vp]),
    ("mls_grid_order", _vp, [_vp]),
    ("mls_knn", _int, [_vp, _int, _vp, _vp, _vp]),
    ("mls_knn_deferred", ctypes.c_int64, [_vp, _vp]),
    ("mls_points_in_boxes", _int, [_vp, _vp, _i64, _vp, _vp]),
    ("mls_knn_sorted", _int, [_vp, _int, _vp, _vp, _vp, _vp]),
    ("mls_project_sorted", _int, [_vp, _vp, _int, ctypes.c_float, _int, _int, _vp, _vp, _vp, _vp, _vp]),
    ("mls_knn_project", _int, [_vp, _int, ctypes.c_float, _int, _int, _vp, _vp, _vp, _vp, _vp]),
    ("mls_knn_project_sorted", _int, [_vp, _int, ctypes.c_float, _int, _int, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("mls_project_backward_sorted", _int, [_vp, _vp, _int, ctypes.c_float, _int, _int, _vp, _vp, _vp, _vp, _vp,
                                           _vp, _vp]),
    ("mls_project", _int, [_vp, _i64, _vp, _int, _flt, _int, _int, _vp, _vp, _vp, _vp, _vp]),
    ("mls_project_noalloc", _int, [_vp, _i64, _vp, _int, _flt, _int, _int, _vp, _vp, _vp, _vp, _vp]),
    ("mls_project_levin", _int, [_vp, _i64, _vp, _int, _flt, _int, _int, _int, _flt, _vp, _vp, _vp, _vp, _vp]),
    ("mls_radius_count", _int, [_vp, _flt, _vp, _vp, _vp]),
    ("mls_radius_rows", _int, [_vp, _flt, _vp, _vp, _vp, _vp]),
    ("mls_project_rows", _int, [_vp, _i64, _vp, _vp, _flt, _int, _int, _int, _vp, _vp, _vp, _vp, _vp]),
    ("mls_compact", _int, [_vp, _i64, _int, _vp, _vp, _vp]),
    ("mls_project_backward", _int, [_vp, _i64, _vp, _int, _flt, _int, _int, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("mls_mean_knn_dist", _int, [_vp, _i64, _vp, _int, _vp, _vp]),
    ("mls_batch_create", _int, [_int, _vp, _vp, ctypes.POINTER(_vp)]),
    ("mls_batch_destroy", None, [_vp]),
    ("mls_batch_total", _i64, [_vp]),
    ("mls_batch_idx_offset", _i64, [_vp, _int]),
    ("mls_batch_set_shape", _int, [_vp, _int, _int, _int]),
    ("mls_batch_get_shape", _int, [_vp, ctypes.POINTER(_int), ctypes.POINTER(_int), ctypes.POINTER(_int)]),
    ("mls_project_batched", _int, [_vp, _vp, _vp, _vp, _vp, _int, _int, _vp, _vp, _vp, _vp]),
    ("mls_batch_capture", _int, [_vp, _vp, _vp, _vp, _vp, _int, _int, _vp, _vp, _vp]),
    ("mls_batch_replay", _int, [_vp, _vp]),
    ("mls_batch_autotune", _int, [_vp, _vp, _vp, _vp, _vp, _int, _int, _vp, _vp, _vp, _int, _vp]),
    ("mls_batch_tune_results", _int, [_vp, _int, _vp, _vp]),
    ("mls_release_scratch", _int, []),
    ("mls_kernel_launches", _i64, []),
    ("mls_last_error", ctypes.c_char_p, []),
    ("mls_status_str", ctypes.c_char_p, [_int]),
]
EXPORTED_SYMBOLS = [s[0] for s in _SIGNATURES]

_lib = None


class MLSError(RuntimeError):
    def __init__(self, fn: str, code: int):
        self.code = code
        msg = lib().mls_last_error().decode() or lib().mls_status_str(code).decode()
        super().__init__(f"{fn} failed ({code}, {lib().mls_status_str(code).decode()}): {msg}")


def lib():
    """The loaded libmls (ctypes.CDLL).  Raises if it has not been built."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise ImportError(f"libmls is not built ({path} missing): run "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        if torch.cuda.is_available():
            torch.cuda.init()           # one CUDA runtime, shared with torch
        dll = ctypes.CDLL(path)
        for name, res, args in _SIGNATURES:
            fn = getattr(dll, name)
            fn.restype = res
            fn.argtypes = args
        _lib = dll
    return _lib


def _check(fn, rc):
    if rc != 0:
        raise MLSError(fn, rc)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _need(t, name, dtype, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


def mls_status_str(code: int) -> str:
    return lib().mls_status_str(code).decode()


def mls_last_error() -> str:
    return lib().mls_last_error().decode()


def mls_release_scratch() -> None:
    """Returns the library's unused scratch memory to the system (synchronises)."""
    _check("mls_release_scratch", lib().mls_release_scratch())


def mls_kernel_launches() -> int:
    return int(lib().mls_kernel_launches())


class Grid:
    """Owner of an mls_grid handle; keeps the point tensor alive."""

    def __init__(self, handle, xyz):
        self.handle = handle
        self.xyz = xyz

    @property
    def n(self) -> int:
        return int(lib().mls_grid_size(self.handle))

    def close(self):
        if self.handle:
            lib().mls_grid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mls_build_grid(xyz: torch.Tensor, cell_size: float = 0.0, k_hint: int = 32, grid: Grid | None = None,
                   stream=None) -> Grid:
    _need(xyz, "xyz", torch.float32)
    if xyz.dim() != 2 or xyz.shape[1] != 3:
        raise ValueError("xyz must be (n, 3)")
    h = ctypes.c_void_p(grid.handle if grid is not None else None)
    rc = lib().mls_build_grid(_ptr(xyz), xyz.shape[0], float(cell_size), int(k_hint), _stream(stream),
                              ctypes.byref(h))
    if rc != 0 and grid is not None:
        grid.xyz = None
    _check("mls_build_grid", rc)
    if grid is not None:
        grid.handle, grid.xyz = h.value, xyz
        return grid
    return Grid(h.value, xyz)


def mls_grid_destroy(grid: Grid) -> None:
    grid.close()


def mls_grid_size(grid: Grid) -> int:
    return grid.n


class _DeviceArray:
    """A device buffer owned by libmls, seen through __cuda_array_interface__."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


def mls_grid_order(grid: Grid) -> torch.Tensor:
    """The grid's order (Hilbert order of the cells; order[s] = point at sorted position s) as an
    int32 CUDA tensor viewing the grid's own buffer: valid until the grid is
    rebuilt or destroyed."""
    p = lib().mls_grid_order(grid.handle)
    if not p:
        raise ValueError("mls_grid_order: the grid is empty")
    return torch.as_tensor(_DeviceArray(p, grid.n, "<i4"), device=grid.xyz.device)


def mls_knn(grid: Grid, k: int, with_key: bool = False, out_idx=None, out_key=None, stream=None):
    """Exact kNN rows (n, k) int32 in original indexing (and keys with
    `with_key`)."""
    n = grid.n
    dev = grid.xyz.device
    if out_idx is None:
        out_idx = torch.empty((n, k), dtype=torch.int32, device=dev)
    _need(out_idx, "out_idx", torch.int32, (n, k))
    if with_key and out_key is None:
        out_key = torch.empty((n, k), dtype=torch.float32, device=dev)
    if out_key is not None:
        _need(out_key, "out_key", torch.float32, (n, k))
    _check("mls_knn", lib().mls_knn(grid.handle, int(k), _ptr(out_idx), _ptr(out_key), _stream(stream)))
    return out_idx, out_key


def mls_knn_sorted(grid: Grid, k: int, with_idx: bool = False, with_key: bool = False, out_pos=None,
                   out_idx=None, out_key=None, stream=None):
    """Rows of sorted positions by sorted position (n, k) int32, and with
    `with_idx` / `with_key` also mls_knn's rows and keys: (pos, idx, key)."""
    n = grid.n
    dev = grid.xyz.device
    out_pos = torch.empty((n, k), dtype=torch.int32, device=dev) if out_pos is None else out_pos
    _need(out_pos, "out_pos", torch.int32, (n, k))
    if with_idx and out_idx is None:
        out_idx = torch.empty((n, k), dtype=torch.int32, device=dev)
    if out_idx is not None:
        _need(out_idx, "out_idx", torch.int32, (n, k))
    if with_key and out_key is None:
        out_key = torch.empty((n, k), dtype=torch.float32, device=dev)
    if out_key is not None:
        _need(out_key, "out_key", torch.float32, (n, k))
    _check("mls_knn_sorted", lib().mls_knn_sorted(grid.handle, int(k), _ptr(out_pos), _ptr(out_idx), _ptr(out_key),
                                                  _stream(stream)))
    return out_pos, out_idx, out_key


def mls_project_sorted(grid: Grid, pos: torch.Tensor, h: float, degree: int = 2, precision: str = "mixed",
                       out_xyz=None, out_normal=None, out_status=None, stream=None, with_state: bool = False,
                       out_state=None):
    """mls_project over the grid's sorted points and mls_knn_sorted's rows;
    outputs in the original order.  With `with_state` also the fit state
    (FIT_STATE_FLOATS, n) by sorted position, for mls_project_backward_sorted:
    (xyz, normal, status[, state])."""
    n = grid.n
    _need(pos, "pos", torch.int32)
    if pos.dim() != 2 or pos.shape[0] != n:
        raise ValueError("pos must be (n, k)")
    dev = grid.xyz.device
    out_xyz = torch.empty((n, 3), dtype=torch.float32, device=dev) if out_xyz is None else out_xyz
    out_normal = torch.empty((n, 3), dtype=torch.float32, device=dev) if out_normal is None else out_normal
    out_status = torch.empty(n, dtype=torch.uint8, device=dev) if out_status is None else out_status
    _need(out_xyz, "out_xyz", torch.float32, (n, 3))
    _need(out_normal, "out_normal", torch.float32, (n, 3))
    _need(out_status, "out_status", torch.uint8, (n,))
    if with_state:
        out_state = torch.empty((FIT_STATE_FLOATS, n), dtype=torch.float32, device=dev) if out_state is None \
            else out_state
        _need(out_state, "out_state", torch.float32, (FIT_STATE_FLOATS, n))
    rc = lib().mls_project_sorted(grid.handle, _ptr(pos), pos.shape[1], float(h), int(degree), PRECISION[precision],
                                  _ptr(out_xyz), _ptr(out_normal), _ptr(out_status),
                                  _ptr(out_state) if with_state else None, _stream(stream))
    _check("mls_project_sorted", rc)
    return (out_xyz, out_normal, out_status, out_state) if with_state else (out_xyz, out_normal, out_status)


def mls_knn_project(grid: Grid, k: int, h: float, degree: int = 2, precision: str = "mixed", with_pos: bool = False,
                    out_xyz=None, out_normal=None, out_status=None, out_pos=None, stream=None):
    """The kNN and the projection in one pass (rows kept on chip, written only
    with with_pos): (xyz (n, 3), normal (n, 3), status (n,)[, pos (n, k)]) in
    the original order (pos: rows of sorted positions, as mls_knn_sorted)."""
    n = grid.n
    dev = grid.xyz.device
    out_xyz = torch.empty((n, 3), dtype=torch.float32, device=dev) if out_xyz is None else out_xyz
    out_normal = torch.empty((n, 3), dtype=torch.float32, device=dev) if out_normal is None else out_normal
    out_status = torch.empty(n, dtype=torch.uint8, device=dev) if out_status is None else out_status
    _need(out_xyz, "out_xyz", torch.float32, (n, 3))
    _need(out_normal, "out_normal", torch.float32, (n, 3))
    _need(out_status, "out_status", torch.uint8, (n,))
    if with_pos:
        out_pos = torch.empty((n, k), dtype=torch.int32, device=dev) if out_pos is None else out_pos
        _need(out_pos, "out_pos", torch.int32, (n, k))
    rc = lib().mls_knn_project(grid.handle, int(k), float(h), int(degree), PRECISION[precision], _ptr(out_xyz),
                               _ptr(out_normal), _ptr(out_status), _ptr(out_pos) if with_pos else None,
                               _stream(stream))
    _check("mls_knn_project", rc)
    return (out_xyz, out_normal, out_status, out_pos) if with_pos else (out_xyz, out_normal, out_status)


def mls_knn_project_sorted(grid: Grid, k: int, h: float, degree: int = 2, precision: str = "mixed",
                           out_pos=None, out_xyz=None, out_normal=None, out_status=None, with_state: bool = False,
                           out_state=None, out_offsets=None, stream=None):
    """mls_knn_sorted and mls_project_sorted pipelined (the projection of the
    points the kNN's first pass finished runs beside its second pass): (pos,
    xyz, normal, status[, state]), the outputs of the two calls; with
    `out_offsets` (n + 1 int32) also the adjoint's bucket offsets."""
    n = grid.n
    dev = grid.xyz.device
    out_pos = torch.empty((n, k), dtype=torch.int32, device=dev) if out_pos is None else out_pos
    out_xyz = torch.empty((n, 3), dtype=torch.float32, device=dev) if out_xyz is None else out_xyz
    out_normal = torch.empty((n, 3), dtype=torch.float32, device=dev) if out_normal is None else out_normal
    out_status = torch.empty(n, dtype=torch.uint8, device=dev) if out_status is None else out_status
    _need(out_pos, "out_pos", torch.int32, (n, k))
    _need(out_xyz, "out_xyz", torch.float32, (n, 3))
    _need(out_normal, "out_normal", torch.float32, (n, 3))
    _need(out_status, "out_status", torch.uint8, (n,))
    if with_state:
        out_state = torch.empty((FIT_STATE_FLOATS, n), dtype=torch.float32, device=dev) if out_state is None \
            else out_state
        _need(out_state, "out_state", torch.float32, (FIT_STATE_FLOATS, n))
    if out_offsets is not None:
        _need(out_offsets, "out_offsets", torch.int32, (n + 1,))
    rc = lib().mls_knn_project_sorted(grid.handle, int(k), float(h), int(degree), PRECISION[precision], _ptr(out_pos),
                                      _ptr(out_xyz), _ptr(out_normal), _ptr(out_status),
                                      _ptr(out_state) if with_state else None, _ptr(out_offsets), _stream(stream))
    _check("mls_knn_project_sorted", rc)
    res = (out_pos, out_xyz, out_normal, out_status)
    return res + (out_state,) if with_state else res


def mls_project_backward_sorted(grid: Grid, pos: torch.Tensor, h: float, gout_xyz: torch.Tensor,
                                gout_normal: torch.Tensor | None = None, degree: int = 2, precision: str = "mixed",
                                out_grad_xyz=None, out_grad_h=None, stream=None, state: torch.Tensor | None = None,
                                offsets: torch.Tensor | None = None):
    """mls_project_backward over the grid's sorted points and mls_knn_sorted's
    rows: (dL/dxyz (n, 3), dL/dh (1,)) in the original order.  `state`: the
    fit state mls_project_sorted saved (then not recomputed)."""
    n = grid.n
    _need(pos, "pos", torch.int32)
    if pos.dim() != 2 or pos.shape[0] != n:
        raise ValueError("pos must be (n, k)")
    _need(gout_xyz, "gout_xyz", torch.float32, (n, 3))
    if gout_normal is not None:
        _need(gout_normal, "gout_normal", torch.float32, (n, 3))
    if state is not None:
        _need(state, "state", torch.float32, (FIT_STATE_FLOATS, n))
    if offsets is not None:
        _need(offsets, "offsets", torch.int32, (n + 1,))
    dev = grid.xyz.device
    out_grad_xyz = torch.empty((n, 3), dtype=torch.float32, device=dev) if out_grad_xyz is None else out_grad_xyz
    out_grad_h = torch.empty(1, dtype=torch.float32, device=dev) if out_grad_h is None else out_grad_h
    _need(out_grad_xyz, "out_grad_xyz", torch.float32, (n, 3))
    _need(out_grad_h, "out_grad_h", torch.float32, (1,))
    rc = lib().mls_project_backward_sorted(grid.handle, _ptr(pos), pos.shape[1], float(h), int(degree),
                                           PRECISION[precision], _ptr(gout_xyz), _ptr(gout_normal),
                                           _ptr(out_grad_xyz), _ptr(out_grad_h), _ptr(state), _ptr(offsets),
                                           _stream(stream))
    _check("mls_project_backward_sorted", rc)
    return out_grad_xyz, out_grad_h


def mls_points_in_boxes(grid: Grid, boxes: torch.Tensor, out_mask=None, stream=None):
    """uint8 mask (n,) over the grid's cloud: 1 where a point lies in any of
    the boxes (m, 6) float32 (lo xyz, hi xyz)."""
    n = grid.n
    boxes = boxes.contiguous()
    _need(boxes, "boxes", torch.float32)
    if boxes.dim() != 2 or boxes.shape[1] != 6:
        raise ValueError("boxes must be (m, 6)")
    if out_mask is None:
        out_mask = torch.zeros(n, dtype=torch.uint8, device=grid.xyz.device)
    _need(out_mask, "out_mask", torch.uint8, (n,))
    _check("mls_points_in_boxes", lib().mls_points_in_boxes(grid.handle, _ptr(boxes), boxes.shape[0], _ptr(out_mask),
                                                            _stream(stream)))
    return out_mask


def mls_knn_deferred(grid: Grid, stream=None) -> int:
    """Queries the last kNN call on `grid` searched outside its runs of
    consecutive queries: the isolated ones taken first and those handed to
    its second (sparse) pass (synchronises the stream)."""
    v = int(lib().mls_knn_deferred(grid.handle, _stream(stream)))
    if v < 0:
        _check("mls_knn_deferred", v)
    return v


def mls_project(xyz: torch.Tensor, idx: torch.Tensor, h: float, degree: int = 2, precision: str = "mixed",
                order: torch.Tensor | None = None, out_xyz=None, out_normal=None, out_status=None,
                want_normal: bool = True, want_status: bool = True, stream=None):
    _need(xyz, "xyz", torch.float32)
    n = xyz.shape[0]
    _need(idx, "idx", torch.int32)
    if idx.dim() != 2 or idx.shape[0] != n:
        raise ValueError("idx must be (n, k)")
    k = idx.shape[1]
    if order is not None:
        _need(order, "order", torch.int32, (n,))
    if out_xyz is None:
        out_xyz = torch.empty_like(xyz)
    _need(out_xyz, "out_xyz", torch.float32, (n, 3))
    if out_normal is None and want_normal:
        out_normal = torch.empty_like(xyz)
    if out_normal is not None:
        _need(out_normal, "out_normal", torch.float32, (n, 3))
    if out_status is None and want_status:
        out_status = torch.empty(n, dtype=torch.uint8, device=xyz.device)
    if out_status is not None:
        _need(out_status, "out_status", torch.uint8, (n,))
    rc = lib().mls_project(_ptr(xyz), n, _ptr(idx), k, float(h), int(degree), PRECISION[precision],
                           _ptr(order), _ptr(out_xyz), _ptr(out_normal), _ptr(out_status), _stream(stream))
    _check("mls_project", rc)
    return out_xyz, out_normal, out_status


def mls_project_levin(xyz: torch.Tensor, idx: torch.Tensor, h: float, degree: int = 2, precision: str = "mixed",
                      max_iter: int = 32, tol: float = 1e-6, order: torch.Tensor | None = None, out_xyz=None,
                      out_normal=None, out_status=None, stream=None):
    """The projection with the weights about q (Sec. 1.4, Eq. 1); see mls.h."""
    _need(xyz, "xyz", torch.float32)
    n = xyz.shape[0]
    _need(idx, "idx", torch.int32)
    if idx.dim() != 2 or idx.shape[0] != n:
        raise ValueError("idx must be (n, k)")
    if order is not None:
        _need(order, "order", torch.int32, (n,))
    out_xyz = torch.empty_like(xyz) if out_xyz is None else out_xyz
    out_normal = torch.empty_like(xyz) if out_normal is None else out_normal
    out_status = torch.empty(n, dtype=torch.uint8, device=xyz.device) if out_status is None else out_status
    _need(out_xyz, "out_xyz", torch.float32, (n, 3))
    _need(out_normal, "out_normal", torch.float32, (n, 3))
    _need(out_status, "out_status", torch.uint8, (n,))
    rc = lib().mls_project_levin(_ptr(xyz), n, _ptr(idx), idx.shape[1], float(h), int(degree), PRECISION[precision],
                                 int(max_iter), float(tol), _ptr(order), _ptr(out_xyz), _ptr(out_normal),
                                 _ptr(out_status), _stream(stream))
    _check("mls_project_levin", rc)
    return out_xyz, out_normal, out_status


def mls_radius_neighbors(grid: Grid, R: float, with_key: bool = False, stream=None):
    """CSR radius-R neighbourhoods of the grid's points: (offsets int64 (n + 1),
    rows int32, keys float32 or None).  Reads the total back (one sync)."""
    n = grid.n
    dev = grid.xyz.device
    count = torch.empty(n, dtype=torch.int32, device=dev)
    offsets = torch.empty(n + 1, dtype=torch.int64, device=dev)
    _check("mls_radius_count", lib().mls_radius_count(grid.handle, float(R), _ptr(count), _ptr(offsets),
                                                        _stream(stream)))
    total = int(offsets[n].item())
    rows = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
    keys = torch.empty(max(total, 1), dtype=torch.float32, device=dev) if with_key else None
    _check("mls_radius_rows", lib().mls_radius_rows(grid.handle, float(R), _ptr(offsets), _ptr(rows), _ptr(keys),
                                                      _stream(stream)))
    return offsets, rows[:total], (keys[:total] if keys is not None else None)


def mls_project_rows(xyz: torch.Tensor, offsets: torch.Tensor, rows: torch.Tensor, h: float, degree: int = 2,
                     precision: str = "mixed", min_neighbors: int = 3, order: torch.Tensor | None = None,
                     stream=None):
    """Projection over CSR neighbourhoods with the outlier rule; returns
    (xyz', normal, status) for every point (outliers unmoved, status 16)."""
    _need(xyz, "xyz", torch.float32)
    n = xyz.shape[0]
    _need(offsets, "offsets", torch.int64, (n + 1,))
    _need(rows, "rows", torch.int32)
    if order is not None:
        _need(order, "order", torch.int32, (n,))
    out = torch.empty_like(xyz)
    nrm = torch.empty_like(xyz)
    st = torch.empty(n, dtype=torch.uint8, device=xyz.device)
    rc = lib().mls_project_rows(_ptr(xyz), n, _ptr(offsets), _ptr(rows), float(h), int(degree), PRECISION[precision],
                                int(min_neighbors), _ptr(order), _ptr(out), _ptr(nrm), _ptr(st), _stream(stream))
    _check("mls_project_rows", rc)
    return out, nrm, st


def mls_compact(status: torch.Tensor, mask: int = MLS_PT_OUTLIER, stream=None) -> torch.Tensor:
    """Indices of the entries with (status & mask) == 0 (one sync for the count)."""
    _need(status, "status", torch.uint8)
    n = status.shape[0]
    kept = torch.empty(n, dtype=torch.int32, device=status.device)
    num = torch.empty(1, dtype=torch.int64, device=status.device)
    _check("mls_compact", lib().mls_compact(_ptr(status), n, int(mask), _ptr(kept), _ptr(num), _stream(stream)))
    return kept[: int(num.item())]


def mls_project_backward(xyz: torch.Tensor, idx: torch.Tensor, h: float, grad_out_xyz: torch.Tensor,
                         grad_out_normal: torch.Tensor | None = None, degree: int = 2, precision: str = "mixed",
                         order: torch.Tensor | None = None, out_grad_xyz=None, out_grad_h=None, stream=None):
    """(dL/dxyz, dL/dh) for L = <grad_out_xyz, xyz'> + <grad_out_normal, normal>."""
    _need(xyz, "xyz", torch.float32)
    n = xyz.shape[0]
    _need(idx, "idx", torch.int32)
    if idx.dim() != 2 or idx.shape[0] != n:
        raise ValueError("idx must be (n, k)")
    _need(grad_out_xyz, "grad_out_xyz", torch.float32, (n, 3))
    if grad_out_normal is not None:
        _need(grad_out_normal, "grad_out_normal", torch.float32, (n, 3))
    if order is not None:
        _need(order, "order", torch.int32, (n,))
    if out_grad_xyz is None:
        out_grad_xyz = torch.empty_like(xyz)
    _need(out_grad_xyz, "out_grad_xyz", torch.float32, (n, 3))
    if out_grad_h is None:
        out_grad_h = torch.empty(1, dtype=torch.float32, device=xyz.device)
    _need(out_grad_h, "out_grad_h", torch.float32, (1,))
    rc = lib().mls_project_backward(_ptr(xyz), n, _ptr(idx), idx.shape[1], float(h), int(degree),
                                    PRECISION[precision], _ptr(order), _ptr(grad_out_xyz), _ptr(grad_out_normal),
                                    _ptr(out_grad_xyz), _ptr(out_grad_h), _stream(stream))
    _check("mls_project_backward", rc)
    return out_grad_xyz, out_grad_h


def mls_mean_knn_dist(xyz: torch.Tensor, idx: torch.Tensor, stream=None) -> torch.Tensor:
    _need(xyz, "xyz", torch.float32)
    _need(idx, "idx", torch.int32)
    out = torch.empty(1, dtype=torch.float64, device=xyz.device)
    _check("mls_mean_knn_dist", lib().mls_mean_knn_dist(_ptr(xyz), xyz.shape[0], _ptr(idx), idx.shape[1],
                                                        _ptr(out), _stream(stream)))
    return out


class Batch:
    """Owner of an mls_batch handle (clouds' sizes and k fixed at creation)."""

    def __init__(self, handle, offsets, ks):
        self.handle = handle
        self.offsets = [int(o) for o in offsets]
        self.ks = [int(k) for k in ks]
        self.total = self.offsets[-1]
        self.idx_len = int(lib().mls_batch_idx_offset(handle, len(self.ks)))
        self._keep = ()             # buffers a captured graph refers to

    def idx_offset(self, cloud: int) -> int:
        return int(lib().mls_batch_idx_offset(self.handle, int(cloud)))

    def close(self):
        if self.handle:
            lib().mls_batch_destroy(self.handle)
            self.handle = None
            self._keep = ()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mls_batch_create(offsets, ks) -> Batch:
    """offsets: B + 1 point offsets (host sequence); ks: B neighbour counts."""
    offsets = [int(o) for o in offsets]
    ks = [int(k) for k in ks]
    if len(offsets) != len(ks) + 1:
        raise ValueError("offsets must have one entry more than ks")
    off = (ctypes.c_int64 * len(offsets))(*offsets)
    kk = (ctypes.c_int32 * max(len(ks), 1))(*ks)
    h = _vp()
    _check("mls_batch_create", lib().mls_batch_create(len(ks), off, kk, ctypes.byref(h)))
    return Batch(h, offsets, ks)


def mls_batch_destroy(batch: Batch) -> None:
    batch.close()


def mls_batch_set_shape(batch: Batch, lanes_per_point: int, threads: int, rounds: int) -> None:
    _check("mls_batch_set_shape", lib().mls_batch_set_shape(batch.handle, int(lanes_per_point), int(threads),
                                                            int(rounds)))
    batch._keep = ()


def mls_batch_get_shape(batch: Batch) -> tuple[int, int, int]:
    g, t, r = _int(), _int(), _int()
    _check("mls_batch_get_shape", lib().mls_batch_get_shape(batch.handle, ctypes.byref(g), ctypes.byref(t),
                                                            ctypes.byref(r)))
    return g.value, t.value, r.value


def _batch_args(batch, xyz, idx, h, order, out_xyz, out_normal, out_status, want_normal, want_status):
    n = batch.total
    _need(xyz, "xyz", torch.float32, (n, 3))
    _need(idx, "idx", torch.int32, (batch.idx_len,))
    _need(h, "h", torch.float32, (len(batch.ks),))
    if order is not None:
        _need(order, "order", torch.int32, (n,))
    if out_xyz is None:
        out_xyz = torch.empty_like(xyz)
    _need(out_xyz, "out_xyz", torch.float32, (n, 3))
    if out_normal is None and want_normal:
        out_normal = torch.empty_like(xyz)
    if out_normal is not None:
        _need(out_normal, "out_normal", torch.float32, (n, 3))
    if out_status is None and want_status:
        out_status = torch.empty(n, dtype=torch.uint8, device=xyz.device)
    if out_status is not None:
        _need(out_status, "out_status", torch.uint8, (n,))
    return out_xyz, out_normal, out_status


def mls_project_batched(batch: Batch, xyz: torch.Tensor, idx: torch.Tensor, h: torch.Tensor, degree: int = 2,
                        precision: str = "mixed", order: torch.Tensor | None = None, out_xyz=None, out_normal=None,
                        out_status=None, want_normal: bool = True, want_status: bool = True, stream=None):
    """xyz (total, 3) float32; idx the concatenated per-cloud rows (flat int32,
    cloud-local indices); h (B,) float32 on the device."""
    out_xyz, out_normal, out_status = _batch_args(batch, xyz, idx, h, order, out_xyz, out_normal, out_status,
                                                  want_normal, want_status)
    rc = lib().mls_project_batched(batch.handle, _ptr(xyz), _ptr(idx), _ptr(order), _ptr(h), int(degree),
                                   PRECISION[precision], _ptr(out_xyz), _ptr(out_normal), _ptr(out_status),
                                   _stream(stream))
    _check("mls_project_batched", rc)
    return out_xyz, out_normal, out_status


def mls_batch_capture(batch: Batch, xyz, idx, h, degree: int = 2, precision: str = "mixed", order=None,
                      out_xyz=None, out_normal=None, out_status=None, want_normal: bool = True,
                      want_status: bool = True):
    """Captures one batched projection into the batch's CUDA graph; returns the
    output tensors the graph writes (kept alive with the inputs by the batch)."""
    out_xyz, out_normal, out_status = _batch_args(batch, xyz, idx, h, order, out_xyz, out_normal, out_status,
                                                  want_normal, want_status)
    rc = lib().mls_batch_capture(batch.handle, _ptr(xyz), _ptr(idx), _ptr(order), _ptr(h), int(degree),
                                 PRECISION[precision], _ptr(out_xyz), _ptr(out_normal), _ptr(out_status))
    _check("mls_batch_capture", rc)
    batch._keep = (xyz, idx, h, order, out_xyz, out_normal, out_status)
    return out_xyz, out_normal, out_status


def mls_batch_replay(batch: Batch, stream=None) -> None:
    _check("mls_batch_replay", lib().mls_batch_replay(batch.handle, _stream(stream)))


def mls_batch_autotune(batch: Batch, xyz, idx, h, degree: int = 2, precision: str = "mixed", order=None,
                       out_xyz=None, out_normal=None, out_status=None, reps: int = 3, stream=None):
    """Times every candidate launch shape and keeps the fastest; returns
    (shape, [(lanes, threads, rounds, ms), ...])."""
    out_xyz, out_normal, out_status = _batch_args(batch, xyz, idx, h, order, out_xyz, out_normal, out_status,
                                                  True, True)
    rc = lib().mls_batch_autotune(batch.handle, _ptr(xyz), _ptr(idx), _ptr(order), _ptr(h), int(degree),
                                  PRECISION[precision], _ptr(out_xyz), _ptr(out_normal), _ptr(out_status),
                                  int(reps), _stream(stream))
    _check("mls_batch_autotune", rc)
    batch._keep = ()
    return mls_batch_get_shape(batch), mls_batch_tune_results(batch)


def mls_batch_tune_results(batch: Batch):
    n = int(lib().mls_batch_tune_results(batch.handle, 0, None, None))
    shapes = (ctypes.c_int32 * (3 * max(n, 1)))()
    ms = (ctypes.c_float * max(n, 1))()
    lib().mls_batch_tune_results(batch.handle, n, shapes, ms)
    return [(shapes[3 * i], shapes[3 * i + 1], shapes[3 * i + 2], float(ms[i])) for i in range(n)]
