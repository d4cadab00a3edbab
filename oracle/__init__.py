"""FP64 CPU oracle for the per-point MLS projection -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (``paper_2401_03365_gb300``)
never does: it has no CPU fallback.  The oracle is a plain single-threaded C
library (``mls_oracle.c``) built with gcc and loaded here through ctypes; it
shares no code with the CUDA path.

Functions (numpy in, numpy out):
  knn_brute(xyz, k)                   O(n^2) ranking, the pin for knn_kdtree
  knn_kdtree(xyz, k, queries=None)    k-d tree kNN (Sec. 2.2's data structure)
  mean_knn_dist(xyz, idx)             bandwidth helper: mean neighbour distance
  project(xyz, idx, h, degree, queries=None)  plane -> polynomial -> projection
                                      (Sec. 1.4, Eq. 1; Algorithm 1)
  project_grad(xyz, idx, h, degree, gp, gn)   FP64 adjoint (not in the paper)
  fit_height(P, w, n, e1, e2, q, h, degree)   polynomial fit over a given frame
  jacobi_eig(A), cholesky_solve(A, b), knn_key(p, q)   building blocks
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import build_oracle, library_path

__all__ = [
    "knn_brute", "knn_kdtree", "mean_knn_dist", "project", "project_grad", "project_levin", "fit_height",
    "jacobi_eig", "cholesky_solve", "knn_key", "STATUS_PLANE_DEGENERATE", "STATUS_POLY_SINGULAR",
    "STATUS_NOT_CONVERGED", "STATUS_OUTLIER", "STATUS_DEGREE_REDUCED", "radius_neighbors", "project_rows",
]

STATUS_PLANE_DEGENERATE = 1
STATUS_POLY_SINGULAR = 2
STATUS_NOT_CONVERGED = 8
STATUS_OUTLIER = 16
STATUS_DEGREE_REDUCED = 32

_lib = None

_f32p = ctypes.POINTER(ctypes.c_float)
_f64p = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        build_oracle()
    lib = ctypes.CDLL(path)
    lib.oracle_knn_key.argtypes = [_f32p, _f32p]
    lib.oracle_knn_key.restype = ctypes.c_float
    lib.oracle_knn_brute.argtypes = [_f32p, _i64, _int, _i32p, _f32p]
    lib.oracle_knn_kdtree.argtypes = [_f32p, _i64, _int, _i64p, _i64, _i32p, _f32p]
    lib.oracle_mean_knn_dist.argtypes = [_f32p, _i64, _i32p, _int]
    lib.oracle_mean_knn_dist.restype = _dbl
    lib.oracle_jacobi_eig.argtypes = [_int, _f64p, _f64p, _f64p]
    lib.oracle_jacobi_eig.restype = None
    lib.oracle_cholesky.argtypes = [_int, _f64p, _f64p, _dbl]
    lib.oracle_cholesky_solve.argtypes = [_int, _f64p, _f64p, _f64p]
    lib.oracle_cholesky_solve.restype = None
    lib.oracle_fit_height.argtypes = [_int, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p, _dbl, _int,
                                      _f64p, _f64p]
    lib.oracle_project.argtypes = [_f32p, _i64, _i32p, _int, _dbl, _int, _i64p, _i64, _f64p, _f64p,
                                   _u8p, _f64p]
    lib.oracle_project_grad.argtypes = [_f32p, _i64, _i32p, _int, _dbl, _int, _f64p, _f64p, _i64p, _i64,
                                        _f64p, _f64p, _f64p]
    lib.oracle_project_levin.argtypes = [_f32p, _i64, _i32p, _int, _dbl, _int, _int, _dbl, _i64p, _i64, _f64p,
                                         _f64p, _u8p, _i32p, _f64p]
    lib.oracle_radius_kdtree.argtypes = [_f32p, _i64, ctypes.c_float, _i64p, _i32p, _i32p]
    lib.oracle_project_rows.argtypes = [_f32p, _i64, _i64p, _i32p, _dbl, _int, _int, _f64p, _f64p, _u8p, _f64p]
    _lib = lib
    return lib


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _xyz(xyz):
    xyz = np.ascontiguousarray(xyz, dtype=np.float32)
    assert xyz.ndim == 2 and xyz.shape[1] == 3
    return xyz


def knn_key(p, q) -> np.float32:
    p = np.ascontiguousarray(p, np.float32)
    q = np.ascontiguousarray(q, np.float32)
    return np.float32(_load().oracle_knn_key(_p(p, _f32p), _p(q, _f32p)))


def knn_brute(xyz, k):
    xyz = _xyz(xyz)
    n = xyz.shape[0]
    idx = np.empty((n, k), np.int32)
    key = np.empty((n, k), np.float32)
    rc = _load().oracle_knn_brute(_p(xyz, _f32p), n, k, _p(idx, _i32p), _p(key, _f32p))
    if rc != 0:
        raise ValueError(f"oracle_knn_brute failed ({rc})")
    return idx, key


def knn_kdtree(xyz, k, queries=None):
    """Rows for all points, or for the listed queries (an empty list only
    builds the tree)."""
    xyz = _xyz(xyz)
    n = xyz.shape[0]
    q = None if queries is None else np.ascontiguousarray(queries, np.int64)
    m = n if q is None else q.shape[0]
    if q is not None and m == 0:
        q = np.zeros(1, np.int64)          # a valid pointer with nq = 0
    idx = np.empty((m, k), np.int32)
    key = np.empty((m, k), np.float32)
    rc = _load().oracle_knn_kdtree(_p(xyz, _f32p), n, k, _p(q, _i64p), m, _p(idx, _i32p),
                                   _p(key, _f32p))
    if rc != 0:
        raise ValueError(f"oracle_knn_kdtree failed ({rc})")
    return idx, key


def mean_knn_dist(xyz, idx):
    xyz = _xyz(xyz)
    idx = np.ascontiguousarray(idx, np.int32)
    return float(_load().oracle_mean_knn_dist(_p(xyz, _f32p), xyz.shape[0], _p(idx, _i32p),
                                              idx.shape[1]))


def project(xyz, idx, h, degree=2, queries=None):
    """Project all points (idx: n rows) or the listed `queries` (idx: one row
    per query, in the same order).  Returns (xyz', normal, status, diag) in
    float64 / uint8; diag columns are (lambda0, lambda1, lambda2, cond of the
    normal matrix, total weight)."""
    xyz = _xyz(xyz)
    idx = np.ascontiguousarray(idx, np.int32)
    n, k = xyz.shape[0], idx.shape[1]
    q = None if queries is None else np.ascontiguousarray(queries, np.int64)
    m = n if q is None else q.shape[0]
    assert idx.shape[0] == m, "one neighbour row per projected point"
    assert idx.min() >= 0 and idx.max() < n
    out = np.empty((m, 3), np.float64)
    nrm = np.empty((m, 3), np.float64)
    st = np.empty(m, np.uint8)
    diag = np.empty((m, 5), np.float64)
    rc = _load().oracle_project(_p(xyz, _f32p), n, _p(idx, _i32p), k, float(h), int(degree),
                                _p(q, _i64p), m, _p(out, _f64p), _p(nrm, _f64p), _p(st, _u8p),
                                _p(diag, _f64p))
    if rc != 0:
        raise ValueError(f"oracle_project failed ({rc})")
    return out, nrm, st, diag


def project_levin(xyz, idx, h, degree=2, max_iter=100, tol=1e-12, queries=None, with_diag=False):
    """The projection with weights about q (Sec. 1.4, Eq. 1), by the fixed
    point iteration from q = r.  Returns (xyz', normal, status, iterations);
    status bit 8 marks points that did not converge within max_iter.  With
    `with_diag`, a fifth array (m x 5) holds this operator's own diagnostics:
    the last plane's eigenvalues, the final fit's condition number and the
    last plane's total weight (columns as in `project`)."""
    xyz = _xyz(xyz)
    idx = np.ascontiguousarray(idx, np.int32)
    n, k = xyz.shape[0], idx.shape[1]
    q = None if queries is None else np.ascontiguousarray(queries, np.int64)
    m = n if q is None else q.shape[0]
    assert idx.shape[0] == m, "one neighbour row per projected point"
    out = np.empty((m, 3), np.float64)
    nrm = np.empty((m, 3), np.float64)
    st = np.empty(m, np.uint8)
    it = np.empty(m, np.int32)
    diag = np.empty((m, 5), np.float64) if with_diag else None
    rc = _load().oracle_project_levin(_p(xyz, _f32p), n, _p(idx, _i32p), k, float(h), int(degree), int(max_iter),
                                      float(tol), _p(q, _i64p), m, _p(out, _f64p), _p(nrm, _f64p), _p(st, _u8p),
                                      _p(it, _i32p), _p(diag, _f64p))
    if rc != 0:
        raise ValueError(f"oracle_project_levin failed ({rc})")
    return (out, nrm, st, it, diag) if with_diag else (out, nrm, st, it)


def radius_neighbors(xyz, R):
    """Radius-R neighbourhoods (key <= fl(R*R), self included, (key, index)
    order) as CSR: (offsets int64 (n + 1), rows int32)."""
    xyz = _xyz(xyz)
    n = xyz.shape[0]
    R2 = np.float32(np.float32(R) * np.float32(R))
    cnt = np.empty(n, np.int32)
    rc = _load().oracle_radius_kdtree(_p(xyz, _f32p), n, float(R2), None, None, _p(cnt, _i32p))
    if rc != 0:
        raise ValueError(f"oracle_radius_kdtree failed ({rc})")
    off = np.zeros(n + 1, np.int64)
    np.cumsum(cnt, out=off[1:])
    rows = np.empty(int(off[-1]), np.int32)
    rc = _load().oracle_radius_kdtree(_p(xyz, _f32p), n, float(R2), _p(off, _i64p), _p(rows, _i32p), _p(cnt, _i32p))
    if rc != 0:
        raise ValueError(f"oracle_radius_kdtree failed ({rc})")
    return off, rows


def project_rows(xyz, offsets, rows, h, degree=2, min_neighbors=3):
    """Projection over CSR neighbourhoods with the outlier rule (status 16)
    and, for small neighbourhoods, a lower degree (status 32: fewer than
    twice the basis size in points).
    Returns (xyz', normal, status, diag) as oracle.project (diag 0 for
    outliers)."""
    xyz = _xyz(xyz)
    n = xyz.shape[0]
    off = np.ascontiguousarray(offsets, np.int64)
    rows = np.ascontiguousarray(rows, np.int32)
    out = np.empty((n, 3), np.float64)
    nrm = np.empty((n, 3), np.float64)
    st = np.empty(n, np.uint8)
    diag = np.empty((n, 5), np.float64)
    rc = _load().oracle_project_rows(_p(xyz, _f32p), n, _p(off, _i64p), _p(rows, _i32p), float(h), int(degree),
                                     int(min_neighbors), _p(out, _f64p), _p(nrm, _f64p), _p(st, _u8p),
                                     _p(diag, _f64p))
    if rc != 0:
        raise ValueError(f"oracle_project_rows failed ({rc})")
    return out, nrm, st, diag


def project_grad(xyz, idx, h, degree, gout_xyz, gout_normal=None, queries=None, with_abs=False):
    """(dL/dxyz, dL/dh).  With `queries`, only those points' terms (idx: one
    row per query) are summed.  With `with_abs`, a third array (n) holds per
    point the sum of the norms of the terms added into its gradient (the
    scale of its rounding error when the terms cancel)."""
    xyz = _xyz(xyz)
    idx = np.ascontiguousarray(idx, np.int32)
    n, k = xyz.shape[0], idx.shape[1]
    q = None if queries is None else np.ascontiguousarray(queries, np.int64)
    m = n if q is None else q.shape[0]
    assert idx.shape[0] == m
    gp = np.ascontiguousarray(gout_xyz, np.float64)
    gn = None if gout_normal is None else np.ascontiguousarray(gout_normal, np.float64)
    grad = np.empty((n, 3), np.float64)
    gh = np.zeros(1, np.float64)
    gabs = np.empty(n, np.float64) if with_abs else None
    rc = _load().oracle_project_grad(_p(xyz, _f32p), n, _p(idx, _i32p), k, float(h), int(degree),
                                     _p(gp, _f64p), _p(gn, _f64p), _p(q, _i64p), m, _p(grad, _f64p),
                                     _p(gh, _f64p), _p(gabs, _f64p))
    if rc != 0:
        raise ValueError(f"oracle_project_grad failed ({rc})")
    return (grad, float(gh[0]), gabs) if with_abs else (grad, float(gh[0]))


def fit_height(P, w, nrm, e1, e2, q, h, degree=2):
    """Coefficients of the height polynomial over a fixed frame, or None when
    the normal equations are singular.  Returns (a, cond)."""
    P = np.ascontiguousarray(P, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    vec = [np.ascontiguousarray(v, np.float64) for v in (nrm, e1, e2, q)]
    a = np.zeros(6, np.float64)
    cond = np.zeros(1, np.float64)
    ok = _load().oracle_fit_height(P.shape[0], _p(P, _f64p), _p(w, _f64p), *[_p(v, _f64p) for v in vec],
                                   float(h), int(degree), _p(a, _f64p), _p(cond, _f64p))
    return (a if ok else None), float(cond[0])


def jacobi_eig(A):
    A = np.array(A, np.float64, copy=True, order="C")
    m = A.shape[0]
    lam = np.empty(m, np.float64)
    V = np.empty((m, m), np.float64)
    _load().oracle_jacobi_eig(m, _p(A, _f64p), _p(lam, _f64p), _p(V, _f64p))
    return lam, V


def cholesky_solve(A, b, rel_tol=1e-12):
    A = np.ascontiguousarray(A, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    m = A.shape[0]
    L = np.empty((m, m), np.float64)
    if not _load().oracle_cholesky(m, _p(A, _f64p), _p(L, _f64p), rel_tol):
        return None
    x = np.empty(m, np.float64)
    _load().oracle_cholesky_solve(m, _p(L, _f64p), _p(b, _f64p), _p(x, _f64p))
    return x
