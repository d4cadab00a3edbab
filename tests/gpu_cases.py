"""Shared inputs and checks for the GPU parity tests (CUDA path vs the oracle)."""
import zlib

import numpy as np

import oracle
from paper_2401_03365_gb300 import workloads

# Well-posed mask for the floating-point tolerances: the plane normal is
# determined to FP32 accuracy only when the eigen-gap is not tiny relative to
# the largest eigenvalue, and the height fit only when its normal matrix is
# not near-singular.  With the fit's moments summed in FP32 (the FP32 and
# mixed forms), a Cholesky pivot carries a relative error of about
# cond * 2^-24, so the singular decision (pivot <= 1e-12 trace) is only
# determined where that is far below 1: cond <= 1e6 (error <= 0.06).  A
# nearly isolated point of the torus (total weight 1.35, cond 8.3e7) is
# singular in FP32 and regular in FP64.
GAP_MIN = 1e-3
COND_MAX = 1e6
POS_TOL = 1e-5        # of the bounding-box diagonal
NORMAL_TOL = 1e-4     # radians
# The canonical sign (largest-magnitude component positive) is decided by the
# same component on both sides when the oracle normal's two largest
# magnitudes differ by more than twice the component error a normal within
# NORMAL_TOL can have, with a factor 2 to spare: there the normals are
# compared with their sign.
SIGN_MARGIN = 4 * NORMAL_TOL


def lattice(n_side, spacing=0.25, seed=0):
    g = np.arange(n_side, dtype=np.float32) * np.float32(spacing)
    pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    return pts[np.random.default_rng(seed).permutation(pts.shape[0])]


def knn_case(name):
    """(xyz float32, k) for the kNN parity cases."""
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    if name == "sphere20k_k20":
        c = workloads.sphere()
        return c.xyz, c.k
    if name == "torus100k_k32":
        c = workloads.torus(n=100_000, seed=12)
        return c.xyz, 32
    if name == "heightfield200k_k64":
        c = workloads.heightfield(n=200_000, seed=13)
        return c.xyz, 64
    if name == "lattice_ties_k27":
        return lattice(12), 27
    if name == "lattice_ties_k64":
        return lattice(10), 64
    if name == "duplicates_k20":
        base = rng.uniform(0, 1, (500, 3)).astype(np.float32)
        return base[rng.integers(0, 500, 5000)], 20
    if name == "clusters_and_outliers_k16":
        a = rng.normal(0, 1e-3, (3000, 3))
        b = rng.normal(5, 1e-2, (3000, 3))
        c = rng.uniform(-50, 50, (40, 3))
        return np.concatenate([a, b, c]).astype(np.float32), 16
    if name == "far_from_origin_k12":
        return (rng.standard_normal((5000, 3)) * 1e-2 + 1000.0).astype(np.float32), 12
    if name == "all_identical_k10":
        return np.full((100, 3), 0.5, np.float32), 10
    if name == "planar_k8":
        p = rng.uniform(-1, 1, (4000, 3)).astype(np.float32)
        p[:, 2] = 0.25
        return p, 8
    if name == "tiny_n_equals_k":
        return rng.standard_normal((5, 3)).astype(np.float32), 5
    if name == "n64_k64":
        return rng.standard_normal((64, 3)).astype(np.float32), 64
    if name == "k1":
        return rng.standard_normal((3000, 3)).astype(np.float32), 1
    if name == "k33_ragged":
        return rng.standard_normal((20_011, 3)).astype(np.float32), 33
    raise KeyError(name)


KNN_CASES = ["sphere20k_k20", "torus100k_k32", "heightfield200k_k64", "lattice_ties_k27", "lattice_ties_k64",
             "duplicates_k20", "clusters_and_outliers_k16", "far_from_origin_k12", "all_identical_k10",
             "planar_k8", "tiny_n_equals_k", "n64_k64", "k1", "k33_ragged"]


def oracle_knn(xyz, k):
    if xyz.shape[0] <= 3000:
        return oracle.knn_brute(xyz, k)
    return oracle.knn_kdtree(xyz, k)


def diag_len(xyz):
    x = xyz.astype(np.float64)
    return float(np.linalg.norm(x.max(0) - x.min(0)))


def well_posed(diag, gap_min=GAP_MIN, cond_max=COND_MAX):
    gap = (diag[:, 1] - diag[:, 0]) / np.maximum(diag[:, 2], 1e-300)
    return (gap >= gap_min) & (diag[:, 3] <= cond_max) & (diag[:, 2] > 0)


def compare_projection(gpu_xyz, gpu_n, gpu_st, o_xyz, o_n, o_st, o_diag, D, pos_tol=POS_TOL,
                       normal_tol=NORMAL_TOL, min_well_posed=0.5, gap_min=GAP_MIN, cond_max=COND_MAX):
    """Element-wise comparison on the well-posed mask; returns a report.
    Normals: the unoriented angle on every well-posed point, and the
    oriented angle (the canonical sign included) on the well-posed points
    whose sign the oracle normal decides by a margin (SIGN_MARGIN)."""
    mask = well_posed(o_diag, gap_min, cond_max)
    assert mask.mean() >= min_well_posed, f"well-posed fraction {mask.mean():.3f}"
    pos_err = np.linalg.norm(gpu_xyz.astype(np.float64) - o_xyz, axis=1) / D
    gn = gpu_n.astype(np.float64)
    cross = np.linalg.norm(np.cross(gn, o_n), axis=1)
    dot = (gn * o_n).sum(1)
    ang = np.arctan2(cross, np.abs(dot))
    oriented = np.arctan2(cross, dot)
    mag = np.sort(np.abs(o_n), axis=1)
    decided = mask & ((mag[:, 2] - mag[:, 1]) > SIGN_MARGIN)
    st_gpu = gpu_st & 3
    rep = {
        "well_posed": float(mask.mean()),
        "max_pos_err": float(pos_err[mask].max()) if mask.any() else 0.0,
        "max_angle": float(ang[mask].max()) if mask.any() else 0.0,
        "max_oriented_angle": float(oriented[decided].max()) if decided.any() else 0.0,
        "sign_undecided_well_posed": int((mask & ~decided).sum()),
        "status_mismatch_well_posed": int((st_gpu[mask] != o_st[mask]).sum()),
        "excluded": int((~mask).sum()),
        "excluded_max_pos_err": float(pos_err[~mask].max()) if (~mask).any() else 0.0,
    }
    if mask.any():
        worst = int(np.argmax(np.where(mask, pos_err, -1)))
        rep["worst_gap"] = float((o_diag[worst, 1] - o_diag[worst, 0]) / o_diag[worst, 2])
    assert rep["status_mismatch_well_posed"] == 0, rep
    assert rep["max_pos_err"] <= pos_tol, rep
    assert rep["max_angle"] <= normal_tol, rep
    assert rep["max_oriented_angle"] <= normal_tol, rep
    return rep


# Adjoint: per point, |g_gpu - g_oracle| <= GRAD_TOL |g_oracle| (relative in
# norm) on every point whose gradient takes terms only from well-posed
# neighbourhoods (the projection's mask applied to every query whose row holds
# the point).  Measured on such points: at most 3.1e-4 (FP32, torus with
# outliers), 1.1e-4 (mixed), 4.1e-5 (bumpy spheres).
GRAD_TOL = 1e-3


def clean_targets(rows, diag, n, queries=None, gap_min=GAP_MIN, cond_max=COND_MAX):
    """Mask over the n points: True where every projected point whose row
    holds the point (rows[s] belongs to queries[s], or to point s) is
    well-posed."""
    q = np.arange(rows.shape[0]) if queries is None else np.asarray(queries)
    good = well_posed(diag, gap_min, cond_max)
    tainted = np.zeros(n, bool)
    tainted[rows[~good].ravel()] = True
    tainted[q[~good]] = True
    return ~tainted


def compare_gradient(g, g_o, clean, tol=GRAD_TOL, min_clean=0.5):
    """Per-point relative error in norm on the clean mask; returns a report
    with the excluded fraction and its worst error."""
    err = np.linalg.norm(np.asarray(g, np.float64) - g_o, axis=1)
    scale = np.linalg.norm(g_o, axis=1)
    rel = err / np.maximum(scale, 1e-300)
    rep = {
        "clean": float(clean.mean()),
        "excluded": int((~clean).sum()),
        "max_rel_err": float(rel[clean].max()) if clean.any() else 0.0,
        "excluded_max_rel_err": float(rel[~clean].max()) if (~clean).any() else 0.0,
    }
    assert clean.mean() >= min_clean, rep
    assert np.all(err[clean] <= tol * scale[clean]), rep
    return rep
