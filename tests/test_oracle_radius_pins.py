"""Pins of the oracle's radius-R neighbourhoods and of the projection over
variable neighbourhoods with the outlier rule (Sec. 1.4, Sec. 3.3)."""
import numpy as np
import pytest

import oracle
from paper_2401_03365_gb300 import workloads


def _np_keys(xyz, i):
    """The FP32 key of every point from point i, one rounding per operation."""
    d = xyz - xyz[i]
    s = d * d
    return (s[:, 0] + s[:, 1]) + s[:, 2]


def _brute(xyz, R):
    R2 = np.float32(np.float32(R) * np.float32(R))
    rows = []
    for i in range(xyz.shape[0]):
        key = _np_keys(xyz, i)
        sel = np.nonzero(key <= R2)[0]
        rows.append(sel[np.lexsort((sel, key[sel]))])
    return rows


@pytest.mark.parametrize("case", ["random", "lattice_ties", "duplicates"])
def test_radius_sets_equal_brute_force(case):
    rng = np.random.default_rng(11)
    if case == "random":
        xyz, R = rng.uniform(0, 1, (1500, 3)).astype(np.float32), 0.09
    elif case == "lattice_ties":          # axis neighbours exactly at R
        g = np.arange(9, dtype=np.float32) * np.float32(0.25)
        xyz = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
        xyz, R = xyz[rng.permutation(xyz.shape[0])], 0.25
    else:
        base = rng.uniform(0, 1, (200, 3)).astype(np.float32)
        xyz, R = base[rng.integers(0, 200, 1200)], 0.05
    off, rows = oracle.radius_neighbors(xyz, R)
    ref = _brute(xyz, R)
    for i in range(xyz.shape[0]):
        assert np.array_equal(rows[off[i]:off[i + 1]], ref[i]), i
    if case == "lattice_ties":
        interior = np.all((xyz > 0.1) & (xyz < 1.9), axis=1)
        assert np.all(np.diff(off)[interior] == 7)      # itself and its six axis neighbours


def test_rows_of_constant_width_reproduce_the_knn_projection():
    c = workloads.sphere(n=3000, seed=12, k=16)
    idx, _ = oracle.knn_kdtree(c.xyz, 16)
    h = 2 * oracle.mean_knn_dist(c.xyz, idx)
    off = np.arange(c.n + 1, dtype=np.int64) * 16
    a = oracle.project_rows(c.xyz, off, idx.ravel(), h, 2, min_neighbors=3)
    b = oracle.project(c.xyz, idx, h, 2)
    for x, y in zip(a, b[:3]):
        assert np.array_equal(x, y)


def test_outlier_rule_counts_the_other_points():
    """A point with fewer than 3 other points within R is an outlier; with
    exactly 3 it is projected."""
    pts = np.array([[0, 0, 0], [0.1, 0, 0], [0, 0.1, 0], [0, 0, 0.1],        # 0: three others
                    [5, 5, 5], [5.1, 5, 5], [5, 5.1, 5],                      # 4: two others
                    [9, 9, 9]], np.float32)                                   # 7: none
    off, rows = oracle.radius_neighbors(pts, 0.12)
    assert list(np.diff(off)) == [4, 2, 2, 2, 3, 2, 2, 1]
    _, _, st, _ = oracle.project_rows(pts, off, rows, 0.2, 0, min_neighbors=3)
    assert st[0] & oracle.STATUS_OUTLIER == 0
    assert all(st[i] & oracle.STATUS_OUTLIER for i in range(1, 8))


def test_small_neighbourhoods_are_fitted_at_a_lower_degree():
    """Reading R8b: a radius neighbourhood of m points (the point included)
    is fitted at degree 2 only when m >= 12, at degree 1 when m >= 6, else at
    degree 0 (status bit 32 when lowered).  Degrees 1 and 0 move the point to
    its weighted plane, p' = q = r - <n, r - c> n (c the weighted centroid, n
    the eigenvector of the smallest eigenvalue of the weighted covariance),
    which is recomputed here with numpy's symmetric eigensolver."""
    rng = np.random.default_rng(7)
    clouds, sizes = [], (5, 6, 11, 12, 20)
    for s, m in enumerate(sizes):
        c = np.array([10.0 * s, 0.0, 0.0])
        p = c + 0.05 * rng.standard_normal((m, 3)) * np.array([1.0, 1.0, 0.2])
        clouds.append(p)
    xyz = np.concatenate(clouds).astype(np.float32)
    off, rows = oracle.radius_neighbors(xyz, 1.0)
    counts = np.diff(off)
    assert list(counts) == [m for m in sizes for _ in range(m)]
    h = 0.08
    out, nrm, st, _ = oracle.project_rows(xyz, off, rows, h, 2, min_neighbors=3)
    reduced = (st & oracle.STATUS_DEGREE_REDUCED) != 0
    assert np.array_equal(reduced, counts < 12)
    x = xyz.astype(np.float64)
    for i in np.nonzero(counts < 12)[0]:
        nb = x[rows[off[i]:off[i + 1]]]
        w = np.exp(-((nb - x[i]) ** 2).sum(1) / h ** 2)
        c = (w[:, None] * nb).sum(0) / w.sum()
        d = nb - c
        C = (w[:, None, None] * d[:, :, None] * d[:, None, :]).sum(0)
        n = np.linalg.eigh(C)[1][:, 0]
        q = x[i] - np.dot(n, x[i] - c) * n
        assert np.linalg.norm(out[i] - q) <= 1e-12, i
        assert abs(abs(np.dot(nrm[i], n)) - 1.0) <= 1e-12
    # rows of 6..11 points at degree 2 give the degree-1 result exactly
    sel = (counts >= 6) & (counts < 12)
    out1, _, st1, _ = oracle.project_rows(xyz, off, rows, h, 1, min_neighbors=3)
    assert np.array_equal(out[sel], out1[sel])
    assert not np.any(st1[sel] & oracle.STATUS_DEGREE_REDUCED)
