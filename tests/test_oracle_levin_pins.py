"""Pins of the oracle's projection with weights about q (Sec. 1.4, Eq. 1):
closed forms the paper's definition reduces to, and invariants."""
import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
from paper_2401_03365_gb300 import workloads


def _paraboloid_with_axis_query(alpha=0.8, z0=0.05, n_side=15, spacing=0.05):
    """A grid point-symmetric about the z axis on z = alpha (x^2 + y^2), and a
    query on the axis at height z0 (not one of the neighbours)."""
    g = (np.arange(n_side) - n_side // 2) * spacing
    X, Y = np.meshgrid(g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), alpha * (X.ravel() ** 2 + Y.ravel() ** 2)], 1)
    pts = np.concatenate([pts, [[0.0, 0.0, z0]]]).astype(np.float32)
    m = pts.shape[0] - 1
    row = np.arange(m, dtype=np.int32)[None, :]
    return pts, row, m


@pytest.mark.parametrize("degree", [0, 1])
def test_axis_query_on_paraboloid_is_the_weighted_height_fixed_point(degree):
    """By symmetry the plane is horizontal and q = (0, 0, D) on the axis; with
    the weights about q, D is the weighted mean height at the fixed point
    D = sum w_j(D) z_j / sum w_j(D), w_j(D) = exp(-(x_j^2 + y_j^2 + (z_j - D)^2) / h^2).
    Degree 0 and 1 fits add nothing on the axis (the heights average to 0
    under the same weights; the linear terms vanish by symmetry), so the
    result is (0, 0, D).  The weights about r instead give the mean height
    with weights about (0, 0, z0): a different point."""
    pts, row, m = _paraboloid_with_axis_query()
    P = pts[:m].astype(np.float64)
    h = 0.12
    r2 = P[:, 0] ** 2 + P[:, 1] ** 2

    def wmean(c):
        w = np.exp(-(r2 + (P[:, 2] - c) ** 2) / h ** 2)
        return (w * P[:, 2]).sum() / w.sum()

    D = brentq(lambda c: wmean(c) - c, -1.0, 1.0, xtol=1e-15)
    out, nrm, st, it = oracle.project_levin(pts, row, h, degree, queries=[m])
    assert st[0] == 0 and it[0] > 1
    assert np.abs(out[0] - [0.0, 0.0, D]).max() < 1e-10
    assert np.abs(np.abs(nrm[0]) - [0.0, 0.0, 1.0]).max() < 1e-12
    simple, _, _, _ = oracle.project(pts, row, h, degree, queries=[m])
    assert abs(simple[0, 2] - wmean(float(pts[m, 2]))) < 1e-10
    assert abs(simple[0, 2] - D) > 1e-4


def test_degree2_reproduces_the_paraboloid_on_the_axis():
    """The quadratic fit reproduces the surface: the result is its vertex."""
    pts, row, m = _paraboloid_with_axis_query()
    out, _, st, _ = oracle.project_levin(pts, row, 0.12, 2, queries=[m])
    assert st[0] == 0
    assert np.abs(out[0]).max() < 1e-10


def test_query_above_a_plane_lands_on_its_foot():
    rng = np.random.default_rng(3)
    P = np.concatenate([rng.uniform(-1, 1, (400, 2)), np.full((400, 1), 0.25)], 1)
    pts = np.concatenate([P, [[0.1, -0.2, 0.4]]]).astype(np.float32)
    row = np.arange(400, dtype=np.int32)[None, :]
    for degree in (0, 1, 2):
        out, nrm, st, _ = oracle.project_levin(pts, row, 0.5, degree, queries=[400])
        assert st[0] == 0
        assert np.abs(out[0] - [pts[400, 0], pts[400, 1], 0.25]).max() < 1e-12
        assert np.abs(nrm[0] - [0, 0, 1]).max() < 1e-12


def test_wide_bandwidth_reduces_to_the_weights_about_r():
    """With h far above the neighbourhood size every weight is 1 to within
    1e-12, wherever the weights are centred: both forms agree (degree 0: the
    coordinates scaled by 1/h leave higher fits singular at such h)."""
    c = workloads.sphere(n=2000, seed=5, k=16)
    rows, _ = oracle.knn_kdtree(c.xyz, 16)
    a, _, sa, _ = oracle.project_levin(c.xyz, rows, 1e5, 0)
    b, _, sb, _ = oracle.project(c.xyz, rows, 1e5, 0)
    ok = (sa == 0) & (sb == 0)
    assert ok.mean() > 0.99
    assert np.abs(a[ok] - b[ok]).max() < 1e-8


def test_rigid_motion_equivariance_exact():
    rng = np.random.default_rng(7)
    c = workloads.torus(n=3000, seed=43, k=16)
    xyz = (np.round(c.xyz.astype(np.float64) * 2 ** 16) / 2 ** 16).astype(np.float32)
    idx, _ = oracle.knn_kdtree(xyz, 16)
    h = 2 * oracle.mean_knn_dist(xyz, idx)
    out, nrm, st, it = oracle.project_levin(xyz, idx, h, 2)
    D = np.linalg.norm(xyz.max(0) - xyz.min(0))
    P = np.eye(3)[rng.permutation(3)] * rng.choice([-1.0, 1.0], 3)[:, None]
    t = rng.integers(-2 ** 17, 2 ** 17, 3) / 2 ** 16
    moved = xyz.astype(np.float64) @ P.T + t
    out2, nrm2, st2, it2 = oracle.project_levin(moved.astype(np.float32), idx, h, 2)
    ok = st == 0
    assert np.array_equal(st, st2)
    assert np.abs(out2[ok] - (out[ok] @ P.T + t)).max() < 1e-10 * D


def test_iteration_limit_sets_the_flag():
    c = workloads.sphere(n=500, seed=6, k=12)
    rows, _ = oracle.knn_kdtree(c.xyz, 12)
    _, _, st, it = oracle.project_levin(c.xyz, rows, 0.2, 2, max_iter=1)
    assert np.all((st & oracle.STATUS_NOT_CONVERGED) != 0) and np.all(it == 1)
    _, _, st, it = oracle.project_levin(c.xyz, rows, 0.2, 2)
    assert np.all((st & oracle.STATUS_NOT_CONVERGED) == 0) and it.max() < 100


def test_diagnostics_of_the_final_plane_on_the_paraboloid_axis():
    """The operator's own diagnostics: at the fixed point q = (0, 0, D) (D
    from brentq, as above) they are the eigenvalues of the weighted
    covariance with the weights about q, and the condition number of the
    degree-1 normal matrix over (x, y) / h with those weights, both computed
    here with numpy."""
    pts, row, m = _paraboloid_with_axis_query()
    P = pts[:m].astype(np.float64)
    h = 0.12
    r2 = P[:, 0] ** 2 + P[:, 1] ** 2

    def weights(c):
        return np.exp(-(r2 + (P[:, 2] - c) ** 2) / h ** 2)

    D = brentq(lambda c: (weights(c) * P[:, 2]).sum() / weights(c).sum() - c, -1.0, 1.0, xtol=1e-15)
    w = weights(D)
    c = (w[:, None] * P).sum(0) / w.sum()
    E = P - c
    C = (w[:, None, None] * E[:, :, None] * E[:, None, :]).sum(0) / w.sum()
    lam = np.linalg.eigvalsh(C)
    phi = np.stack([np.ones(m), P[:, 0] / h, P[:, 1] / h], 1)
    A = (w[:, None, None] * phi[:, :, None] * phi[:, None, :]).sum(0)
    ev = np.linalg.eigvalsh(A)
    _, _, st, _, diag = oracle.project_levin(pts, row, h, 1, queries=[m], with_diag=True)
    assert st[0] == 0
    assert np.allclose(diag[0, :3], lam, rtol=1e-9, atol=1e-14)
    assert abs(diag[0, 3] / (ev[-1] / ev[0]) - 1.0) < 1e-9
    assert abs(diag[0, 4] / w.sum() - 1.0) < 1e-9


def test_diagnostics_reduce_to_the_weights_about_r_for_a_wide_bandwidth():
    c = workloads.sphere(n=2000, seed=5, k=16)
    rows, _ = oracle.knn_kdtree(c.xyz, 16)
    _, _, sa, _, da = oracle.project_levin(c.xyz, rows, 1e5, 0, with_diag=True)
    _, _, sb, db = oracle.project(c.xyz, rows, 1e5, 0)
    ok = (sa == 0) & (sb == 0)
    assert ok.mean() > 0.99
    assert np.allclose(da[ok][:, [0, 1, 2, 4]], db[ok][:, [0, 1, 2, 4]], rtol=1e-6, atol=1e-12)
    assert np.allclose(da[ok][:, 3], 1.0) and np.allclose(db[ok][:, 3], 1.0)
