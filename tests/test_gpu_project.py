"""GPU projection (mls_project through the C ABI, on the GPU's own kNN rows)
against the FP64 oracle (on the oracle's own kNN rows), element by element on
the well-posed mask: positions within 1e-5 of the bounding-box diagonal,
normals within 1e-4 rad, equal status bits."""
import numpy as np
import pytest
import torch

import oracle
from paper_2401_03365_gb300 import workloads
from tests.gpu_cases import compare_projection, diag_len, knn_case, oracle_knn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    from paper_2401_03365_gb300 import build, capi
    build.build()
    return capi


def gpu_pipeline(capi, xyz, k, h, degree, precision, use_order=True):
    x = torch.from_numpy(xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, k)
    idx, _ = capi.mls_knn(grid, k)
    order = capi.mls_grid_order(grid) if use_order else None
    out, nrm, st = capi.mls_project(x, idx, h, degree, precision, order=order)
    torch.cuda.synchronize()
    res = out.cpu().numpy(), nrm.cpu().numpy(), st.cpu().numpy(), idx.cpu().numpy()
    grid.close()
    return res


def h32(xyz, idx):
    return float(np.float32(2.0 * oracle.mean_knn_dist(xyz, idx)))


@pytest.mark.parametrize("precision", ["fp32", "mixed", "fp64"])
@pytest.mark.parametrize("degree", [0, 1, 2])
def test_sphere20k(capi, precision, degree):
    c = workloads.sphere()
    idx_o, _ = oracle.knn_kdtree(c.xyz, c.k)
    h = h32(c.xyz, idx_o)
    o_xyz, o_n, o_st, o_diag = oracle.project(c.xyz, idx_o, h, degree)
    g_xyz, g_n, g_st, g_idx = gpu_pipeline(capi, c.xyz, c.k, h, degree, precision)
    assert np.array_equal(g_idx, idx_o)
    D = diag_len(c.xyz)
    if precision == "fp64":
        compare_projection(g_xyz, g_n, g_st, o_xyz, o_n, o_st, o_diag, D, pos_tol=1e-7, normal_tol=1e-6,
                           gap_min=1e-5, cond_max=1e12)
    else:
        compare_projection(g_xyz, g_n, g_st, o_xyz, o_n, o_st, o_diag, D)
    if precision == "mixed":
        assert set(np.unique(g_st)) <= {0, 4}


@pytest.mark.parametrize("precision", ["fp32", "mixed", "fp64"])
def test_torus_with_outliers(capi, precision):
    c = workloads.torus(n=100_000, seed=12)
    idx_o, _ = oracle.knn_kdtree(c.xyz, c.k)
    h = h32(c.xyz, idx_o)
    o = oracle.project(c.xyz, idx_o, h, 2)
    g_xyz, g_n, g_st, g_idx = gpu_pipeline(capi, c.xyz, c.k, h, 2, precision)
    D = diag_len(c.xyz)
    kw = dict(pos_tol=1e-7, normal_tol=1e-6, gap_min=1e-5, cond_max=1e12) if precision == "fp64" else {}
    compare_projection(g_xyz, g_n, g_st, *o, D, min_well_posed=0.3, **kw)


def test_heightfield_k64(capi):
    c = workloads.heightfield(n=200_000, seed=13)
    idx_o, _ = oracle.knn_kdtree(c.xyz, c.k)
    h = h32(c.xyz, idx_o)
    o = oracle.project(c.xyz, idx_o, h, 2)
    g = gpu_pipeline(capi, c.xyz, c.k, h, 2, "mixed")
    compare_projection(*g[:3], *o, diag_len(c.xyz), min_well_posed=0.3)


def test_bumpy_sphere_fp32(capi):
    c = workloads.bumpy_sphere(n=100_000, seed=15)
    idx_o, _ = oracle.knn_kdtree(c.xyz, c.k)
    h = h32(c.xyz, idx_o)
    o = oracle.project(c.xyz, idx_o, h, 2)
    g = gpu_pipeline(capi, c.xyz, c.k, h, 2, "fp32", use_order=False)
    compare_projection(*g[:3], *o, diag_len(c.xyz))


def test_full_size_torus_sampled(capi):
    """The benchmark workload (2M points, k = 32, mixed): the GPU projects
    every point; the oracle projects a seeded sample of 20k points using its
    own k-d tree rows."""
    c = workloads.torus()
    rng = np.random.default_rng(7)
    q = np.sort(rng.choice(c.n, 20_000, replace=False))
    rows, _ = oracle.knn_kdtree(c.xyz, c.k, queries=q)
    x = c.xyz.astype(np.float64)
    d = np.linalg.norm(x[rows] - x[q][:, None, :], axis=2)
    h = float(np.float32(2.0 * d[rows != q[:, None]].mean()))
    o = oracle.project(c.xyz, rows, h, 2, queries=q)
    g_xyz, g_n, g_st, g_idx = gpu_pipeline(capi, c.xyz, c.k, h, 2, "mixed")
    assert np.array_equal(g_idx[q], rows)
    compare_projection(g_xyz[q], g_n[q], g_st[q], *o, diag_len(c.xyz), min_well_posed=0.3)


@pytest.mark.parametrize("case", ["lattice_ties_k27", "planar_k8", "all_identical_k10", "tiny_n_equals_k",
                                  "k33_ragged", "duplicates_k20"])
def test_edge_cases(capi, case):
    xyz, k = knn_case(case)
    idx_o, _ = oracle_knn(xyz, k)
    h = h32(xyz, idx_o)
    if not h > 0:
        h = 0.5
    o_xyz, o_n, o_st, o_diag = oracle.project(xyz, idx_o, h, 2)
    for precision in ("fp32", "mixed", "fp64"):
        g_xyz, g_n, g_st, _ = gpu_pipeline(capi, xyz, k, h, 2, precision)
        D = max(diag_len(xyz), 1e-30)
        # the oracle's degenerate points output r exactly: so must the GPU
        deg = o_st == oracle.STATUS_PLANE_DEGENERATE
        if precision != "fp32":
            assert np.array_equal(g_st[deg] & 1, o_st[deg])
            assert np.array_equal(g_xyz[deg], xyz[deg])
        compare_projection(g_xyz, g_n, g_st, o_xyz, o_n, o_st, o_diag, D, min_well_posed=0.0)


def test_deterministic(capi):
    c = workloads.torus(n=100_000, seed=12)
    a = gpu_pipeline(capi, c.xyz, c.k, 0.01, 2, "mixed")
    b = gpu_pipeline(capi, c.xyz, c.k, 0.01, 2, "mixed")
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_order_does_not_change_results(capi):
    c = workloads.sphere(n=30_000, seed=3)
    a = gpu_pipeline(capi, c.xyz, c.k, 0.08, 2, "fp32", use_order=True)
    b = gpu_pipeline(capi, c.xyz, c.k, 0.08, 2, "fp32", use_order=False)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
