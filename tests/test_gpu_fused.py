"""The kNN and the projection in one pass (mls_knn_project, through the C ABI;
Algorithm 1: each point's neighbourhood, then its plane, polynomial and
projection): the rows it can write are the kNN rows bit for bit, and its
results match the oracle's projection (Sec. 1.4, Eq. 1) on the oracle's rows
at the projection tests' tolerances, and the two-pass sorted path's."""
import numpy as np
import pytest
import torch

import oracle
from paper_2401_03365_gb300 import workloads
from tests.gpu_cases import compare_projection, diag_len, knn_case, oracle_knn

pytestmark = pytest.mark.gpu

FUSED_CASES = ["sphere20k_k20", "torus100k_k32", "lattice_ties_k27", "duplicates_k20", "clusters_and_outliers_k16",
               "far_from_origin_k12", "tiny_n_equals_k", "k1"]


@pytest.fixture(scope="module")
def capi():
    from paper_2401_03365_gb300 import build, capi
    build.build()
    return capi


def _h32(xyz, rows):
    """2 x the mean distance to the other points of each row, as float."""
    return float(np.float32(2.0 * oracle.mean_knn_dist(xyz, rows)))


@pytest.mark.parametrize("case", FUSED_CASES)
def test_fused_rows_are_the_knn_rows(capi, case):
    xyz, k = knn_case(case)
    x = torch.from_numpy(xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, k)
    _, _, _, pos = capi.mls_knn_project(grid, k, 0.5, 2, "mixed", with_pos=True)
    pos_ref, _, _ = capi.mls_knn_sorted(grid, k)
    order = capi.mls_grid_order(grid).cpu().numpy()
    torch.cuda.synchronize()
    grid.close()
    assert torch.equal(pos, pos_ref)
    p = pos.cpu().numpy()
    rows = np.empty_like(p)
    rows[order] = order[p]          # row of point order[s] = order of row s
    assert np.array_equal(rows, oracle_knn(xyz, k)[0])


@pytest.mark.parametrize("precision", ["mixed", "fp32"])
@pytest.mark.parametrize("degree", [0, 1, 2])
def test_fused_matches_oracle(capi, degree, precision):
    """A 120k-point torus with 1 % outliers: positions and oriented normals
    against the oracle on well-posed neighbourhoods, statuses equal there."""
    c = workloads.torus(n=120_000, seed=45)
    rows_o, _ = oracle.knn_kdtree(c.xyz, c.k)
    h = _h32(c.xyz, rows_o)
    x = torch.from_numpy(c.xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, c.k)
    g = capi.mls_knn_project(grid, c.k, h, degree, precision)
    torch.cuda.synchronize()
    grid.close()
    o = oracle.project(c.xyz, rows_o, h, degree)
    rep = compare_projection(*(t.cpu().numpy() for t in g), *o, diag_len(c.xyz), min_well_posed=0.3)
    print(rep)


@pytest.mark.parametrize("precision", ["mixed", "fp32"])
@pytest.mark.parametrize("degree", [1, 2])
def test_fused_equals_two_pass(capi, degree, precision):
    """Same rows, same points, same per-point routine: the outputs of
    mls_knn_sorted + mls_project_sorted, bit for bit."""
    c = workloads.torus(n=150_000, seed=46)
    x = torch.from_numpy(c.xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, c.k)
    h = 0.012
    a = capi.mls_knn_project(grid, c.k, h, degree, precision)
    pos, _, _ = capi.mls_knn_sorted(grid, c.k)
    b = capi.mls_project_sorted(grid, pos, h, degree, precision)
    torch.cuda.synchronize()
    grid.close()
    for u, v in zip(a, b):
        assert torch.equal(u, v)


@pytest.mark.parametrize("case", ["lattice_ties_k27", "duplicates_k20", "tiny_n_equals_k", "k1", "planar_k8",
                                  "all_identical_k10"])
def test_fused_edge_cases(capi, case):
    """Ties, duplicates, n = k, k = 1, a plane, identical points: the oracle
    on its own rows (degenerate points output the point itself)."""
    xyz, k = knn_case(case)
    rows_o, _ = oracle_knn(xyz, k)
    h = _h32(xyz, rows_o) if k > 1 else 0.5
    if not h > 0:
        h = 0.5
    o = oracle.project(xyz, rows_o, h, 2)
    x = torch.from_numpy(xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, k)
    g_xyz, g_n, g_st = (t.cpu().numpy() for t in capi.mls_knn_project(grid, k, h, 2, "mixed"))
    torch.cuda.synchronize()
    grid.close()
    deg = o[2] == oracle.STATUS_PLANE_DEGENERATE
    assert np.array_equal(g_st[deg] & 1, o[2][deg])
    assert np.array_equal(g_xyz[deg], xyz[deg])
    compare_projection(g_xyz, g_n, g_st, *o, max(diag_len(xyz), 1e-30), min_well_posed=0.0)


def test_fused_full_size_torus(capi):
    """The 2M-point benchmark cloud (k = 32, degree 2, mixed): every output
    equals the two-pass path's, and a seeded sample of 20k points matches the
    oracle on its own k-d tree rows."""
    c = workloads.torus()
    rng = np.random.default_rng(47)
    q = np.sort(rng.choice(c.n, 20_000, replace=False))
    rows_o, _ = oracle.knn_kdtree(c.xyz, c.k, queries=q)
    x64 = c.xyz.astype(np.float64)
    d = np.linalg.norm(x64[rows_o] - x64[q][:, None, :], axis=2)
    h = float(np.float32(2.0 * d[rows_o != q[:, None]].mean()))
    x = torch.from_numpy(c.xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, c.k)
    a = capi.mls_knn_project(grid, c.k, h, 2, "mixed", with_pos=True)
    pos, _, _ = capi.mls_knn_sorted(grid, c.k)
    b = capi.mls_project_sorted(grid, pos, h, 2, "mixed")
    order = capi.mls_grid_order(grid).cpu().numpy()
    torch.cuda.synchronize()
    grid.close()
    assert torch.equal(a[3], pos)
    for u, v in zip(a[:3], b):
        assert torch.equal(u, v)
    p = a[3].cpu().numpy()
    inv = np.empty_like(order)
    inv[order] = np.arange(order.shape[0], dtype=order.dtype)
    assert np.array_equal(order[p[inv[q]]], rows_o)
    o = oracle.project(c.xyz, rows_o, h, 2, queries=q)
    compare_projection(*(t.cpu().numpy()[q] for t in a[:3]), *o, diag_len(c.xyz), min_well_posed=0.3)


def test_fused_argument_errors(capi):
    xyz, k = knn_case("torus100k_k32")
    x = torch.from_numpy(xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, 33)
    for kk, h, prec, code in ((33, 0.1, "mixed", -2), (0, 0.1, "mixed", -2), (32, 0.0, "mixed", -1),
                              (32, float("nan"), "mixed", -1), (32, 0.1, "fp64", -1)):
        with pytest.raises(capi.MLSError) as e:
            capi.mls_knn_project(grid, kk, h, 2, prec)
        assert e.value.code == code
    with pytest.raises(capi.MLSError) as e:
        capi.mls_knn_project(grid, 32, 0.1, 3, "mixed")
    assert e.value.code == -3
    torch.cuda.synchronize()
    grid.close()
