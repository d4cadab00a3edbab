"""GPU kNN (mls_build_grid + mls_knn through the C ABI) against the oracle:
identical index rows and bit-identical keys."""
import numpy as np
import pytest
import torch

import oracle
from tests.gpu_cases import KNN_CASES, knn_case, oracle_knn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    from paper_2401_03365_gb300 import build, capi
    build.build()
    return capi


def _gpu_knn(capi, xyz, k):
    x = torch.from_numpy(xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, k)
    idx, key = capi.mls_knn(grid, k, with_key=True)
    order = capi.mls_grid_order(grid).cpu().numpy()
    torch.cuda.synchronize()
    grid.close()
    return idx.cpu().numpy(), key.cpu().numpy(), order


@pytest.mark.parametrize("case", KNN_CASES)
def test_knn_bit_exact(capi, case):
    xyz, k = knn_case(case)
    idx_o, key_o = oracle_knn(xyz, k)
    idx_g, key_g, order = _gpu_knn(capi, xyz, k)
    bad = np.nonzero((idx_g != idx_o).any(1))[0]
    assert bad.size == 0, f"{bad.size} rows differ, first {bad[:5]}: gpu {idx_g[bad[0]]} oracle {idx_o[bad[0]]}"
    assert np.array_equal(key_g.view(np.uint32), key_o.view(np.uint32))
    assert np.array_equal(np.sort(order), np.arange(xyz.shape[0]))


def test_knn_full_size_torus_sampled(capi):
    """2M-point torus with outliers (the benchmark workload): the GPU rows of a
    seeded sample of queries, the first and last points of the grid order
    and every outlier-region point in the sample, against the oracle's k-d
    tree over the whole cloud."""
    from paper_2401_03365_gb300 import workloads
    c = workloads.torus()
    idx_g, key_g, order = _gpu_knn(capi, c.xyz, c.k)
    rng = np.random.default_rng(99)
    q = np.unique(np.concatenate([rng.integers(0, c.n, 20_000), order[:64], order[-64:]]))
    idx_o, key_o = oracle.knn_kdtree(c.xyz, c.k, queries=q)
    assert np.array_equal(idx_g[q], idx_o)
    assert np.array_equal(key_g[q].view(np.uint32), key_o.view(np.uint32))


def test_knn_deterministic_and_grid_reuse(capi):
    """A rebuilt handle orders the keys only from one level below its last
    base level: rows stay exact when it is rebuilt on another cloud (whose
    base level may be finer), on the first again, and with another k."""
    xyz, k = knn_case("torus100k_k32")
    x = torch.from_numpy(xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, k)
    a, _ = capi.mls_knn(grid, k)
    a = a.clone()
    # rebuild in place on another cloud, then on the first again
    ys, _ = knn_case("sphere20k_k20")
    y = torch.from_numpy(ys).cuda()
    grid = capi.mls_build_grid(y, 0.0, k, grid=grid)
    b, _ = capi.mls_knn(grid, k)
    b = b.clone()
    grid = capi.mls_build_grid(x, 0.0, k, grid=grid)
    c, _ = capi.mls_knn(grid, k)
    c = c.clone()
    grid = capi.mls_build_grid(x, 0.0, 8, grid=grid)
    d, _ = capi.mls_knn(grid, 8)
    grid = capi.mls_build_grid(x, 0.0, 8, grid=grid)
    e, _ = capi.mls_knn(grid, 8)
    torch.cuda.synchronize()
    grid.close()
    assert torch.equal(a, c)
    assert np.array_equal(a.cpu().numpy(), oracle_knn(xyz, k)[0])
    assert np.array_equal(b.cpu().numpy(), oracle_knn(ys, k)[0])
    idx8 = oracle_knn(xyz, 8)[0]
    assert np.array_equal(d.cpu().numpy(), idx8)
    assert np.array_equal(e.cpu().numpy(), idx8)


def test_rebuild_from_a_much_sparser_cloud(capi):
    """A handle built on 2,000 points of a torus, then rebuilt on 100,000
    points of the same torus: the partial sort (from one level below the
    sparse cloud's base) cannot resolve the dense cloud's base level, so the
    build sorts again in full; rows exact either way."""
    from paper_2401_03365_gb300 import workloads
    sparse = workloads.torus(n=2_000, seed=31, outlier_frac=0.0).xyz
    dense = workloads.torus(n=100_000, seed=32, outlier_frac=0.0).xyz
    k = 16
    grid = capi.mls_build_grid(torch.from_numpy(sparse).cuda(), 0.0, k)
    a, _ = capi.mls_knn(grid, k)
    a = a.clone()
    xd = torch.from_numpy(dense).cuda()
    grid = capi.mls_build_grid(xd, 0.0, k, grid=grid)
    b, _ = capi.mls_knn(grid, k)
    b = b.clone()
    grid = capi.mls_build_grid(xd, 0.0, k, grid=grid)
    c, _ = capi.mls_knn(grid, k)
    torch.cuda.synchronize()
    grid.close()
    assert np.array_equal(a.cpu().numpy(), oracle_knn(sparse, k)[0])
    idx_d = oracle_knn(dense, k)[0]
    assert np.array_equal(b.cpu().numpy(), idx_d)
    assert np.array_equal(c.cpu().numpy(), idx_d)


@pytest.mark.parametrize("cell_size", [0.002, 0.05, 1.0])
def test_knn_independent_of_cell_size(capi, cell_size):
    xyz, k = knn_case("sphere20k_k20")
    x = torch.from_numpy(xyz).cuda()
    grid = capi.mls_build_grid(x, cell_size, k)
    idx, _ = capi.mls_knn(grid, k)
    torch.cuda.synchronize()
    grid.close()
    idx_o, _ = oracle.knn_kdtree(xyz, k)
    assert np.array_equal(idx.cpu().numpy(), idx_o)


def test_isolated_queries(capi):
    """From 2^18 points, queries alone in a cell two base cells wide are taken
    first by the chain pass and searched in full: a 300,000-point torus with
    1 % outliers, plus single outliers far away and pairs of outliers that
    share a cell (those go through the chain's own deferral).  Every row and
    key equals the oracle's, rows of sorted positions included, and the kNN
    reports at least the planted far outliers as searched outside the runs."""
    from paper_2401_03365_gb300 import workloads
    rng = np.random.default_rng(101)
    c = workloads.torus(n=300_000, seed=100)
    far = rng.uniform(-1, 1, (30, 3)) * np.array([6.0, 6.0, 3.0]) + np.array([0.0, 0.0, 4.0])
    pairs = np.repeat(rng.uniform(-1, 1, (10, 3)) * 3.0 + np.array([0.0, 0.0, -4.0]), 2, axis=0)
    pairs[1::2] += 1e-4
    xyz = np.concatenate([c.xyz, far, pairs]).astype(np.float32)
    k = 32
    idx_o, key_o = oracle.knn_kdtree(xyz, k)
    x = torch.from_numpy(xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, k)
    idx_g, key_g = capi.mls_knn(grid, k, with_key=True)
    searched = capi.mls_knn_deferred(grid)
    pos, idx_s, _ = capi.mls_knn_sorted(grid, k, with_idx=True)
    order = capi.mls_grid_order(grid).cpu().numpy()
    torch.cuda.synchronize()
    grid.close()
    assert np.array_equal(idx_g.cpu().numpy(), idx_o)
    assert np.array_equal(key_g.cpu().numpy().view(np.uint32), key_o.view(np.uint32))
    assert np.array_equal(idx_s.cpu().numpy(), idx_o)
    p = pos.cpu().numpy()
    rows = np.empty_like(p)
    rows[order] = order[p]
    assert np.array_equal(rows, idx_o)
    assert searched >= far.shape[0]


def test_single_point(capi):
    """n = k = 1: the one point is alone in every cell; its row is itself."""
    xyz = np.array([[0.25, -1.5, 3.0]], np.float32)
    idx, key, order = _gpu_knn(capi, xyz, 1)
    assert idx.tolist() == [[0]] and key.tolist() == [[0.0]] and order.tolist() == [0]
