"""mls_knn_project_sorted (the kNN and the projection pipelined, through the C
ABI; Algorithm 1's neighbourhoods and Sec. 1.4's projection): every output,
the rows and the fit state included, equals mls_knn_sorted followed by
mls_project_sorted bit for bit (those two are oracle-checked elsewhere), and a
sample of the 2M-point cloud matches the oracle directly."""
import numpy as np
import pytest
import torch

import oracle
from paper_2401_03365_gb300 import workloads
from tests.gpu_cases import compare_projection, diag_len, knn_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    from paper_2401_03365_gb300 import build, capi
    build.build()
    return capi


def _both(capi, grid, k, h, degree, precision, state):
    a = capi.mls_knn_project_sorted(grid, k, h, degree, precision, with_state=state)
    pos, _, _ = capi.mls_knn_sorted(grid, k)
    b = capi.mls_project_sorted(grid, pos, h, degree, precision, with_state=state)
    return a, (pos,) + tuple(b)


@pytest.mark.parametrize("state", [False, True])
@pytest.mark.parametrize("precision", ["mixed", "fp32"])
@pytest.mark.parametrize("degree", [0, 1, 2])
def test_pipelined_equals_the_two_calls(capi, degree, precision, state):
    c = workloads.torus(n=150_000, seed=57)
    x = torch.from_numpy(c.xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, c.k)
    a, b = _both(capi, grid, c.k, 0.012, degree, precision, state)
    torch.cuda.synchronize()
    grid.close()
    assert len(a) == len(b)
    for u, v in zip(a, b):
        assert torch.equal(u, v)


@pytest.mark.parametrize("case", ["clusters_and_outliers_k16", "lattice_ties_k64", "duplicates_k20", "tiny_n_equals_k",
                                  "k1", "k33_ragged", "far_from_origin_k12"])
def test_pipelined_edge_cases(capi, case):
    """Many sparse queries, k = 64 and 33, ties, duplicates, n = k, k = 1."""
    xyz, k = knn_case(case)
    x = torch.from_numpy(xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, k)
    h = float(max(diag_len(xyz), 1e-3)) * 0.02
    a, b = _both(capi, grid, k, h, 2, "mixed", True)
    torch.cuda.synchronize()
    grid.close()
    for u, v in zip(a, b):
        assert torch.equal(u, v)


def test_pipelined_repeated_and_rebuilt(capi):
    """The grid's side stream and events are reused across calls and grid
    rebuilds; every call still equals the two-call form."""
    c1 = workloads.torus(n=80_000, seed=58)
    c2 = workloads.bumpy_sphere(n=60_000, seed=59)
    grid = None
    for c in (c1, c2, c1):
        x = torch.from_numpy(c.xyz).cuda()
        grid = capi.mls_build_grid(x, 0.0, c.k, grid=grid)
        for _ in range(2):
            a, b = _both(capi, grid, c.k, 0.02, 2, "mixed", False)
            for u, v in zip(a, b):
                assert torch.equal(u, v)
    torch.cuda.synchronize()
    grid.close()


def test_pipelined_full_size_torus(capi):
    """The benchmark cloud (2M points, k = 32, mixed, state saved): equal to
    the two calls; a seeded 20k sample against the oracle on its own rows."""
    c = workloads.torus()
    rng = np.random.default_rng(60)
    q = np.sort(rng.choice(c.n, 20_000, replace=False))
    rows_o, _ = oracle.knn_kdtree(c.xyz, c.k, queries=q)
    x64 = c.xyz.astype(np.float64)
    d = np.linalg.norm(x64[rows_o] - x64[q][:, None, :], axis=2)
    h = float(np.float32(2.0 * d[rows_o != q[:, None]].mean()))
    x = torch.from_numpy(c.xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, c.k)
    a, b = _both(capi, grid, c.k, h, 2, "mixed", True)
    order = capi.mls_grid_order(grid).cpu().numpy()
    torch.cuda.synchronize()
    grid.close()
    for u, v in zip(a, b):
        assert torch.equal(u, v)
    p = a[0].cpu().numpy()
    inv = np.empty_like(order)
    inv[order] = np.arange(order.shape[0], dtype=order.dtype)
    assert np.array_equal(order[p[inv[q]]], rows_o)
    o = oracle.project(c.xyz, rows_o, h, 2, queries=q)
    compare_projection(*(t.cpu().numpy()[q] for t in a[1:4]), *o, diag_len(c.xyz), min_well_posed=0.3)


def test_pipelined_argument_errors(capi):
    xyz, k = knn_case("torus100k_k32")
    x = torch.from_numpy(xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, k)
    for kk, h, prec, deg, code in ((65, 0.1, "mixed", 2, -2), (32, -1.0, "mixed", 2, -1), (32, 0.1, "fp64", 2, -1),
                                   (32, 0.1, "mixed", 5, -3)):
        with pytest.raises(capi.MLSError) as e:
            capi.mls_knn_project_sorted(grid, kk, h, deg, prec)
        assert e.value.code == code
    torch.cuda.synchronize()
    grid.close()


@pytest.mark.parametrize("precision", ["mixed", "fp32"])
def test_offsets_from_the_pipelined_call(capi, precision):
    """The adjoint's bucket offsets counted beside the forward: the gradients
    (coordinates and h) equal those of the adjoint counting its own, bit for
    bit, with and without the fit state."""
    c = workloads.torus(n=150_000, seed=61)
    x = torch.from_numpy(c.xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, c.k)
    off = torch.empty(c.n + 1, dtype=torch.int32, device="cuda")
    pos, _, _, _, state = capi.mls_knn_project_sorted(grid, c.k, 0.012, 2, precision, with_state=True,
                                                      out_offsets=off)
    gen = torch.Generator(device="cuda").manual_seed(62)
    gp = torch.randn(c.n, 3, device="cuda", generator=gen)
    gn = 0.1 * torch.randn(c.n, 3, device="cuda", generator=gen)
    for st in (state, None):
        a, ah = capi.mls_project_backward_sorted(grid, pos, 0.012, gp, gn, 2, precision, state=st, offsets=off)
        b, bh = capi.mls_project_backward_sorted(grid, pos, 0.012, gp, gn, 2, precision, state=st)
        assert torch.equal(a, b) and torch.equal(ah, bh)
    # the offsets are the exclusive prefix of the reverse degrees
    deg = torch.bincount(pos.reshape(-1).long(), minlength=c.n)
    ref = torch.zeros(c.n + 1, dtype=torch.int64, device="cuda")
    ref[1:] = torch.cumsum(deg, 0)
    torch.cuda.synchronize()
    grid.close()
    assert torch.equal(off.long(), ref)
