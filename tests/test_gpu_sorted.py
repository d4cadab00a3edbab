"""The projection in the grid's own order (mls_knn_sorted + mls_project_sorted,
through the C ABI): rows of sorted positions that are the kNN rows, and results
bit-identical to mls_project's on the matching original-index rows, hence
within the oracle tolerances wherever mls_project is."""
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


def _setup(capi, xyz, k):
    x = torch.from_numpy(xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, k)
    pos, idx, key = capi.mls_knn_sorted(grid, k, with_idx=True, with_key=True)
    order = capi.mls_grid_order(grid).clone()
    return x, grid, pos, idx, key, order


@pytest.mark.parametrize("case", ["sphere20k_k20", "torus100k_k32", "heightfield200k_k64", "lattice_ties_k27",
                                  "duplicates_k20", "k33_ragged", "tiny_n_equals_k"])
def test_sorted_rows_are_the_knn_rows(capi, case):
    xyz, k = knn_case(case)
    x, grid, pos, idx, key, order = _setup(capi, xyz, k)
    plain, plain_key = capi.mls_knn(grid, k, with_key=True)
    torch.cuda.synchronize()
    grid.close()
    o = order.cpu().numpy()
    p = pos.cpu().numpy()
    i = idx.cpu().numpy()
    # row s of pos, mapped through the order, is the row of point order[s]
    assert np.array_equal(o[p], i[o])
    assert torch.equal(idx, plain) and torch.equal(key, plain_key)
    assert np.array_equal(i, oracle_knn(xyz, k)[0])


@pytest.mark.parametrize("precision", ["mixed", "fp32"])
@pytest.mark.parametrize("degree", [0, 1, 2])
def test_sorted_projection_equals_mls_project(capi, degree, precision):
    c = workloads.torus(n=120_000, seed=41)
    x, grid, pos, idx, _, order = _setup(capi, c.xyz, c.k)
    h = 2.0 * float(capi.mls_mean_knn_dist(x, idx).item())
    a = capi.mls_project_sorted(grid, pos, h, degree, precision)
    b = capi.mls_project(x, idx, h, degree, precision, order=order)
    torch.cuda.synchronize()
    grid.close()
    for u, v in zip(a, b):
        assert torch.equal(u, v)
    if degree == 2:
        rows = idx.cpu().numpy()
        o_xyz, o_n, o_st, o_diag = oracle.project(c.xyz, rows, float(np.float32(h)), degree)
        rep = compare_projection(*(t.cpu().numpy() for t in a), o_xyz, o_n, o_st, o_diag, diag_len(c.xyz),
                                 min_well_posed=0.3)
        print(rep)


def test_sorted_projection_full_size_torus(capi):
    """The 2M-point benchmark cloud, rows without their original-index copy:
    every output equals mls_project's."""
    c = workloads.torus()
    x = torch.from_numpy(c.xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, c.k)
    pos, none_idx, _ = capi.mls_knn_sorted(grid, c.k)
    assert none_idx is None
    idx, _ = capi.mls_knn(grid, c.k)
    order = capi.mls_grid_order(grid)
    h = 2.0 * float(capi.mls_mean_knn_dist(x, idx).item())
    a = capi.mls_project_sorted(grid, pos, h, 2, "mixed")
    b = capi.mls_project(x, idx, h, 2, "mixed", order=order)
    torch.cuda.synchronize()
    grid.close()
    for u, v in zip(a, b):
        assert torch.equal(u, v)


def test_sorted_argument_errors(capi):
    xyz, k = knn_case("k1")
    x, grid, pos, idx, _, _ = _setup(capi, xyz, k)
    with pytest.raises(capi.MLSError) as e:
        capi.mls_project_sorted(grid, pos, 0.1, 2, "fp64")
    assert e.value.code == -1
    with pytest.raises(capi.MLSError) as e:
        capi.mls_project_sorted(grid, pos, -1.0, 2, "mixed")
    assert e.value.code == -1
    with pytest.raises(capi.MLSError) as e:
        capi.mls_knn_sorted(grid, 65)
    assert e.value.code == -2
    torch.cuda.synchronize()
    grid.close()


@pytest.mark.parametrize("precision", ["mixed", "fp32"])
@pytest.mark.parametrize("degree", [1, 2])
def test_sorted_backward_equals_mls_project_backward(capi, degree, precision):
    """The adjoint in the grid's order: bit-identical gradients (coordinates
    and h) to mls_project_backward with the grid's order."""
    c = workloads.torus(n=120_000, seed=42)
    x, grid, pos, idx, _, order = _setup(capi, c.xyz, c.k)
    h = 2.0 * float(capi.mls_mean_knn_dist(x, idx).item())
    gen = torch.Generator(device="cuda").manual_seed(43)
    gp = torch.randn(c.n, 3, device="cuda", generator=gen)
    gn = 0.1 * torch.randn(c.n, 3, device="cuda", generator=gen)
    a, ah = capi.mls_project_backward_sorted(grid, pos, h, gp, gn, degree, precision)
    b, bh = capi.mls_project_backward(x, idx, h, gp, gn, degree, precision, order=order)
    torch.cuda.synchronize()
    grid.close()
    assert torch.equal(a, b) and torch.equal(ah, bh)


def test_sorted_autograd_equals_the_state_calls(capi):
    """The autograd Function in the grid's order saves the forward's fit state
    and its backward reads it: its gradients equal those of
    mls_project_sorted (with_state) + mls_project_backward_sorted(state) bit
    for bit, and are within rounding of the recomputing unsorted form's."""
    from paper_2401_03365_gb300 import mls
    c = workloads.bumpy_sphere(n=50_000, seed=44)
    x, grid, pos, idx, _, order = _setup(capi, c.xyz, c.k)
    gen = torch.Generator(device="cuda").manual_seed(45)
    gp = torch.randn(c.n, 3, device="cuda", generator=gen)
    gn = 0.1 * torch.randn(c.n, 3, device="cuda", generator=gen)
    xg = x.clone().requires_grad_(True)
    ht = torch.tensor(0.03, device="cuda", requires_grad=True)
    out, nrm, _ = mls.project_differentiable(xg, idx, ht, 2, "fp32", order=order, grid=grid, pos=pos)
    # a linear loss: its cotangents are gp and gn exactly
    ((out * gp).sum() + (nrm * gn).sum()).backward()
    o2, n2, _, state = capi.mls_project_sorted(grid, pos, 0.03, 2, "fp32", with_state=True)
    assert torch.equal(out.detach(), o2) and torch.equal(nrm.detach(), n2)
    gx, gh = capi.mls_project_backward_sorted(grid, pos, 0.03, gp, gn, 2, "fp32", state=state)
    gx_u, gh_u = capi.mls_project_backward(x, idx, 0.03, gp, gn, 2, "fp32", order=order)
    torch.cuda.synchronize()
    grid.close()
    assert torch.equal(xg.grad, gx) and torch.equal(ht.grad.reshape(1), gh)
    scale = gx_u.norm(dim=1).median()
    assert float((gx - gx_u).norm(dim=1).median()) <= 1e-5 * float(scale)
    assert abs(float(gh) - float(gh_u)) <= 1e-3 * abs(float(gh_u))