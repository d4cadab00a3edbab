"""GPU adjoint (mls_project_backward through the C ABI) against the FP64
oracle's adjoint, itself pinned to central differences on the CPU.  Every
point whose gradient takes terms only from well-posed neighbourhoods must be
within 1e-3 of the oracle's gradient, relative in norm; the rest are counted
and their worst error reported."""
import numpy as np
import pytest
import torch

import oracle
from paper_2401_03365_gb300 import workloads
from tests.gpu_cases import GRAD_TOL, clean_targets, compare_gradient

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    from paper_2401_03365_gb300 import build, capi
    build.build()
    return capi


def _setup(capi, cloud, k, degree, seed):
    x = torch.from_numpy(cloud.xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, k)
    idx, _ = capi.mls_knn(grid, k)
    order = capi.mls_grid_order(grid).clone()
    torch.cuda.synchronize()
    grid.close()
    idx_o, _ = oracle.knn_kdtree(cloud.xyz, k)
    assert np.array_equal(idx.cpu().numpy(), idx_o)
    h = float(np.float32(2.0 * oracle.mean_knn_dist(cloud.xyz, idx_o)))
    rng = np.random.default_rng(seed)
    gp = rng.standard_normal((cloud.n, 3)).astype(np.float32)
    gn = rng.standard_normal((cloud.n, 3)).astype(np.float32)
    return x, idx, order, idx_o, h, gp, gn


@pytest.mark.parametrize("degree", [1, 2])
@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_backward_matches_oracle_adjoint(capi, degree, precision):
    c = workloads.bumpy_sphere(n=20_000, seed=31, k=16)
    x, idx, order, idx_o, h, gp, gn = _setup(capi, c, 16, degree, 7)
    gx, gh = capi.mls_project_backward(x, idx, h, torch.from_numpy(gp).cuda(), torch.from_numpy(gn).cuda(),
                                       degree, precision, order=order)
    torch.cuda.synchronize()
    g_o, gh_o = oracle.project_grad(c.xyz, idx_o, h, degree, gp.astype(np.float64), gn.astype(np.float64))
    diag = oracle.project(c.xyz, idx_o, h, degree)[3]
    clean = clean_targets(idx_o, diag, c.n)
    rep = compare_gradient(gx.cpu().numpy(), g_o, clean, min_clean=0.99)
    print(rep)
    # dL/dh sums every point's term: held to the same relative bound
    assert abs(float(gh.item()) - gh_o) <= GRAD_TOL * abs(gh_o)


def test_backward_with_outliers_matches_on_well_posed_neighbourhoods(capi):
    """Noisy torus with outliers: points whose gradient comes only from
    well-posed neighbourhoods (every point that has them as a neighbour is
    well-posed) match the oracle."""
    c = workloads.torus(n=60_000, seed=17)
    x, idx, order, idx_o, h, gp, gn = _setup(capi, c, 32, 2, 8)
    gx, gh = capi.mls_project_backward(x, idx, h, torch.from_numpy(gp).cuda(), torch.from_numpy(gn).cuda(),
                                       2, "mixed", order=order)
    torch.cuda.synchronize()
    g_o, _ = oracle.project_grad(c.xyz, idx_o, h, 2, gp.astype(np.float64), gn.astype(np.float64))
    _, _, _, diag = oracle.project(c.xyz, idx_o, h, 2)
    # a target is clean when every source that lists it is well-posed
    clean = clean_targets(idx_o, diag, c.n)
    rep = compare_gradient(gx.cpu().numpy(), g_o, clean, min_clean=0.9)
    print(rep)


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_backward_torus_all_points(capi, precision):
    """200,000 torus points with outliers, every point compared (FP32 and
    mixed): the clean mask holds ~99 %."""
    c = workloads.torus(n=200_000, seed=21)
    x, idx, order, idx_o, h, gp, gn = _setup(capi, c, 32, 2, 9)
    gx, _ = capi.mls_project_backward(x, idx, h, torch.from_numpy(gp).cuda(), torch.from_numpy(gn).cuda(),
                                      2, precision, order=order)
    torch.cuda.synchronize()
    g_o, _ = oracle.project_grad(c.xyz, idx_o, h, 2, gp.astype(np.float64), gn.astype(np.float64))
    diag = oracle.project(c.xyz, idx_o, h, 2)[3]
    rep = compare_gradient(gx.cpu().numpy(), g_o, clean_targets(idx_o, diag, c.n), min_clean=0.95)
    print(rep)


def test_backward_deterministic(capi):
    c = workloads.torus(n=100_000, seed=18)
    x = torch.from_numpy(c.xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, 32)
    idx, _ = capi.mls_knn(grid, 32)
    order = capi.mls_grid_order(grid).clone()
    gp = torch.randn(c.n, 3, device="cuda")
    a, ah = capi.mls_project_backward(x, idx, 0.02, gp, None, 2, "mixed", order=order)
    a, ah = a.clone(), ah.clone()
    b, bh = capi.mls_project_backward(x, idx, 0.02, gp, None, 2, "mixed")
    torch.cuda.synchronize()
    grid.close()
    assert torch.equal(a, b) and torch.equal(ah, bh)


def test_backward_independent_of_processing_order(capi):
    """Each gradient is the exact (fixed-point) sum of its terms, rounded
    once: a random processing order gives bit-identical coordinates' gradients
    to the grid order; dL/dh (double partial sums per block) agrees to
    rounding."""
    c = workloads.bumpy_sphere(n=60_000, seed=19)
    x = torch.from_numpy(c.xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, 32)
    idx, _ = capi.mls_knn(grid, 32)
    order = capi.mls_grid_order(grid).clone()
    gen = torch.Generator(device="cuda").manual_seed(20)
    gp = torch.randn(c.n, 3, device="cuda", generator=gen)
    gn = 0.1 * torch.randn(c.n, 3, device="cuda", generator=gen)
    perm = torch.randperm(c.n, device="cuda", generator=gen).to(torch.int32)
    a, ah = capi.mls_project_backward(x, idx, 0.03, gp, gn, 2, "mixed", order=order)
    a, ah = a.clone(), ah.clone()
    b, bh = capi.mls_project_backward(x, idx, 0.03, gp, gn, 2, "mixed", order=perm)
    torch.cuda.synchronize()
    grid.close()
    assert torch.equal(a, b)
    assert abs(float(ah) - float(bh)) <= 1e-6 * abs(float(ah))


def test_autograd_function(capi):
    from paper_2401_03365_gb300 import mls
    c = workloads.bumpy_sphere(n=10_000, seed=40, k=16)
    x = torch.from_numpy(c.xyz).cuda().requires_grad_(True)
    grid = capi.mls_build_grid(x.detach(), 0.0, 16)
    idx, _ = capi.mls_knn(grid, 16)
    torch.cuda.synchronize()
    grid.close()
    h = torch.tensor(0.05, device="cuda", requires_grad=True)
    out, nrm, st = mls.project_differentiable(x, idx, h)
    loss = (out.norm(dim=1) - 1.0).pow(2).sum() + 0.1 * nrm[:, 2].sum()
    loss.backward()
    gp = (2 * (out.norm(dim=1) - 1.0) / out.norm(dim=1)).unsqueeze(1) * out
    gn = torch.zeros_like(nrm)
    gn[:, 2] = 0.1
    gx, gh = capi.mls_project_backward(x.detach(), idx, 0.05, gp.detach().contiguous(), gn)
    torch.cuda.synchronize()
    assert torch.allclose(x.grad, gx, rtol=1e-4, atol=1e-6 * gx.abs().max().item())
    assert torch.allclose(h.grad.reshape(1), gh, rtol=1e-4)


def test_backward_full_size_torus_sampled(capi):
    """The benchmark workload (2M points with outliers, k = 32, mixed, grid
    order): the gradient at a seeded sample of points j equals the sum over
    the queries whose rows hold j (and j itself); the oracle's adjoint over
    exactly those queries gives it in FP64."""
    c = workloads.torus()
    x = torch.from_numpy(c.xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, c.k)
    idx, _ = capi.mls_knn(grid, c.k)
    order = capi.mls_grid_order(grid)
    h = 2.0 * float(capi.mls_mean_knn_dist(x, idx).item())
    rng = np.random.default_rng(31)
    gp = rng.standard_normal((c.n, 3)).astype(np.float32)
    gn = (0.1 * rng.standard_normal((c.n, 3))).astype(np.float32)
    gx, _ = capi.mls_project_backward(x, idx, h, torch.from_numpy(gp).cuda(), torch.from_numpy(gn).cuda(), 2,
                                      "mixed", order=order)
    torch.cuda.synchronize()
    grid.close()
    rows = idx.cpu().numpy()
    g = gx.cpu().numpy().astype(np.float64)
    targets = np.sort(rng.choice(c.n, 300, replace=False))
    hit = np.isin(rows, targets).any(axis=1)
    hit[targets] = True
    queries = np.nonzero(hit)[0]
    # the sampled rows must be the oracle's own rows
    rows_o, _ = oracle.knn_kdtree(c.xyz, c.k, queries=queries)
    assert np.array_equal(rows_o, rows[queries])
    hf = float(np.float32(h))
    g_o, _ = oracle.project_grad(c.xyz, rows_o, hf, 2, gp.astype(np.float64), gn.astype(np.float64),
                                 queries=queries)
    # clean targets: every query whose row holds them is well-posed
    diag = oracle.project(c.xyz, rows_o, hf, 2, queries=queries)[3]
    clean = clean_targets(rows_o, diag, c.n, queries=queries)[targets]
    rep = compare_gradient(g[targets], g_o[targets], clean, min_clean=0.9)
    print(rep)
