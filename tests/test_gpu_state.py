"""The fit state saved by the forward for the adjoint (mls_project_sorted with
d_state, mls_project_backward_sorted reading it; through the C ABI): the
forward's outputs are unchanged by saving it, the saved frame, eigenvalues
and status agree with the outputs and with the oracle's plane fit (Sec. 1.4,
Eq. 1), and the gradients of the adjoint that reads it match the FP64
oracle's adjoint at the adjoint tests' tolerance on every clean point."""
import numpy as np
import pytest
import torch

import oracle
from paper_2401_03365_gb300 import workloads
from tests.gpu_cases import GRAD_TOL, clean_targets, compare_gradient, well_posed

pytestmark = pytest.mark.gpu

ST_N, ST_M, ST_LAM, ST_A, ST_STATUS = 4, 1, 13, 16, 28


@pytest.fixture(scope="module")
def capi():
    from paper_2401_03365_gb300 import build, capi
    build.build()
    return capi


def _grid(capi, xyz, k):
    x = torch.from_numpy(xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, k)
    pos, idx, _ = capi.mls_knn_sorted(grid, k, with_idx=True)
    order = capi.mls_grid_order(grid).clone()
    return x, grid, pos, idx, order


@pytest.mark.parametrize("precision", ["mixed", "fp32"])
@pytest.mark.parametrize("degree", [0, 1, 2])
def test_saving_the_state_leaves_the_outputs_unchanged(capi, degree, precision):
    c = workloads.torus(n=120_000, seed=49)
    x, grid, pos, idx, order = _grid(capi, c.xyz, c.k)
    h = 2.0 * float(capi.mls_mean_knn_dist(x, idx).item())
    a = capi.mls_project_sorted(grid, pos, h, degree, precision)
    b = capi.mls_project_sorted(grid, pos, h, degree, precision, with_state=True)
    torch.cuda.synchronize()
    grid.close()
    for u, v in zip(a, b[:3]):
        assert torch.equal(u, v)
    state, o = b[3].cpu().numpy(), order.cpu().numpy()
    # by sorted position s: the status and the normal of point order[s]
    st = state[ST_STATUS].view(np.int32)
    assert np.array_equal(st, b[2].cpu().numpy()[o].astype(np.int32))
    assert np.array_equal(state[ST_N:ST_N + 3].T, b[1].cpu().numpy()[o])
    # coefficients past the basis size are zero
    m = {0: 1, 1: 3, 2: 6}[degree]
    assert not state[ST_A + m:ST_A + 6].any()


def test_saved_eigenvalues_match_the_oracle_plane(capi):
    """The saved covariance eigenvalues (of the unnormalised weighted
    covariance) in ratio to the largest, against the oracle's, on the
    well-posed points of a torus with outliers."""
    c = workloads.torus(n=100_000, seed=50)
    x, grid, pos, idx, order = _grid(capi, c.xyz, c.k)
    rows = idx.cpu().numpy()
    h = float(np.float32(2.0 * oracle.mean_knn_dist(c.xyz, rows)))
    _, _, _, state = capi.mls_project_sorted(grid, pos, h, 2, "mixed", with_state=True)
    torch.cuda.synchronize()
    grid.close()
    o = order.cpu().numpy()
    lam = np.empty((c.n, 3))
    lam[o] = state.cpu().numpy()[ST_LAM:ST_LAM + 3].T
    diag = oracle.project(c.xyz, rows, h, 2)[3]
    good = well_posed(diag)
    assert good.mean() > 0.3
    r_gpu = lam[good, :2] / lam[good, 2:3]
    r_o = diag[good, :2] / diag[good, 2:3]
    gap_gpu = r_gpu[:, 1] - r_gpu[:, 0]
    gap_o = r_o[:, 1] - r_o[:, 0]
    # the FP32 moments carry ~k eps of the largest eigenvalue (k = 32: 2e-6)
    assert np.all(np.abs(r_gpu - r_o) <= 1e-5 + 1e-4 * r_o), np.abs(r_gpu - r_o).max()
    assert np.all(np.abs(gap_gpu - gap_o) <= 1e-3 * gap_o + 1e-5), np.abs(gap_gpu - gap_o).max()


@pytest.mark.parametrize("degree", [1, 2])
@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_adjoint_from_the_state_matches_oracle(capi, degree, precision):
    c = workloads.bumpy_sphere(n=20_000, seed=51, k=16)
    x, grid, pos, idx, order = _grid(capi, c.xyz, 16)
    rows = idx.cpu().numpy()
    idx_o, _ = oracle.knn_kdtree(c.xyz, 16)
    assert np.array_equal(rows, idx_o)
    h = float(np.float32(2.0 * oracle.mean_knn_dist(c.xyz, idx_o)))
    rng = np.random.default_rng(52)
    gp = rng.standard_normal((c.n, 3)).astype(np.float32)
    gn = rng.standard_normal((c.n, 3)).astype(np.float32)
    _, _, _, state = capi.mls_project_sorted(grid, pos, h, degree, precision, with_state=True)
    gx, gh = capi.mls_project_backward_sorted(grid, pos, h, torch.from_numpy(gp).cuda(), torch.from_numpy(gn).cuda(),
                                              degree, precision, state=state)
    torch.cuda.synchronize()
    grid.close()
    g_o, gh_o = oracle.project_grad(c.xyz, idx_o, h, degree, gp.astype(np.float64), gn.astype(np.float64))
    diag = oracle.project(c.xyz, idx_o, h, degree)[3]
    rep = compare_gradient(gx.cpu().numpy(), g_o, clean_targets(idx_o, diag, c.n), min_clean=0.99)
    print(rep)
    assert abs(float(gh.item()) - gh_o) <= GRAD_TOL * abs(gh_o)


def test_adjoint_from_the_state_torus_with_outliers(capi):
    """200,000 torus points with outliers, mixed: every clean point."""
    c = workloads.torus(n=200_000, seed=53)
    x, grid, pos, idx, order = _grid(capi, c.xyz, c.k)
    idx_o, _ = oracle.knn_kdtree(c.xyz, c.k)
    assert np.array_equal(idx.cpu().numpy(), idx_o)
    h = float(np.float32(2.0 * oracle.mean_knn_dist(c.xyz, idx_o)))
    rng = np.random.default_rng(54)
    gp = rng.standard_normal((c.n, 3)).astype(np.float32)
    gn = (0.1 * rng.standard_normal((c.n, 3))).astype(np.float32)
    _, _, _, state = capi.mls_project_sorted(grid, pos, h, 2, "mixed", with_state=True)
    gx, _ = capi.mls_project_backward_sorted(grid, pos, h, torch.from_numpy(gp).cuda(), torch.from_numpy(gn).cuda(),
                                             2, "mixed", state=state)
    torch.cuda.synchronize()
    grid.close()
    g_o, _ = oracle.project_grad(c.xyz, idx_o, h, 2, gp.astype(np.float64), gn.astype(np.float64))
    diag = oracle.project(c.xyz, idx_o, h, 2)[3]
    rep = compare_gradient(gx.cpu().numpy(), g_o, clean_targets(idx_o, diag, c.n), min_clean=0.95)
    print(rep)


def test_adjoint_from_the_state_full_size_torus_sampled(capi):
    """The benchmark step's form (2M points with outliers, k = 32, mixed, the
    state saved and read): the gradient at 300 seeded points against the
    oracle's adjoint over every query whose row holds them."""
    c = workloads.torus()
    x, grid, pos, idx, order = _grid(capi, c.xyz, c.k)
    h = 2.0 * float(capi.mls_mean_knn_dist(x, idx).item())
    rng = np.random.default_rng(55)
    gp = rng.standard_normal((c.n, 3)).astype(np.float32)
    gn = (0.1 * rng.standard_normal((c.n, 3))).astype(np.float32)
    _, _, _, state = capi.mls_project_sorted(grid, pos, h, 2, "mixed", with_state=True)
    gx, _ = capi.mls_project_backward_sorted(grid, pos, h, torch.from_numpy(gp).cuda(), torch.from_numpy(gn).cuda(),
                                             2, "mixed", state=state)
    torch.cuda.synchronize()
    grid.close()
    rows = idx.cpu().numpy()
    g = gx.cpu().numpy().astype(np.float64)
    targets = np.sort(rng.choice(c.n, 300, replace=False))
    hit = np.isin(rows, targets).any(axis=1)
    hit[targets] = True
    queries = np.nonzero(hit)[0]
    rows_o, _ = oracle.knn_kdtree(c.xyz, c.k, queries=queries)
    assert np.array_equal(rows_o, rows[queries])
    hf = float(np.float32(h))
    g_o, _ = oracle.project_grad(c.xyz, rows_o, hf, 2, gp.astype(np.float64), gn.astype(np.float64),
                                 queries=queries)
    diag = oracle.project(c.xyz, rows_o, hf, 2, queries=queries)[3]
    clean = clean_targets(rows_o, diag, c.n, queries=queries)[targets]
    rep = compare_gradient(g[targets], g_o[targets], clean, min_clean=0.9)
    print(rep)


def test_state_argument_checks(capi):
    c = workloads.torus(n=5_000, seed=56)
    x, grid, pos, idx, order = _grid(capi, c.xyz, c.k)
    gp = torch.zeros(c.n, 3, device="cuda")
    with pytest.raises(ValueError):
        capi.mls_project_backward_sorted(grid, pos, 0.02, gp, None, 2, "mixed",
                                         state=torch.zeros((capi.FIT_STATE_FLOATS, c.n - 1), device="cuda"))
    torch.cuda.synchronize()
    grid.close()


@pytest.mark.parametrize("precision", ["mixed", "fp32"])
def test_bandwidth_below_the_spacing_gives_finite_gradients(capi, precision):
    """h below the point spacing (a 150k torus at h = 0.012): outliers whose
    neighbours all lie many h away get negligible weights, and reading R9
    makes their planes degenerate (status bit 1 wherever the oracle's
    normalised covariance is at most 2^-40 D^2, D the largest distance from
    the point to a row entry).  Every gradient is finite,
    from the saved state and recomputed, with both cotangents."""
    c = workloads.torus(n=150_000, seed=61)
    x, grid, pos, idx, order = _grid(capi, c.xyz, c.k)
    h = 0.012
    _, _, st, state = capi.mls_project_sorted(grid, pos, h, 2, precision, with_state=True)
    gen = torch.Generator(device="cuda").manual_seed(62)
    gp = torch.randn(c.n, 3, device="cuda", generator=gen)
    gn = 0.1 * torch.randn(c.n, 3, device="cuda", generator=gen)
    a, ah = capi.mls_project_backward_sorted(grid, pos, h, gp, gn, 2, precision, state=state)
    b, bh = capi.mls_project_backward_sorted(grid, pos, h, gp, gn, 2, precision)
    torch.cuda.synchronize()
    grid.close()
    for g in (a, ah, b, bh):
        assert bool(torch.isfinite(g).all())
    rows = idx.cpu().numpy()
    diag = oracle.project(c.xyz, rows, h, 2)[3]
    x64 = c.xyz.astype(np.float64)
    D2 = ((x64[rows] - x64[:, None, :]) ** 2).sum(2).max(1)
    r9 = diag[:, 2] <= 2.0 ** -40 * D2
    assert r9.sum() > 10
    assert np.all(st.cpu().numpy()[r9] & 1)
