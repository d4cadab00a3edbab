"""The differentiable workload: 1M points on a sphere with 64 Gaussian bumps,
k = 32, FP32 forward and backward of L = sum_i (|p'_i| - rho(p'_i / |p'_i|))^2,
the squared radial residual of each projected point to the analytic surface
(the distance to the surface has no closed form).  Gradients with respect to
the coordinates through project_differentiable (the adjoint kernel) are checked
against FP64 central differences of the oracle's projection on a seeded
2,000-point subset; dL/dh against FP64 differences over a 2,000-query subset.
A coordinate is checked when every projected point whose row holds it is
well-posed (the projection's mask), against the bound 1e-3 of the norm of the
oracle's gradient at that point; the rest are counted and reported."""
import numpy as np
import pytest
import torch

import oracle
from paper_2401_03365_gb300 import workloads
from tests.gpu_cases import GRAD_TOL, well_posed

pytestmark = pytest.mark.gpu


def _loss_torch(p, c):
    r = p.norm(dim=1)
    u = p / r[:, None]
    centres = torch.as_tensor(c.meta["centres"], dtype=p.dtype, device=p.device)
    amps = torch.as_tensor(c.meta["amps"], dtype=p.dtype, device=p.device)
    widths = torch.as_tensor(c.meta["widths"], dtype=p.dtype, device=p.device)
    rho = 1.0 + (amps[None, :] * torch.exp(-(1.0 - u @ centres.T) / widths[None, :] ** 2)).sum(1)
    return (r - rho) ** 2


def _loss_np(p, c):
    r = np.linalg.norm(p, axis=1)
    rho = workloads.bumpy_radius(p / r[:, None], c.meta["centres"], c.meta["amps"], c.meta["widths"])
    return (r - rho) ** 2


@pytest.fixture(scope="module")
def c5():
    from paper_2401_03365_gb300 import build, capi, mls
    build.build()
    c = workloads.bumpy_sphere()
    x = torch.from_numpy(c.xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, c.k)
    idx, _ = capi.mls_knn(grid, c.k)
    order = capi.mls_grid_order(grid).clone()
    h = float(np.float32(2.0 * float(capi.mls_mean_knn_dist(x, idx).item())))
    torch.cuda.synchronize()
    grid.close()
    return c, x, idx, order, h, mls, capi


def test_coordinate_gradient_against_fp64_differences(c5):
    c, x, idx, order, h, mls, _ = c5
    xg = x.clone().requires_grad_(True)
    ht = torch.tensor(h, device="cuda", requires_grad=True)
    out, _, _ = mls.project_differentiable(xg, idx, ht, 2, "fp32", order=order)
    _loss_torch(out, c).sum().backward()
    g = xg.grad.cpu().numpy().astype(np.float64)
    rows = idx.cpu().numpy()
    k = rows.shape[1]
    # reverse adjacency: the queries whose rows hold each point
    by_target = np.argsort(rows.ravel(), kind="stable")
    off = np.concatenate([[0], np.cumsum(np.bincount(rows.ravel(), minlength=c.n))])
    rng = np.random.default_rng(51)
    js = rng.choice(c.n, 2000, replace=False)
    axes = rng.integers(0, 3, 2000)
    affs = [np.unique(np.concatenate([by_target[off[j]:off[j + 1]] // k, [j]])) for j in js]
    every = np.unique(np.concatenate(affs))
    # the rows used are the oracle's own
    rows_o, _ = oracle.knn_kdtree(c.xyz, k, queries=every)
    assert np.array_equal(rows_o, rows[every])
    # the oracle's projection of those queries: its well-posed mask, and the
    # loss cotangent at its outputs for its own adjoint (the scale of each
    # point's gradient)
    o_xyz, _, _, diag = oracle.project(c.xyz, rows_o, h, 2, queries=every)
    good = np.zeros(c.n, bool)
    good[every] = well_posed(diag)
    po = torch.from_numpy(o_xyz).requires_grad_(True)
    _loss_torch(po, c).sum().backward()
    gp = np.zeros((c.n, 3))
    gp[every] = po.grad.numpy()
    g_o, _ = oracle.project_grad(c.xyz, rows_o, h, 2, gp, queries=every)
    xyz = c.xyz.copy()
    # Richardson-extrapolated central differences: steps 2^-19 and 2^-20
    # (about 1e-4 h), exact and symmetric in float32 for |x| < 1.99, so the
    # O(s^2) terms cancel between the two (the eigenvector's curvature grows
    # like 1/gap^2, and a single step of 1e-3 h was 2 % off at gap 1e-3)
    assert np.abs(xyz[js, axes]).max() < 1.99

    def central(j, a, aff, s):
        x0 = xyz[j, a]
        vals = []
        for v in (np.float32(x0 + s), np.float32(x0 - s)):
            xyz[j, a] = v
            o, _, _, _ = oracle.project(xyz, rows[aff], h, 2, queries=aff)
            vals.append(_loss_np(o, c).sum())
        xyz[j, a] = x0
        return (vals[0] - vals[1]) / (2 * s)

    fd = np.empty(2000)
    for t, (j, a, aff) in enumerate(zip(js, axes, affs)):
        fd[t] = (4 * central(j, a, aff, 2.0 ** -20) - central(j, a, aff, 2.0 ** -19)) / 3
    clean = np.array([good[aff].all() for aff in affs])
    scale = np.linalg.norm(g_o[js], axis=1)
    # the FP64 differences agree with the oracle's adjoint (its own pin, here
    # on this workload) far inside the bound
    assert np.all(np.abs(fd - g_o[js, axes])[clean] <= 1e-2 * GRAD_TOL * scale[clean])
    err = np.abs(g[js, axes] - fd)
    rep = {"clean": float(clean.mean()), "excluded": int((~clean).sum()),
           "max_rel_err": float((err / scale)[clean].max()),
           "excluded_max_rel_err": float((err / scale)[~clean].max()) if (~clean).any() else 0.0}
    print(rep)
    assert clean.mean() >= 0.99, rep
    assert np.all(err[clean] <= GRAD_TOL * scale[clean]), rep


def test_bandwidth_gradient_against_fp64_differences(c5):
    c, x, idx, order, h, mls, _ = c5
    rng = np.random.default_rng(52)
    S = np.sort(rng.choice(c.n, 2000, replace=False))
    mask = torch.zeros(c.n, device="cuda")
    mask[torch.from_numpy(S).cuda()] = 1.0
    ht = torch.tensor(h, device="cuda", requires_grad=True)
    out, _, _ = mls.project_differentiable(x, idx, ht, 2, "fp32", order=order)
    (_loss_torch(out, c) * mask).sum().backward()
    gh = float(ht.grad.item())
    rows = idx.cpu().numpy()[S]
    dh = 1e-4 * h
    vals = [_loss_np(oracle.project(c.xyz, rows, h + s, 2, queries=S)[0], c).sum() for s in (dh, -dh)]
    fd = (vals[0] - vals[1]) / (2 * dh)
    assert abs(gh - fd) <= GRAD_TOL * abs(fd), (gh, fd)
