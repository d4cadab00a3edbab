"""The differentiable workload: 1M points on a sphere with 64 Gaussian bumps,
k = 32, FP32 forward and backward of L = sum_i (|p'_i| - rho(p'_i / |p'_i|))^2,
the squared radial residual of each projected point to the analytic surface
(the distance to the surface has no closed form).  Gradients with respect to
the coordinates through project_differentiable (the adjoint kernel) are checked
against FP64 central differences of the oracle's projection on a seeded
2,000-point subset; dL/dh against FP64 differences over a 2,000-query subset."""
import numpy as np
import pytest
import torch

import oracle
from paper_2401_03365_gb300 import workloads

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
    xyz = c.xyz.copy()
    fd = np.empty(2000)
    for t, (j, a) in enumerate(zip(js, axes)):
        aff = np.unique(np.concatenate([by_target[off[j]:off[j + 1]] // k, [j]]))
        x0 = xyz[j, a]
        step = np.float32(1e-3 * h)
        xp, xm = np.float32(x0 + step), np.float32(x0 - step)
        vals = []
        for v in (xp, xm):
            xyz[j, a] = v
            o, _, _, _ = oracle.project(xyz, rows[aff], h, 2, queries=aff)
            vals.append(_loss_np(o, c).sum())
        xyz[j, a] = x0
        fd[t] = (vals[0] - vals[1]) / (float(xp) - float(xm))
    gj = g[js, axes]
    scale = np.abs(fd)
    ref = np.median(scale)
    bad = np.abs(gj - fd) > 2e-3 * scale + 2e-3 * ref
    assert bad.mean() <= 0.005, (np.sort(np.abs(gj - fd) / (scale + ref))[-8:], ref)


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
    assert abs(gh - fd) <= 2e-3 * abs(fd) + 1e-9, (gh, fd)
