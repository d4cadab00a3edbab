"""mls_project_levin (weights about q, Sec. 1.4, Eq. 1) against the oracle's
fixed-point form, element by element on the well-posed mask taken from that
operator's own diagnostics (eigen-gap of its last plane, condition of its
final fit).  Only the points the oracle leaves unconverged are left out, and
on every other well-posed point the GPU must have converged too."""
import numpy as np
import pytest
import torch

import oracle
from paper_2401_03365_gb300 import workloads
from tests.gpu_cases import compare_projection, diag_len, well_posed

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    from paper_2401_03365_gb300 import build, capi
    build.build()
    return capi


def _case(c, k):
    rows, _ = oracle.knn_kdtree(c.xyz, k)
    h = float(np.float32(2.0 * oracle.mean_knn_dist(c.xyz, rows)))
    return rows, h


@pytest.mark.parametrize("precision", ["mixed", "fp32"])
@pytest.mark.parametrize("degree", [0, 1, 2])
def test_sphere(capi, precision, degree):
    c = workloads.sphere()
    rows, h = _case(c, c.k)
    o_xyz, o_n, o_st, o_it, diag = oracle.project_levin(c.xyz, rows, h, degree, with_diag=True)
    assert np.all((o_st & oracle.STATUS_NOT_CONVERGED) == 0)
    x = torch.from_numpy(c.xyz).cuda()
    idx = torch.from_numpy(rows.astype(np.int32)).cuda()
    g_xyz, g_n, g_st = capi.mls_project_levin(x, idx, h, degree, precision, max_iter=32, tol=1e-6)
    g_st = g_st.cpu().numpy()
    assert np.all((g_st & capi.MLS_PT_NOT_CONVERGED)[well_posed(diag)] == 0)
    compare_projection(g_xyz.cpu().numpy(), g_n.cpu().numpy(), g_st, o_xyz, o_n, o_st & 3, diag, diag_len(c.xyz))


def test_torus_with_outliers_in_morton_order(capi):
    c = workloads.torus(n=100_000, seed=12)
    rows, h = _case(c, c.k)
    o_xyz, o_n, o_st, _, diag = oracle.project_levin(c.xyz, rows, h, 2, with_diag=True)
    x = torch.from_numpy(c.xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, c.k)
    idx, _ = capi.mls_knn(grid, c.k)
    assert np.array_equal(idx.cpu().numpy(), rows)
    order = capi.mls_grid_order(grid)
    g = capi.mls_project_levin(x, idx, h, 2, "mixed", max_iter=64, tol=1e-6, order=order)
    torch.cuda.synchronize()
    grid.close()
    g_conv = (g[2].cpu().numpy() & capi.MLS_PT_NOT_CONVERGED) == 0
    # only the points the oracle leaves unconverged are left out (a slowly
    # contracting iteration is still moving there); the GPU must have
    # converged wherever the oracle did on a well-posed point
    ok = (o_st & oracle.STATUS_NOT_CONVERGED) == 0
    assert np.all(g_conv[ok & well_posed(diag)])
    rep = compare_projection(*(t.cpu().numpy()[ok] for t in g), o_xyz[ok], o_n[ok], o_st[ok] & 3, diag[ok],
                             diag_len(c.xyz), min_well_posed=0.3)
    print("oracle unconverged:", int((~ok).sum()), rep)


def test_paraboloid_axis_fixed_point(capi):
    """The oracle pin's configuration: degree 0 lands on the weighted-height
    fixed point on the axis."""
    alpha, z0, n_side, spacing, h = 0.8, 0.05, 15, 0.05, 0.12
    g = (np.arange(n_side) - n_side // 2) * spacing
    X, Y = np.meshgrid(g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), alpha * (X.ravel() ** 2 + Y.ravel() ** 2)], 1)
    pts = np.concatenate([pts, [[0.0, 0.0, z0]]]).astype(np.float32)
    m = pts.shape[0] - 1
    rows = np.tile(np.arange(m, dtype=np.int32), (m + 1, 1))[:, :64]     # 64 nearest are not needed here:
    rows[m] = np.argsort(np.linalg.norm(pts[:m] - pts[m], axis=1), kind="stable")[:64]
    o, _, o_st, _ = oracle.project_levin(pts, rows[m:], h, 0, queries=[m])
    x = torch.from_numpy(pts).cuda()
    idx = torch.from_numpy(rows).cuda()
    g_xyz, _, g_st = capi.mls_project_levin(x, idx, h, 0, "mixed", max_iter=64, tol=1e-7)
    assert o_st[0] == 0 and int(g_st[m].item()) & 3 == 0
    assert np.abs(g_xyz[m].cpu().numpy() - o[0]).max() < 1e-6


def test_argument_errors(capi):
    x = torch.zeros((100, 3), device="cuda")
    idx = torch.zeros((100, 8), dtype=torch.int32, device="cuda")
    for kw, code in [({"max_iter": 0}, -1), ({"max_iter": 65}, -1), ({"tol": 0.0}, -1), ({"precision": "fp64"}, -1)]:
        with pytest.raises(capi.MLSError) as e:
            capi.mls_project_levin(x, idx, 0.1, 2, **kw)
        assert e.value.code == code
