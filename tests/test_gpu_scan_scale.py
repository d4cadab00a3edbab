"""The scan-scale workload: 50M points on the height field (density ramp 10x,
noise 0.002), k = 64, mixed.  The GPU searches and projects every point; the
oracle's k-d tree over the whole cloud gives the rows of a seeded 20,000-query
sample (bit-exact), and its projection of those queries the parity reference.
As configured, the noise exceeds the neighbourhood size in the sparse part of
the ramp, so many neighbourhoods are ill-posed: the comparison runs on the
well-posed mask, whose fraction is reported and bounded below."""
import numpy as np
import pytest
import torch

import oracle
from paper_2401_03365_gb300 import workloads
from tests.gpu_cases import compare_projection, diag_len

pytestmark = pytest.mark.gpu


def test_heightfield_50m_k64_sampled():
    from paper_2401_03365_gb300 import build, capi
    build.build()
    c = workloads.heightfield()
    x = torch.from_numpy(c.xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, c.k)
    idx, key = capi.mls_knn(grid, c.k, with_key=True)
    order = capi.mls_grid_order(grid)
    rng = np.random.default_rng(61)
    q = np.sort(rng.choice(c.n, 20_000, replace=False))
    qt = torch.from_numpy(q).cuda()
    rows_g = idx[qt].cpu().numpy()
    keys_g = key[qt].cpu().numpy()
    del key
    rows_o, keys_o = oracle.knn_kdtree(c.xyz, c.k, queries=q)
    assert np.array_equal(rows_g, rows_o)
    assert np.array_equal(keys_g.view(np.uint32), keys_o.view(np.uint32))
    xd = c.xyz.astype(np.float64)
    d = np.linalg.norm(xd[rows_o] - xd[q][:, None, :], axis=2)
    h = float(np.float32(2.0 * d[rows_o != q[:, None]].mean()))
    g_xyz, g_n, g_st = capi.mls_project(x, idx, h, 2, "mixed", order=order)
    torch.cuda.synchronize()
    grid.close()
    o = oracle.project(c.xyz, rows_o, h, 2, queries=q)
    rep = compare_projection(g_xyz[qt].cpu().numpy(), g_n[qt].cpu().numpy(), g_st[qt].cpu().numpy(), *o,
                             diag_len(c.xyz), min_well_posed=0.2)
    print("well-posed fraction", rep["well_posed"])
