"""The sharding driver's GPU steps (GpuOps over libmls, device tensors): the
box test kernel against brute force, one rank, and three ranks emulated in
one process (boxes, selection, records and the local search, with the
exchange done by handing the records over: no collective).  Ranks on several
GPUs run only as CPU processes here (tests/test_shard_cpu.py)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2401_03365_gb300 import workloads
from tests.gpu_cases import compare_projection, diag_len

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2401_03365_gb300 import build, capi, shard
    build.build()
    return capi, shard


def test_points_in_boxes_matches_brute_force(mods):
    capi, _ = mods
    c = workloads.torus(n=50_000, seed=61, k=16)
    x = torch.from_numpy(c.xyz).cuda()
    rng = np.random.default_rng(62)
    ctr = c.xyz[rng.integers(0, c.n, 300)].astype(np.float64)
    half = np.exp(rng.uniform(np.log(1e-4), np.log(0.5), (300, 1))) * rng.uniform(0.2, 1.0, (300, 3))
    boxes = np.concatenate([ctr - half, ctr + half], 1).astype(np.float32)
    boxes[0] = [0.1, 0.1, 0.1, -0.1, 0.1, 0.1]               # empty (lo > hi)
    boxes[1] = [np.nan, 0, 0, 1, 1, 1]                        # NaN: selects nothing
    boxes[2] = np.concatenate([c.xyz[7], c.xyz[7]])           # a single point, closed box
    boxes[3] = [-10, -10, -10, 10, 10, 10]                    # larger than the cloud
    grid = capi.mls_build_grid(x, 0.0, 16)
    mask = capi.mls_points_in_boxes(grid, torch.from_numpy(boxes).cuda()).cpu().numpy().astype(bool)
    torch.cuda.synchronize()
    grid.close()
    p = c.xyz[:, None, :]
    with np.errstate(invalid="ignore"):
        ref = ((p >= boxes[None, :, :3]) & (p <= boxes[None, :, 3:])).all(-1).any(-1)
    assert np.array_equal(mask, ref)
    assert mask[7] and mask.all()                             # box 3 holds everything


def test_gpu_ops_single_rank(mods):
    _, shard = mods
    c = workloads.torus(n=60_000, seed=8, k=32)
    ops = shard.GpuOps()
    x = torch.from_numpy(c.xyz).cuda()
    order = ops.order(x, c.k)
    assert torch.equal(torch.sort(order).values, torch.arange(c.n, device="cuda"))
    rows_o, _ = oracle.knn_kdtree(c.xyz, c.k)
    h = float(np.float32(2.0 * oracle.mean_knn_dist(c.xyz, rows_o)))
    res = shard.sharded_project(x, torch.arange(c.n, device="cuda"), c.k, h, ops)
    assert np.array_equal(res.rows.cpu().numpy(), rows_o)
    o = oracle.project(c.xyz, rows_o, h, 2)
    compare_projection(res.xyz.cpu().numpy(), res.normal.cpu().numpy(), res.status.cpu().numpy(), *o,
                       diag_len(c.xyz), min_well_posed=0.3)


def test_three_emulated_ranks_equal_the_whole_cloud(mods):
    _, shard = mods
    c = workloads.torus(n=60_000, seed=63, k=32)
    ops = shard.GpuOps()
    x = torch.from_numpy(c.xyz).cuda()
    order = ops.order(x, c.k)
    parts = shard.morton_partition(order, 3)
    rows_o, _ = oracle.knn_kdtree(c.xyz, c.k)
    h = float(np.float32(2.0 * oracle.mean_knn_dist(c.xyz, rows_o)))
    own = [(x[p].contiguous(), p) for p in parts]
    boxes = []
    for xyz, _ in own:
        _, key = ops.knn(xyz, c.k)
        boxes.append(shard.request_boxes(xyz, key[:, c.k - 1], 256))
    seen = np.zeros(c.n, int)
    o = oracle.project(c.xyz, rows_o, h, 2)
    for r, (xyz, ids) in enumerate(own):
        recs = [shard.select_for(own[s][0], own[s][1], boxes[r], ops) for s in range(3) if s != r]
        halo_xyz, halo_ids = shard.unpack_records(recs, x.device)
        assert 0 < halo_ids.shape[0] < c.n
        res = shard.local_search(xyz, ids, halo_xyz, halo_ids, c.k, h, ops)
        gid = res.global_ids.cpu().numpy()
        seen[gid] += 1
        assert np.array_equal(res.rows.cpu().numpy(), rows_o[gid])
        compare_projection(res.xyz.cpu().numpy(), res.normal.cpu().numpy(), res.status.cpu().numpy(),
                           *(a[gid] for a in o), diag_len(c.xyz), min_well_posed=0.3)
    assert np.all(seen == 1)
