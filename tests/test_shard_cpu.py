"""Sharding of one cloud over CPU ranks (gloo, 127.0.0.1): contiguous ranges
of a Morton order, one halo exchange of float4 records, then the local search
and projection.  With the FP64 oracle as every rank's local step, the ranks'
rows and projected points must equal the single-process oracle's, bit for
bit, also when a rank holds no points or fewer than k."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class OracleOps:
    """The oracle as the local step of every rank (test infrastructure), on
    CPU tensors."""

    def knn(self, xyz, k):
        import torch
        import oracle
        idx, key = oracle.knn_kdtree(xyz.numpy(), k)
        return torch.from_numpy(idx), torch.from_numpy(key)

    def in_boxes(self, xyz, boxes):
        import torch
        x = xyz.numpy().astype(np.float64)[:, None, :]
        b = boxes.numpy().astype(np.float64)[None]
        return torch.from_numpy(((x >= b[..., :3]) & (x <= b[..., 3:])).all(-1).any(-1))

    def project(self, xyz, rows, h, degree, precision):
        import torch
        import oracle
        out, nrm, st, _ = oracle.project(xyz.numpy(), rows.numpy(), h, degree)
        return torch.from_numpy(out), torch.from_numpy(nrm), torch.from_numpy(st)


def zorder(xyz, bits=10):
    """A Morton order of the points (quantised to 2^bits per axis)."""
    x = xyz.astype(np.float64)
    q = ((x - x.min(0)) / (np.ptp(x, 0).max() + 1e-30) * ((1 << bits) - 1)).astype(np.int64)
    key = np.zeros(x.shape[0], np.int64)
    for b in range(bits):
        for a in range(3):
            key |= ((q[:, a] >> b) & 1) << (3 * b + a)
    return np.argsort(key, kind="stable")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, xyz, k, h, out, cuts=None):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2401_03365_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        order = torch.from_numpy(zorder(xyz))
        if cuts is None:
            ids = shard.morton_partition(order, world)[rank]
        else:
            ids = order[cuts[rank]:cuts[rank + 1]]
        res = shard.sharded_project(torch.from_numpy(xyz)[ids], ids, k, h, OracleOps(), block=64)
        out[rank] = tuple(t.numpy() if hasattr(t, "numpy") else t
                          for t in (res.global_ids, res.rows, res.xyz, res.normal, res.status, res.halo))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _cloud():
    from paper_2401_03365_gb300 import workloads
    c = workloads.torus(n=5000, seed=7, k=16)
    import oracle
    rows, _ = oracle.knn_kdtree(c.xyz, c.k)
    h = float(np.float32(2.0 * oracle.mean_knn_dist(c.xyz, rows)))
    return c.xyz, c.k, h, rows


def _run(world, cuts=None):
    import oracle
    xyz, k, h, rows = _cloud()
    ref_xyz, ref_n, ref_st, _ = oracle.project(xyz, rows, h, 2)
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), xyz, k, h, out, cuts), nprocs=world, join=True)
        res = dict(out)
    seen = np.zeros(xyz.shape[0], int)
    for r in range(world):
        ids, r_rows, r_xyz, r_n, r_st, halo = res[r]
        seen[ids] += 1
        assert np.array_equal(r_rows, rows[ids])
        assert np.array_equal(r_xyz, ref_xyz[ids])
        assert np.array_equal(r_n, ref_n[ids])
        assert np.array_equal(r_st, ref_st[ids])
    assert np.all(seen == 1)
    return res, xyz.shape[0]


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_rows_and_projection_equal_the_whole_cloud(world):
    res, n = _run(world)
    for r in range(world):
        assert 0 < res[r][5] < n            # a halo, not the whole cloud


def test_a_rank_with_no_points_and_one_with_fewer_than_k():
    """Three ranks: the first holds nothing (it asks for nothing and returns
    empty results), the second 5 points (< k = 16: it asks for every point),
    the third the rest."""
    res, n = _run(3, cuts=[0, 0, 5, 5000])
    assert res[0][0].shape[0] == 0 and res[0][1].shape == (0, 16)
    assert res[1][5] == n - 5               # every other point was sent to it


def test_request_boxes_cover_every_neighbour():
    """Helper check on one process: each point's global neighbours lie in the
    box of its block."""
    sys.path.insert(0, ROOT)
    from paper_2401_03365_gb300 import shard
    import oracle
    xyz, k, h, rows = _cloud()
    import torch
    order = zorder(xyz)
    own = order[: xyz.shape[0] // 2]
    _, key = oracle.knn_kdtree(xyz[own], k)
    boxes = shard.request_boxes(torch.from_numpy(xyz[own]), torch.from_numpy(key[:, k - 1]), block=64)
    assert boxes.dtype == torch.float32
    for b in range(len(boxes)):
        blk = own[b * 64:(b + 1) * 64]
        nb = np.unique(rows[blk].ravel())
        assert OracleOps().in_boxes(torch.from_numpy(xyz[nb]), boxes[b:b + 1]).all()
