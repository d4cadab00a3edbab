"""Sharding of one cloud over CPU ranks (gloo, 127.0.0.1): contiguous ranges
of a Morton order, one halo exchange, then the local search and projection.
With the FP64 oracle as every rank's local step, the ranks' rows and
projected points must equal the single-process oracle's, bit for bit."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class OracleOps:
    """The oracle as the local step of every rank (test infrastructure)."""

    def knn(self, xyz, k):
        import oracle
        return oracle.knn_kdtree(xyz, k)

    def project(self, xyz, rows, h, degree, precision):
        import oracle
        out, nrm, st, _ = oracle.project(xyz, rows, h, degree)
        return out, nrm, st


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


def _rank_main(rank, world, port, xyz, k, h, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2401_03365_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        parts = shard.morton_partition(zorder(xyz), world)
        ids = parts[rank]
        res = shard.sharded_project(xyz[ids], ids, k, h, OracleOps(), block=64)
        out[rank] = (res.global_ids, res.rows, res.xyz, res.normal, res.status, res.halo)
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


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_rows_and_projection_equal_the_whole_cloud(world):
    import oracle
    xyz, k, h, rows = _cloud()
    ref_xyz, ref_n, ref_st, _ = oracle.project(xyz, rows, h, 2)
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), xyz, k, h, out), nprocs=world, join=True)
        res = dict(out)
    seen = np.zeros(xyz.shape[0], int)
    for r in range(world):
        ids, r_rows, r_xyz, r_n, r_st, halo = res[r]
        seen[ids] += 1
        assert np.array_equal(r_rows, rows[ids])
        assert np.array_equal(r_xyz, ref_xyz[ids])
        assert np.array_equal(r_n, ref_n[ids])
        assert np.array_equal(r_st, ref_st[ids])
        assert 0 < halo < xyz.shape[0]          # a halo, not the whole cloud
    assert np.all(seen == 1)


def test_request_boxes_cover_every_neighbour():
    """Helper check on one process: each point's global neighbours lie in the
    box of its block."""
    sys.path.insert(0, ROOT)
    from paper_2401_03365_gb300 import shard
    import oracle
    xyz, k, h, rows = _cloud()
    order = zorder(xyz)
    own = order[: xyz.shape[0] // 2]
    _, key = oracle.knn_kdtree(xyz[own], k)
    boxes = shard.request_boxes(xyz[own], key[:, k - 1], block=64)
    for b in range(len(boxes)):
        blk = own[b * 64:(b + 1) * 64]
        nb = np.unique(rows[blk].ravel())
        assert shard.in_boxes(xyz[nb], boxes[b:b + 1]).all()
