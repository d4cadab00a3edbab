"""One cloud split over ranks: contiguous ranges of a space-filling-curve order
plus one halo exchange.

The per-point projection (Algorithm 1) is independent from point to point,
so a cloud can be cut into contiguous ranges of a locality-preserving order
(the grid's Hilbert order on a GPU, a Morton order in the CPU tests), one per
rank (the paper's contiguous segments, Sec. 2.1).  A rank's queries need the
points of other ranks that lie within their k-th neighbour distance, so one
exchange step precedes the exact search:

  1. local kNN on the rank's own points: the k-th key of each point is an
     upper bound of its k-th key over the whole cloud;
  2. request boxes: each block of consecutive own points gives the box of the
     block grown by the square root of the block's largest local k-th key
     (every global neighbour of the block's points lies inside it);
  3. every rank gathers all boxes and sends each other rank its points that
     fall inside that rank's boxes (coordinates and global ids);
  4. the own and received points, ordered by global id so that ties rank as
     they would over the whole cloud, are searched again: the rows of the own
     points are then the global kNN rows, bit for bit, and the projection of
     the own points uses only points present on the rank.

The local computations come from an `ops` object (morton_order, knn,
project), so the same driver runs over libmls on a GPU (`GpuOps`) and, in
the CPU tests, over other implementations.  Communication uses
torch.distributed (NCCL between GPUs, gloo between CPU processes).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch
import torch.distributed as dist


def _world(group):
    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size(group), dist.get_rank(group)
    return 1, 0


def morton_partition(order: np.ndarray, world: int):
    """Contiguous ranges of a space-filling-curve order (any permutation is
    exact; locality only keeps the halo small), one per rank: index arrays."""
    n = order.shape[0]
    cuts = [(n * r) // world for r in range(world + 1)]
    return [np.asarray(order[cuts[r]:cuts[r + 1]]) for r in range(world)]


def request_boxes(xyz: np.ndarray, kth_key: np.ndarray, block: int = 256, margin: float = 1e-6) -> np.ndarray:
    """Boxes (m, 6: lo xyz, hi xyz) covering the k-th-neighbour balls of
    consecutive blocks of points, in FP64, grown by a relative margin for
    the float rounding of the keys."""
    n = xyz.shape[0]
    if n == 0:
        return np.zeros((0, 6))
    x = xyz.astype(np.float64)
    r = np.sqrt(kth_key.astype(np.float64))
    starts = np.arange(0, n, block)
    lo = np.minimum.reduceat(x, starts, axis=0)
    hi = np.maximum.reduceat(x, starts, axis=0)
    rad = np.maximum.reduceat(r, starts)
    span = np.abs(x).max() if n else 0.0
    grow = rad * (1.0 + margin) + margin * (span + 1e-30)
    return np.concatenate([lo - grow[:, None], hi + grow[:, None]], axis=1)


def in_boxes(xyz: np.ndarray, boxes: np.ndarray) -> np.ndarray:
    """Mask of the points inside any of the boxes."""
    if boxes.shape[0] == 0 or xyz.shape[0] == 0:
        return np.zeros(xyz.shape[0], bool)
    x = xyz.astype(np.float64)
    mask = np.zeros(x.shape[0], bool)
    for b in boxes:
        mask |= np.all((x >= b[:3]) & (x <= b[3:]), axis=1)
    return mask


def _exchange(send, group, device):
    """send[r]: 1-D float64 array for rank r.  Returns the arrays received
    from every rank (own entry passed through)."""
    world, rank = _world(group)
    sizes = torch.tensor([len(s) for s in send], dtype=torch.int64, device=device)
    all_sizes = [torch.zeros_like(sizes) for _ in range(world)]
    dist.all_gather(all_sizes, sizes, group=group)
    recv_sizes = [int(all_sizes[r][rank]) for r in range(world)]
    bufs = [torch.empty(recv_sizes[r], dtype=torch.float64, device=device) for r in range(world)]
    reqs = []
    for r in range(world):
        if r == rank:
            continue
        if len(send[r]):
            reqs.append(dist.isend(torch.as_tensor(send[r], dtype=torch.float64).to(device), r, group=group))
        if recv_sizes[r]:
            reqs.append(dist.irecv(bufs[r], r, group=group))
    for q in reqs:
        q.wait()
    bufs[rank] = torch.as_tensor(send[rank], dtype=torch.float64)
    return [b.cpu().numpy() for b in bufs]


@dataclass
class ShardResult:
    global_ids: np.ndarray    # own points' global ids
    rows: np.ndarray          # (n_own, k) global ids of the neighbours
    xyz: np.ndarray           # projected points
    normal: np.ndarray
    status: np.ndarray
    halo: int                 # points received


def sharded_project(own_xyz: np.ndarray, own_ids: np.ndarray, k: int, h: float, ops, degree: int = 2,
                    precision: str = "mixed", group=None, block: int = 256, device="cpu") -> ShardResult:
    """Exact kNN rows and projection of this rank's points (own_xyz, float32,
    with global ids own_ids, a contiguous range of the order) within a cloud spread
    over the ranks of `group`."""
    world, rank = _world(group)
    own_xyz = np.ascontiguousarray(own_xyz, np.float32)
    own_ids = np.asarray(own_ids, np.int64)
    halo_xyz = np.zeros((0, 3), np.float32)
    halo_ids = np.zeros(0, np.int64)
    if world > 1:
        # 1-2: local bound and request boxes (empty shards request nothing)
        if own_xyz.shape[0] >= k:
            _, key = ops.knn(own_xyz, k)
            boxes = request_boxes(own_xyz, key[:, k - 1], block)
        else:
            boxes = np.array([[-np.inf] * 3 + [np.inf] * 3])
        # 3: every rank's boxes, then the points each other rank asked for
        box_lists = _exchange([boxes.ravel()] * world, group, device)
        send = []
        for r in range(world):
            if r == rank:
                send.append(np.zeros(0))
                continue
            m = in_boxes(own_xyz, box_lists[r].reshape(-1, 6))
            send.append(np.concatenate([own_xyz[m].astype(np.float64).ravel(), own_ids[m].astype(np.float64)]))
        got = _exchange(send, group, device)
        for r in range(world):
            if r == rank or got[r].size == 0:
                continue
            cnt = got[r].size // 4
            halo_xyz = np.concatenate([halo_xyz, got[r][:3 * cnt].reshape(cnt, 3).astype(np.float32)])
            halo_ids = np.concatenate([halo_ids, got[r][3 * cnt:].astype(np.int64)])
    # 4: the own and received points in global-id order, searched and projected
    all_xyz = np.concatenate([own_xyz, halo_xyz])
    all_ids = np.concatenate([own_ids, halo_ids])
    perm = np.argsort(all_ids, kind="stable")
    sx, sid = all_xyz[perm], all_ids[perm]
    kk = min(k, sx.shape[0])
    rows_local, _ = ops.knn(sx, kk)
    out, nrm, st = ops.project(sx, rows_local, h, degree, precision)
    own_pos = np.searchsorted(sid, own_ids)
    return ShardResult(own_ids, sid[rows_local[own_pos]], out[own_pos], nrm[own_pos], st[own_pos],
                       int(halo_ids.shape[0]))


class GpuOps:
    """The local steps on the GPU, through libmls (numpy in and out)."""

    def __init__(self, device="cuda"):
        self.device = device

    def morton_order(self, xyz, k_hint=32):
        from . import capi
        x = torch.from_numpy(np.ascontiguousarray(xyz, np.float32)).to(self.device)
        grid = capi.mls_build_grid(x, 0.0, k_hint)
        try:
            order = capi.mls_grid_order(grid).cpu().numpy().copy()
        finally:
            torch.cuda.current_stream().synchronize()
            grid.close()
        return order

    def knn(self, xyz, k):
        from . import capi
        x = torch.from_numpy(np.ascontiguousarray(xyz, np.float32)).to(self.device)
        grid = capi.mls_build_grid(x, 0.0, k)
        try:
            idx, key = capi.mls_knn(grid, k, with_key=True)
            res = idx.cpu().numpy(), key.cpu().numpy()
        finally:
            torch.cuda.current_stream().synchronize()
            grid.close()
        return res

    def project(self, xyz, rows, h, degree, precision):
        from . import capi
        x = torch.from_numpy(np.ascontiguousarray(xyz, np.float32)).to(self.device)
        idx = torch.from_numpy(np.ascontiguousarray(rows, np.int32)).to(self.device)
        out, nrm, st = capi.mls_project(x, idx, h, degree, precision)
        return out.cpu().numpy(), nrm.cpu().numpy(), st.cpu().numpy()
