"""One cloud split over ranks: contiguous ranges of a space-filling-curve order
plus one halo exchange, with the data in each rank's device memory.

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
     (every global neighbour of the block's points lies inside it), rounded
     outwards to float;
  3. every rank gathers all boxes and sends each other rank its points that
     fall inside that rank's boxes, as float4 records (x, y, z and the global
     id's bits), device to device;
  4. the own and received points, ordered by global id so that ties rank as
     they would over the whole cloud, are searched again: the rows of the own
     points are then the global kNN rows, bit for bit, and the projection of
     the own points uses only points present on the rank.

The local computations come from an `ops` object (knn, in_boxes, project,
all on torch tensors of the ops' device), so the same driver runs over libmls
on a GPU (`GpuOps`: the box test is the mls_points_in_boxes kernel over the
rank's grid) and, in the CPU tests, over other implementations.
Communication uses torch.distributed on the same tensors (NCCL between GPUs,
gloo between CPU processes).  Global ids must be below 2^31.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch
import torch.distributed as dist


def _world(group):
    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size(group), dist.get_rank(group)
    return 1, 0


def morton_partition(order: torch.Tensor, world: int):
    """Contiguous ranges of a space-filling-curve order (any permutation is
    exact; locality only keeps the halo small), one per rank."""
    n = order.shape[0]
    cuts = [(n * r) // world for r in range(world + 1)]
    return [order[cuts[r]:cuts[r + 1]] for r in range(world)]


def request_boxes(xyz: torch.Tensor, kth_key: torch.Tensor, block: int = 256, margin: float = 1e-6) -> torch.Tensor:
    """Boxes (m, 6 float32: lo xyz, hi xyz) covering the k-th-neighbour balls
    of consecutive blocks of points: computed in FP64, grown by a relative
    margin for the float rounding of the keys, then rounded outwards."""
    n = xyz.shape[0]
    if n == 0:
        return torch.zeros((0, 6), dtype=torch.float32, device=xyz.device)
    x = xyz.to(torch.float64)
    r = kth_key.to(torch.float64).sqrt()
    m = (n + block - 1) // block
    pad = m * block - n
    if pad:                     # repeat the last point: it changes no block's extent
        x = torch.cat([x, x[-1:].expand(pad, 3)])
        r = torch.cat([r, r[-1:].expand(pad)])
    xb = x.view(m, block, 3)
    lo = xb.min(dim=1).values
    hi = xb.max(dim=1).values
    rad = r.view(m, block).max(dim=1).values
    span = float(x.abs().max())
    grow = (rad * (1.0 + margin) + margin * (span + 1e-30))[:, None]
    lo, hi = lo - grow, hi + grow
    lo32, hi32 = lo.to(torch.float32), hi.to(torch.float32)
    lo32 = torch.where(lo32.to(torch.float64) > lo, torch.nextafter(lo32, torch.full_like(lo32, -float("inf"))), lo32)
    hi32 = torch.where(hi32.to(torch.float64) < hi, torch.nextafter(hi32, torch.full_like(hi32, float("inf"))), hi32)
    return torch.cat([lo32, hi32], dim=1)


def _everything(boxes: torch.Tensor) -> bool:
    """True when a box is unbounded (a rank with fewer than k points asks for
    every point)."""
    return bool(torch.isinf(boxes).any()) if boxes.numel() else False


def _exchange(send, group):
    """send[r]: (m_r, c) float32 tensor for rank r (own entry ignored).
    Returns the tensors received from every rank (own entry empty), on the
    same device."""
    world, rank = _world(group)
    dev = send[0].device
    width = send[0].shape[1]
    sizes = torch.tensor([s.shape[0] for s in send], dtype=torch.int64, device=dev)
    all_sizes = [torch.zeros_like(sizes) for _ in range(world)]
    dist.all_gather(all_sizes, sizes, group=group)
    recv = [torch.empty((int(all_sizes[r][rank]) if r != rank else 0, width), dtype=torch.float32, device=dev)
            for r in range(world)]
    ops = []
    for r in range(world):
        if r == rank:
            continue
        if send[r].shape[0]:
            ops.append(dist.P2POp(dist.isend, send[r].contiguous(), r, group=group))
        if recv[r].shape[0]:
            ops.append(dist.P2POp(dist.irecv, recv[r], r, group=group))
    if ops:
        for q in dist.batch_isend_irecv(ops):
            q.wait()
    return recv


def _all_boxes(boxes: torch.Tensor, group):
    """Every rank's boxes (list indexed by rank)."""
    world, rank = _world(group)
    dev = boxes.device
    n = torch.tensor([boxes.shape[0]], dtype=torch.int64, device=dev)
    counts = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(counts, n, group=group)
    mx = max(int(c) for c in counts)
    padded = torch.full((mx, 6), float("nan"), dtype=torch.float32, device=dev)
    padded[:boxes.shape[0]] = boxes
    got = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(got, padded, group=group)
    return [got[r][:int(counts[r])] for r in range(world)]


@dataclass
class ShardResult:
    global_ids: torch.Tensor    # own points' global ids (int64)
    rows: torch.Tensor          # (n_own, k) global ids of the neighbours (int64)
    xyz: torch.Tensor           # projected points
    normal: torch.Tensor
    status: torch.Tensor
    halo: int                   # points received


def sharded_project(own_xyz: torch.Tensor, own_ids: torch.Tensor, k: int, h: float, ops, degree: int = 2,
                    precision: str = "mixed", group=None, block: int = 256) -> ShardResult:
    """Exact kNN rows and projection of this rank's points (own_xyz float32
    (n, 3), global ids own_ids, a contiguous range of the order, on the ops'
    device) within a cloud spread over the ranks of `group`."""
    world, rank = _world(group)
    own_xyz = own_xyz.to(torch.float32).contiguous()
    own_ids = own_ids.to(torch.int64)
    dev = own_xyz.device
    halo_xyz = torch.zeros((0, 3), dtype=torch.float32, device=dev)
    halo_ids = torch.zeros(0, dtype=torch.int64, device=dev)
    if world > 1:
        # 1-2: local bound and request boxes (a shard with fewer than k
        # points asks for everything, an empty one for nothing)
        if own_xyz.shape[0] >= k:
            _, key = ops.knn(own_xyz, k)
            boxes = request_boxes(own_xyz, key[:, k - 1], block)
        elif own_xyz.shape[0] > 0:
            boxes = torch.tensor([[-float("inf")] * 3 + [float("inf")] * 3], dtype=torch.float32, device=dev)
        else:
            boxes = torch.zeros((0, 6), dtype=torch.float32, device=dev)
        # 3: every rank's boxes, then the points each other rank asked for
        box_lists = _all_boxes(boxes, group)
        send = [select_for(own_xyz, own_ids, box_lists[r], ops) if r != rank else own_xyz.new_zeros((0, 4))
                for r in range(world)]
        got = _exchange(send, group)
        halo_xyz, halo_ids = unpack_records([got[r] for r in range(world) if r != rank], dev)
    return local_search(own_xyz, own_ids, halo_xyz, halo_ids, k, h, ops, degree, precision)


def select_for(own_xyz: torch.Tensor, own_ids: torch.Tensor, boxes: torch.Tensor, ops) -> torch.Tensor:
    """The own points inside another rank's boxes as float4 records (x, y, z,
    the global id's int32 bits), ready to send."""
    if own_xyz.shape[0] == 0 or boxes.shape[0] == 0:
        return own_xyz.new_zeros((0, 4))
    m = torch.ones(own_xyz.shape[0], dtype=torch.bool, device=own_xyz.device) if _everything(boxes) \
        else ops.in_boxes(own_xyz, boxes)
    records = torch.cat([own_xyz, own_ids.to(torch.int32).view(torch.float32)[:, None]], dim=1)
    return records[m]


def unpack_records(parts, device):
    """Received float4 records -> (xyz (m, 3) float32, global ids (m,) int64)."""
    parts = [p for p in parts if p.shape[0]]
    if not parts:
        return (torch.zeros((0, 3), dtype=torch.float32, device=device),
                torch.zeros(0, dtype=torch.int64, device=device))
    rec = torch.cat(parts)
    return rec[:, :3].contiguous(), rec[:, 3].contiguous().view(torch.int32).to(torch.int64)


def local_search(own_xyz, own_ids, halo_xyz, halo_ids, k, h, ops, degree=2, precision="mixed") -> ShardResult:
    """Step 4: the own and received points in global-id order, searched and
    projected; the rows and results of the own points."""
    dev = own_xyz.device
    if own_xyz.shape[0] == 0:
        e = own_xyz[:0]
        return ShardResult(own_ids, torch.zeros((0, k), dtype=torch.int64, device=dev), e, e,
                           torch.zeros(0, dtype=torch.uint8, device=dev), int(halo_ids.shape[0]))
    all_xyz = torch.cat([own_xyz, halo_xyz])
    all_ids = torch.cat([own_ids, halo_ids])
    sid, perm = torch.sort(all_ids, stable=True)
    sx = all_xyz[perm].contiguous()
    kk = min(k, sx.shape[0])
    rows_local, _ = ops.knn(sx, kk)
    out, nrm, st = ops.project(sx, rows_local, h, degree, precision)
    own_pos = torch.searchsorted(sid, own_ids)
    return ShardResult(own_ids, sid[rows_local[own_pos].long()], out[own_pos], nrm[own_pos], st[own_pos],
                       int(halo_ids.shape[0]))


class GpuOps:
    """The local steps on the GPU, through libmls, on CUDA tensors."""

    def __init__(self, device="cuda"):
        self.device = device

    def order(self, xyz: torch.Tensor, k_hint: int = 32) -> torch.Tensor:
        """The grid's (Hilbert) order of the points (int64 indices)."""
        from . import capi
        grid = capi.mls_build_grid(xyz.contiguous(), 0.0, k_hint)
        try:
            return capi.mls_grid_order(grid).to(torch.int64)
        finally:
            torch.cuda.current_stream().synchronize()
            grid.close()

    def knn(self, xyz: torch.Tensor, k: int):
        from . import capi
        grid = capi.mls_build_grid(xyz.contiguous(), 0.0, k)
        try:
            return capi.mls_knn(grid, k, with_key=True)
        finally:
            torch.cuda.current_stream().synchronize()
            grid.close()

    def in_boxes(self, xyz: torch.Tensor, boxes: torch.Tensor) -> torch.Tensor:
        from . import capi
        grid = capi.mls_build_grid(xyz.contiguous(), 0.0, 16)
        try:
            return capi.mls_points_in_boxes(grid, boxes.contiguous()).bool()
        finally:
            torch.cuda.current_stream().synchronize()
            grid.close()

    def project(self, xyz: torch.Tensor, rows: torch.Tensor, h: float, degree: int, precision: str):
        from . import capi
        return capi.mls_project(xyz.contiguous(), rows.to(torch.int32).contiguous(), h, degree, precision)
