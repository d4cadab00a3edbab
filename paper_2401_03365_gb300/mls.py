"""User-facing MLS projection on the GPU (Sec. 1.4, Eq. 1; Algorithm 1).

    out = project(xyz, k=32)            # grid -> kNN -> h -> projection
    out.xyz, out.normal, out.status, out.idx, out.h

Every step runs in libmls; this module only sequences the C-ABI calls.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import capi


@dataclass
class Projection:
    xyz: torch.Tensor        # (n, 3) float32, projected points
    normal: torch.Tensor     # (n, 3) float32, plane normals (canonical sign)
    status: torch.Tensor     # (n,) uint8, capi.MLS_PT_* bits
    idx: torch.Tensor        # (n, k) int32 neighbour rows
    h: float                 # bandwidth used


class Pipeline:
    """Reusable buffers for repeated projections of clouds of one size:
    the grid handle, the neighbour rows (by original index, and by sorted
    position for the projection in the grid's order) and the outputs."""

    def __init__(self, n: int, k: int, device="cuda"):
        self.n, self.k = n, k
        self.grid = None
        self.idx = torch.empty((n, k), dtype=torch.int32, device=device)
        self.pos = torch.empty((n, k), dtype=torch.int32, device=device)
        self.out_xyz = torch.empty((n, 3), dtype=torch.float32, device=device)
        self.out_normal = torch.empty((n, 3), dtype=torch.float32, device=device)
        self.out_status = torch.empty(n, dtype=torch.uint8, device=device)

    def neighbours(self, xyz: torch.Tensor, cell_size: float = 0.0):
        self.grid = capi.mls_build_grid(xyz, cell_size, self.k, grid=self.grid)
        capi.mls_knn_sorted(self.grid, self.k, out_pos=self.pos, out_idx=self.idx)
        return self.idx

    def bandwidth(self, xyz: torch.Tensor) -> float:
        """h = 2 x mean distance to the other neighbours (a host read)."""
        return 2.0 * float(capi.mls_mean_knn_dist(xyz, self.idx).item())

    def project(self, xyz: torch.Tensor, h: float, degree: int = 2, precision: str = "mixed"):
        """The projection of the cloud the grid was built on: in the grid's
        order (mls_project_sorted) for FP32 and mixed, mls_project for FP64."""
        if precision == "fp64":
            capi.mls_project(xyz, self.idx, h, degree, precision, order=capi.mls_grid_order(self.grid),
                             out_xyz=self.out_xyz, out_normal=self.out_normal, out_status=self.out_status)
        else:
            capi.mls_project_sorted(self.grid, self.pos, h, degree, precision, out_xyz=self.out_xyz,
                                    out_normal=self.out_normal, out_status=self.out_status)
        return self.out_xyz, self.out_normal, self.out_status

    def close(self):
        if self.grid is not None:
            self.grid.close()
            self.grid = None


class ProjectFunction(torch.autograd.Function):
    """Differentiable MLS projection: forward mls_project, backward
    mls_project_backward (gradients for the coordinates and h; the neighbour
    rows are constants); with the grid the rows came from and its rows of
    sorted positions, mls_project_sorted and mls_project_backward_sorted (the
    same forward results, in the grid's order).  The plain form saves only
    xyz, the rows and h, and its backward recomputes every per-point frame;
    the grid-order form also saves the fit state (MLS_FIT_STATE_FLOATS floats
    per point), which its backward reads instead."""

    @staticmethod
    def forward(ctx, xyz, h, idx, degree, precision, order, grid=None, pos=None):
        hv = float(h)
        fit_state = None
        if grid is not None and pos is not None and precision != "fp64":
            out, nrm, st, fit_state = capi.mls_project_sorted(grid, pos, hv, degree, precision, with_state=True)
        else:
            out, nrm, st = capi.mls_project(xyz, idx, hv, degree, precision, order=order)
        ctx.save_for_backward(xyz, idx, order if order is not None else torch.empty(0, dtype=torch.int32))
        ctx.hv, ctx.degree, ctx.precision, ctx.has_order = hv, degree, precision, order is not None
        ctx.sorted = (grid, pos, fit_state) if fit_state is not None else None
        ctx.h_shape = h.shape if isinstance(h, torch.Tensor) else None
        ctx.mark_non_differentiable(st)
        return out, nrm, st

    @staticmethod
    def backward(ctx, g_out, g_n, g_st):
        xyz, idx, order = ctx.saved_tensors
        if g_out is None:
            g_out = torch.zeros_like(xyz)
        if ctx.sorted is not None:
            grid, pos, fit_state = ctx.sorted
            gx, gh = capi.mls_project_backward_sorted(grid, pos, ctx.hv, g_out.contiguous(),
                                                      None if g_n is None else g_n.contiguous(), ctx.degree,
                                                      ctx.precision, state=fit_state)
            ctx.sorted = None
        else:
            gx, gh = capi.mls_project_backward(xyz, idx, ctx.hv, g_out.contiguous(),
                                               None if g_n is None else g_n.contiguous(), ctx.degree, ctx.precision,
                                               order=order if ctx.has_order else None)
        gh_out = gh.reshape(ctx.h_shape).to(torch.float32) if ctx.h_shape is not None else None
        return gx, gh_out, None, None, None, None, None, None


def project_differentiable(xyz: torch.Tensor, idx: torch.Tensor, h, degree: int = 2, precision: str = "mixed",
                           order: torch.Tensor | None = None, grid=None, pos: torch.Tensor | None = None):
    """(xyz', normal, status) with autograd to xyz and h (a tensor).  With
    `grid` (built on xyz) and `pos` (its mls_knn_sorted rows) the forward
    runs in the grid's order."""
    if not isinstance(h, torch.Tensor):
        h = torch.tensor(float(h), dtype=torch.float32, device=xyz.device)
    return ProjectFunction.apply(xyz, h, idx, degree, precision, order, grid, pos)


def knn(xyz: torch.Tensor, k: int, with_key: bool = False, cell_size: float = 0.0):
    grid = capi.mls_build_grid(xyz, cell_size, k)
    try:
        idx, key = capi.mls_knn(grid, k, with_key=with_key)
        order = capi.mls_grid_order(grid).clone()
    finally:
        torch.cuda.current_stream().synchronize()
        grid.close()
    return idx, key, order


def project(xyz: torch.Tensor, k: int = 32, h: float | None = None, degree: int = 2,
            precision: str = "mixed") -> Projection:
    p = Pipeline(xyz.shape[0], k, xyz.device)
    try:
        p.neighbours(xyz)
        if h is None:
            h = p.bandwidth(xyz)
        p.project(xyz, h, degree, precision)
        torch.cuda.current_stream().synchronize()
    finally:
        p.close()
    return Projection(p.out_xyz, p.out_normal, p.out_status, p.idx, h)


@dataclass
class RadiusProjection:
    xyz: torch.Tensor        # (m, 3) projected points that are kept (outliers dropped)
    normal: torch.Tensor     # (m, 3)
    kept: torch.Tensor       # (m,) int32 indices of the kept input points
    status: torch.Tensor     # (n,) uint8 status of every input point (bit 16: outlier)
    offsets: torch.Tensor    # (n + 1,) int64 CSR offsets of the radius neighbourhoods
    rows: torch.Tensor       # int32 neighbour indices
    h: float


def project_radius(xyz: torch.Tensor, R: float, h: float | None = None, degree: int = 2,
                   precision: str = "mixed", min_neighbors: int = 3) -> RadiusProjection:
    """The paper's neighbourhood definition (Sec. 1.4: the points within radius
    R) with its outlier rule (Sec. 3.3: fewer than 3 neighbours -> removed):
    radius rows on the GPU, the projection over them, the compaction.
    h defaults to R (the Gaussian's width equal to the search radius)."""
    grid = capi.mls_build_grid(xyz, 0.0, 16)
    try:
        offsets, rows, _ = capi.mls_radius_neighbors(grid, R)
        order = capi.mls_grid_order(grid)
        hh = float(R if h is None else h)
        out, nrm, st = capi.mls_project_rows(xyz, offsets, rows, hh, degree, precision, min_neighbors, order=order)
        kept = capi.mls_compact(st, capi.MLS_PT_OUTLIER)
        torch.cuda.current_stream().synchronize()
    finally:
        grid.close()
    k = kept.long()
    return RadiusProjection(out[k], nrm[k], kept, st, offsets, rows, hh)
