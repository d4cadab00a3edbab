// Box membership for the halo exchange of one cloud split over ranks (the
// paper's contiguous segments, Sec. 2.1, with an exact exchange in place of
// its ring of borders): which of a rank's points lie inside the boxes
// another rank asks for.
//
// One warp per box, over the grid built on the rank's points: at the finest
// level with a table on which the box (grown by the frame's rounding bound
// eps) spans at most kBoxSpan cells per axis, the warp looks up the box's
// cells in the level's hash table and tests the points of the occupied ones
// against the box itself.  A point filed under a cell lies at most eps
// outside it, so every point inside the box is in one of the cells visited.
#include <algorithm>
#include <cmath>

#include "grid.cuh"

namespace mls {

namespace {

constexpr int kBoxSpan = 4;        // cells per axis at the chosen level
constexpr int kBoxThreads = 256;

__global__ void __launch_bounds__(kBoxThreads) k_points_in_boxes(GridView g, const float *__restrict__ boxes,
                                                                 int64_t m, uint8_t *__restrict__ mask) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (kBoxThreads / 32);
    for (int64_t b = (blockIdx.x * (int64_t)kBoxThreads + threadIdx.x) >> 5; b < m; b += warps) {
        float lo[3], hi[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = __ldg(boxes + 6 * b + a);
            hi[a] = __ldg(boxes + 6 * b + 3 + a);
        }
        if (!(lo[0] <= hi[0] && lo[1] <= hi[1] && lo[2] <= hi[2])) continue;   // empty (or NaN) box
        // level-0 cell range of the box grown by eps (clamped to the grid)
        uint32_t c0[3], c1[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            c0[a] = cell_coord(fmaxf(lo[a] - g.frame.eps, -3.0e38f), g.frame.origin[a], g.frame.inv_s0);
            c1[a] = cell_coord(fminf(hi[a] + g.frame.eps, 3.0e38f), g.frame.origin[a], g.frame.inv_s0);
        }
        int L = g.base_level;
        while (L < g.top_level && ((c1[0] >> L) - (c0[0] >> L) >= kBoxSpan || (c1[1] >> L) - (c0[1] >> L) >= kBoxSpan ||
                                   (c1[2] >> L) - (c0[2] >> L) >= kBoxSpan))
            ++L;
        const int nx = (int)((c1[0] >> L) - (c0[0] >> L)) + 1, ny = (int)((c1[1] >> L) - (c0[1] >> L)) + 1,
                  nz = (int)((c1[2] >> L) - (c0[2] >> L)) + 1;
        const int ncell = nx * ny * nz;     // at most kBoxSpan^3 = 64 (or the top level's single cell)
        const LevelTable &t = g.level[L];
        for (int c = 0; c < ncell; ++c) {
            const uint32_t x = (c0[0] >> L) + (uint32_t)(c % nx), y = (c0[1] >> L) + (uint32_t)((c / nx) % ny),
                           z = (c0[2] >> L) + (uint32_t)(c / (nx * ny));
            int32_t id = -1;
            if (lane == 0) id = lookup_cell(t, morton3(x, y, z));
            id = __shfl_sync(0xffffffffu, id, 0);
            if (id < 0) continue;
            const int32_t s = __ldg(t.cell_start + id), e = __ldg(t.cell_start + id + 1);
            for (int32_t p = s + lane; p < e; p += 32) {
                const float4 q = __ldg(g.pts + p);
                if (q.x >= lo[0] && q.x <= hi[0] && q.y >= lo[1] && q.y <= hi[1] && q.z >= lo[2] && q.z <= hi[2])
                    mask[__float_as_int(q.w)] = 1;
            }
        }
    }
}

}  // namespace

int launch_points_in_boxes(const mls_grid *grid, const float *boxes, int64_t m, uint8_t *mask, cudaStream_t st) {
    if (m < 1) return MLS_OK;
    const int64_t need = (m + kBoxThreads / 32 - 1) / (kBoxThreads / 32);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sm_count() * 8));
    k_points_in_boxes<<<blocks, kBoxThreads, 0, st>>>(grid->view, boxes, m, mask);
    count_launches(1);
    MLS_CUDA_TRY(cudaGetLastError());
    return MLS_OK;
}

}  // namespace mls
