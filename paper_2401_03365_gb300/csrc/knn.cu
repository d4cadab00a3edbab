// The plain kNN launches (rows, keys, sorted positions) and the radius
// neighbourhoods, over the warp search of knn_search.cuh.
#include "knn_search.cuh"

namespace mls {

namespace {

// ---- radius neighbourhoods (Sec. 1.4: the points within radius R) --------
//
// One warp per query, runs of 32 consecutive queries in the grid order per
// warp (the cube of cells stays cached between them).  Every point with key
// <= R2 is kept, the same cube search and culling as the kNN with the fixed
// bound R2; ROWS = false counts them, ROWS = true ranks them by (key, index)
// into the query's CSR row.  More than kCap in a row is reported through
// *overflow (the largest count seen) and the row is left unwritten.

template <bool ROWS>
__global__ void __launch_bounds__(kChainThreads) k_radius(GridView g, float R2, int32_t *__restrict__ count,
                                                         const int64_t *__restrict__ offsets,
                                                         int32_t *__restrict__ rows, float *__restrict__ keys,
                                                         int *__restrict__ overflow) {
    __shared__ WarpBuf bufs[kChainWarps];
    const int lane = threadIdx.x & 31;
    WarpBuf &wb = bufs[threadIdx.x >> 5];
    const float eps2 = 2.0f * g.frame.eps;
    const float reach = sqrtf(R2) * kGrow * kGrow + eps2;
    int lev = g.base_level;
    while (lev < g.top_level && !(2.0f * g.side[lev] > reach)) ++lev;
    const float lim = (reach + eps2) * kGrow;
    const float lim2 = lim * lim;
    const Bins bins{0.f, R2 > 0.f ? 32.0f / R2 : 0.f};
    const int64_t n_warps = (int64_t)gridDim.x * kChainWarps;
    Cube cb;
    cb.st = wb.cube_start + lane;
    cb.ct = wb.cube_count + lane;
    for (int64_t run = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; run * 32 < g.n; run += n_warps) {
        const int64_t end = min((int64_t)g.n, run * 32 + 32);
        for (int64_t sp = run * 32; sp < end; ++sp) {
            const float4 q = __ldg(g.pts + sp);
            const uint64_t key0 = __ldg(g.keys + sp);
            const uint32_t c0[3] = {compact3(key0), compact3(key0 >> 1), compact3(key0 >> 2)};
            load_cube(g, lev, c0, cb, lane);
            // inlined here: the radius kernel has no other large body to share
            // the instruction cache with
            const int S = scan_keep_body<1>(cell_geom(g, cb), cb, wb, q, lim2, R2, bins, lane, false);
            const int64_t qi = (int64_t)__float_as_int(q.w);
            if (!ROWS) {
                if (lane == 0) count[qi] = S;
            } else if (S > kCap) {
                if (lane == 0) atomicMax(overflow, S);
            } else {
                rank_and_write(wb, S, bins, S, lane, 0, 0,
                               RowOut{rows + offsets[qi], keys ? keys + offsets[qi] : nullptr, nullptr});
            }
        }
    }
}

// ---- isolated queries ------------------------------------------------------
//
// A query alone in its cell one level above the base (a cell two base cells
// wide) is an outlier whose cube of base cells is nearly empty: its search
// climbs to coarse levels and scans many points.  Such queries are flagged in
// skip[] (every query's flag is written) and listed in the work-list layout (count at iso[1], next at
// iso[2], sorted positions from iso[8]) and, when `list` is given, in it too
// (count *count); their number is added to gwork[3], the grid's record of
// the queries searched outside the chain's runs.  Cells are sorted ranges,
// so a query is alone exactly when its sorted neighbours lie in other cells.

constexpr int kIsoThreads = 256;
constexpr int kIsoPer = 8;      // queries per thread

__global__ void __launch_bounds__(kIsoThreads) k_isolated(GridView g, int lev, uint8_t *__restrict__ skip,
                                                          int *__restrict__ iso, int32_t *__restrict__ list,
                                                          int32_t *__restrict__ count, int *__restrict__ gwork) {
    __shared__ int nblk, base_w, base_l;
    if (threadIdx.x == 0) nblk = 0;
    __syncthreads();
    const int64_t n = g.n;
    const int64_t s0 = (int64_t)blockIdx.x * kIsoThreads * kIsoPer + threadIdx.x;
    const int sh = 3 * lev;
    unsigned mask = 0u;
#pragma unroll
    for (int u = 0; u < kIsoPer; ++u) {
        const int64_t sp = s0 + (int64_t)u * kIsoThreads;
        if (sp < n) {
            const uint64_t c = __ldg(g.keys + sp) >> sh;
            const bool alone = (sp == 0 || (__ldg(g.keys + sp - 1) >> sh) != c) &&
                               (sp + 1 == n || (__ldg(g.keys + sp + 1) >> sh) != c);
            skip[sp] = alone ? 1 : 0;
            if (alone) mask |= 1u << u;
        }
    }
    int at = mask ? atomicAdd(&nblk, __popc(mask)) : 0;
    __syncthreads();
    if (threadIdx.x == 0 && nblk > 0) {
        base_w = atomicAdd(&iso[1], nblk);
        base_l = list ? atomicAdd(count, nblk) : 0;
        atomicAdd(&gwork[3], nblk);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kIsoPer; ++u)
        if ((mask >> u) & 1u) {
            const int32_t sp = (int32_t)(s0 + (int64_t)u * kIsoThreads);
            iso[8 + base_w + at] = sp;
            if (list) list[base_l + at] = sp;
            ++at;
        }
}

}  // namespace

// The kNN's two passes, for callers that put work between them: the chain
// pass (queries in sparse neighbourhoods listed in grid->work; with `skip`
// and `iso`, the flagged queries are taken first from the list iso, see
// k_knn_chain), then the sparse pass over grid->work's list (blocks_per_sm >
// 0: that many blocks per SM instead of a full wave, leaving room for other
// work beside it).  The chain pass takes its queries from a queue in
// grid->work, which `reset` starts afresh.
int launch_knn_chain_pass(const mls_grid *grid, int k, int32_t *idx, float *key, int32_t *pos, cudaStream_t st,
                          const uint8_t *skip, int *iso, int blocks_per_sm, bool reset) {
    const int64_t n = grid->n;
    const int sms = sm_count();
    auto chain = skip ? (k <= 32 ? k_knn_chain<1, PlainRows, true> : k_knn_chain<2, PlainRows, true>)
                      : (k <= 32 ? k_knn_chain<1, PlainRows> : k_knn_chain<2, PlainRows>);
    // all shared memory to the carveout, so that every block the registers
    // allow is resident; one resident wave of blocks, queries taken dynamically
    MLS_CUDA_TRY(cudaFuncSetAttribute(chain, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      cudaSharedmemCarveoutMaxShared));
    int per_sm = 1;
    MLS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chain, kChainThreads, 0));
    per_sm = blocks_per_sm > 0 ? blocks_per_sm : std::max(per_sm, 1);
    const int64_t runs = (n + kMinChunk - 1) / kMinChunk;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * per_sm,
                                                                    (runs + kChainWarps - 1) / kChainWarps));
    if (reset) MLS_CUDA_TRY(cudaMemsetAsync(grid->work, 0, 8 * sizeof(int), st));
    chain<<<blocks, kChainThreads, 0, st>>>(grid->view, k, grid->work, RowOut{idx, key, pos}, PlainRows{}, skip, iso);
    count_launches(1);
    MLS_CUDA_TRY(cudaGetLastError());
    return MLS_OK;
}

int launch_knn_sparse_pass(const mls_grid *grid, int k, int32_t *idx, float *key, int32_t *pos, cudaStream_t st,
                           int blocks_per_sm) {
    const int sms = sm_count();
    auto chain = k <= 32 ? k_knn_chain<1, PlainRows> : k_knn_chain<2, PlainRows>;
    auto sparse = k <= 32 ? k_knn_sparse<1, PlainRows> : k_knn_sparse<2, PlainRows>;
    MLS_CUDA_TRY(cudaFuncSetAttribute(sparse, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      cudaSharedmemCarveoutMaxShared));
    int per_sm = 1;
    MLS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chain, kChainThreads, 0));
    per_sm = blocks_per_sm > 0 ? blocks_per_sm : std::max(per_sm, 1);
    sparse<<<sms * per_sm, kChainThreads, 0, st>>>(grid->view, k, grid->work, RowOut{idx, key, pos}, PlainRows{});
    count_launches(1);
    MLS_CUDA_TRY(cudaGetLastError());
    return MLS_OK;
}

// Below this many points the kNN does not list its isolated queries: its
// second pass is then short, and the extra launch costs more than it hides.
constexpr int64_t kIsolateMinPoints = 1 << 18;

bool knn_isolates(const mls_grid *grid) { return grid->n >= kIsolateMinPoints; }

// The isolated queries (k_isolated) of the grid, for a chain pass launched
// after it without `reset`: clears the grid's work counters, then writes
// skip[] (n bytes) and lists them in iso (n + 8 ints) and, when given, in
// list (*count must start at zero).
int launch_knn_isolated(const mls_grid *grid, uint8_t *skip, int *iso, int32_t *list, int32_t *count,
                        cudaStream_t st) {
    const int64_t n = grid->n;
    const int lev = std::min(grid->view.base_level + 1, grid->view.top_level);
    const int64_t per_block = (int64_t)kIsoThreads * kIsoPer;
    MLS_CUDA_TRY(cudaMemsetAsync(grid->work, 0, 8 * sizeof(int), st));
    MLS_CUDA_TRY(cudaMemsetAsync(iso, 0, 8 * sizeof(int), st));
    k_isolated<<<(int)((n + per_block - 1) / per_block), kIsoThreads, 0, st>>>(grid->view, lev, skip, iso, list,
                                                                               count, grid->work);
    count_launches(1);
    MLS_CUDA_TRY(cudaGetLastError());
    return MLS_OK;
}

// From kIsolateMinPoints points, the isolated queries first (taken by every
// warp of the chain pass before its runs), then the chain pass over the
// rest, then the sparse pass over what the chain pass left.
int launch_knn(const mls_grid *grid, int k, int32_t *idx, float *key, int32_t *pos, cudaStream_t st) {
    const int64_t n = grid->n;
    ScratchSet scratch(st);
    uint8_t *skip = nullptr;
    int *iso = nullptr;
    int rc;
    if (knn_isolates(grid)) {
        MLS_CUDA_TRY(scratch.alloc(&skip, (size_t)n));
        MLS_CUDA_TRY(scratch.alloc(&iso, (size_t)(n + 8) * sizeof(int)));
        rc = launch_knn_isolated(grid, skip, iso, nullptr, nullptr, st);
        if (rc == MLS_OK) rc = launch_knn_chain_pass(grid, k, idx, key, pos, st, skip, iso, 0, false);
    } else {
        rc = launch_knn_chain_pass(grid, k, idx, key, pos, st, nullptr, nullptr, 0, true);
    }
    if (rc != MLS_OK) return rc;
    return launch_knn_sparse_pass(grid, k, idx, key, pos, st, 0);
}

}  // namespace mls

namespace mls {

int launch_radius(const mls_grid *grid, float R2, int32_t *count, const int64_t *offsets, int32_t *rows,
                  float *keys, int *overflow, cudaStream_t st) {
    const int sms = sm_count();
    const int64_t runs = (grid->n + 31) / 32;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 4, (runs + kChainWarps - 1) / kChainWarps));
    if (rows) {
        MLS_CUDA_TRY(cudaFuncSetAttribute(k_radius<true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          cudaSharedmemCarveoutMaxShared));
        k_radius<true><<<blocks, kChainThreads, 0, st>>>(grid->view, R2, count, offsets, rows, keys, overflow);
    } else {
        MLS_CUDA_TRY(cudaFuncSetAttribute(k_radius<false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          cudaSharedmemCarveoutMaxShared));
        k_radius<false><<<blocks, kChainThreads, 0, st>>>(grid->view, R2, count, offsets, rows, keys, overflow);
    }
    count_launches(1);
    MLS_CUDA_TRY(cudaGetLastError());
    return MLS_OK;
}

}  // namespace mls
