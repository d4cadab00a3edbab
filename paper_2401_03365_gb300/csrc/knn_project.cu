// The neighbour search and the projection in one pass (Algorithm 1: the
// neighbourhood of each point, then its plane, polynomial and projection),
// without the round trip of the rows through memory.
//
// The kNN's warps (knn_search.cuh) keep, besides the optional row output, the
// rows of their last 32 finished queries in a per-warp buffer of 32 x k
// sorted positions (entry j of buffer slot b at j * 32 + b: lane b reads its
// row with coalesced loads).  When 32 have been collected, and when the warp
// runs out of queries, lane b projects the query in slot b with project_point
// (one lane per point, as the projection kernel), over the grid's sorted
// points.  Queries deferred to the sparse pass are collected and projected
// there the same way.  The buffers (4 k KB per warp) stay in L2; the rows
// are written to memory only when the caller asks for them.
//
// The mixed form defers its FP64 points (0.3 % of the points of a scan) as
// the projection kernel does: their sorted positions and rows go to a list,
// finished by a third, compact pass, so that no warp runs FP64 arithmetic
// with one lane active.  A point that finds the list full is finished in
// place.  Results are those of mls_knn_sorted followed by
// mls_project_sorted: the same rows, the same points, the same per-point
// arithmetic.
#include "knn_search.cuh"
#include "project_point.cuh"

namespace mls {

namespace {

// Rows of the warp's current batch plus the sorted position of each query
// in it (the query of slot b on lane b).
struct BatchRows : RowOut {
    int32_t *bat;
    int slot;

    __device__ __forceinline__ void put(int32_t qi, int64_t sp, int k, int rank, int32_t i, float key_,
                                        int32_t p) const {
        RowOut::put(qi, sp, k, rank, i, key_, p);
        bat[rank * 32 + slot] = p;
    }
};

// The points of the mixed form that need an FP64 step: sorted position and
// row of each (capacity cap; *count may pass cap, the excess finished in
// place).
struct Deferred {
    int32_t *sp;
    int32_t *rows;      // cap x k
    int32_t *count;
    int cap;
};

__device__ __forceinline__ void write_result(float *out_xyz, float *out_n, uint8_t *status, int64_t i,
                                             const float o[3], const float nf[3], uint8_t st) {
    out_xyz[3 * i] = o[0];
    out_xyz[3 * i + 1] = o[1];
    out_xyz[3 * i + 2] = o[2];
    if (out_n) {
        out_n[3 * i] = nf[0];
        out_n[3 * i + 1] = nf[1];
        out_n[3 * i + 2] = nf[2];
    }
    if (status) status[i] = st;
}

// Projects the `count` queries of a batch, lane b the query at sorted
// position `mine` with the row in slot b of `bat`.  Out of line: one body
// per kernel, called once per 32 queries.
template <int DEG, int PREC>
__device__ __noinline__ void project_batch(const float4 *pts, const int32_t *bat, int k, float h, float *out_xyz,
                                           float *out_n, uint8_t *status, Deferred def, int count, int32_t mine,
                                           int lane) {
    if (lane >= count) return;
    const float4 r4 = __ldg(pts + mine);
    const auto row = [&](int j) { return bat[j * 32 + lane]; };
    float o[3], nf[3];
    uint8_t st;
    if (PREC == MLS_PREC_MIXED) {
        st = project_point<DEG, MLS_PREC_MIXED, false, true>(pts, row, k, 0, 1, h, r4.x, r4.y, r4.z, o, nf);
        if (st == kDeferFP64) {
            const int d = atomicAdd(def.count, 1);
            if (d < def.cap) {
                def.sp[d] = mine;
                for (int j = 0; j < k; ++j) def.rows[(int64_t)d * k + j] = row(j);
                return;
            }
            st = project_point<DEG, MLS_PREC_MIXED>(pts, row, k, 0, 1, h, r4.x, r4.y, r4.z, o, nf);
        }
    } else {
        st = project_point<DEG, PREC>(pts, row, k, 0, 1, h, r4.x, r4.y, r4.z, o, nf);
    }
    write_result(out_xyz, out_n, status, __float_as_int(r4.w), o, nf, st);
}

// The deferred points, one thread each, with their FP64 steps.
template <int DEG>
__global__ void __launch_bounds__(128) k_fused_deferred(const float4 *__restrict__ pts, int k, float h, Deferred def,
                                                        float *__restrict__ out_xyz, float *__restrict__ out_n,
                                                        uint8_t *__restrict__ status) {
    const int count = min(*def.count, def.cap);
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < count; d += gridDim.x * blockDim.x) {
        const float4 r4 = __ldg(pts + def.sp[d]);
        const int32_t *row = def.rows + (int64_t)d * k;
        float o[3], nf[3];
        const uint8_t st = project_point<DEG, MLS_PREC_MIXED>(
            pts, [&](int j) { return __ldg(row + j); }, k, 0, 1, h, r4.x, r4.y, r4.z, o, nf);
        write_result(out_xyz, out_n, status, __float_as_int(r4.w), o, nf, st);
    }
}

template <int DEG, int PREC>
struct ProjectBatch {
    // Four blocks per SM: the projection needs 64 registers (the kNN alone
    // runs at five blocks of 48).
    static constexpr int kBlocksPerSm = 5;

    const float4 *pts;      // the grid's sorted points (w = original index bits)
    int32_t *bat_all;       // every warp's buffer, 32 k entries each
    int k;
    float h;
    float *out_xyz, *out_n;
    uint8_t *status;
    Deferred def;           // the mixed form's FP64 points
    int32_t *bat = nullptr; // this warp's buffer
    int count = 0;          // queries collected (warp-uniform)
    int32_t mine = 0;       // lane b: sorted position of the query in slot b

    __device__ __forceinline__ void start(int64_t warp, int) { bat = bat_all + warp * 32 * (int64_t)k; }

    __device__ __forceinline__ BatchRows rows(const RowOut &out) const { return BatchRows{out, bat, count}; }

    __device__ __forceinline__ void done(int64_t sp, int lane) {
        if (lane == count) mine = (int32_t)sp;
        if (++count == 32) finish(lane);
    }

    __device__ __forceinline__ void finish(int lane) {
        if (count == 0) return;
        __syncwarp();       // the rows written by the other lanes are visible
        project_batch<DEG, PREC>(pts, bat, k, h, out_xyz, out_n, status, def, count, mine, lane);
        count = 0;
        __syncwarp();       // every lane has read the buffer before it is refilled
    }
};

template <int DEG, int PREC>
int launch_fused(const mls_grid *grid, int k, float h, float *out_xyz, float *out_n, uint8_t *status, int32_t *pos,
                 cudaStream_t st) {
    const int64_t n = grid->n;
    const int sms = sm_count();
    using Fin = ProjectBatch<DEG, PREC>;
    auto chain = k_knn_chain<1, Fin>;
    auto sparse = k_knn_sparse<1, Fin>;
    MLS_CUDA_TRY(cudaFuncSetAttribute(chain, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      cudaSharedmemCarveoutMaxShared));
    MLS_CUDA_TRY(cudaFuncSetAttribute(sparse, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      cudaSharedmemCarveoutMaxShared));
    int chain_per_sm = 1, sparse_per_sm = 1;
    MLS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&chain_per_sm, chain, kChainThreads, 0));
    MLS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sparse_per_sm, sparse, kChainThreads, 0));
    chain_per_sm = std::max(chain_per_sm, 1);
    sparse_per_sm = std::max(sparse_per_sm, 1);
    const int64_t runs = (n + kMinChunk - 1) / kMinChunk;
    const int chain_blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)sms * chain_per_sm, (runs + kChainWarps - 1) / kChainWarps));
    const int sparse_blocks = sms * sparse_per_sm;
    // one buffer per warp of the larger launch (the sparse pass reuses them
    // after the chain pass, in stream order)
    const int64_t warps = (int64_t)std::max(chain_blocks, sparse_blocks) * kChainWarps;
    ScratchSet scratch(st);
    int32_t *bat = nullptr;
    MLS_CUDA_TRY(scratch.alloc(&bat, (size_t)warps * 32 * k * sizeof(int32_t)));
    // the FP64 list: room for 1/32 of the points (about ten times what a
    // scan needs); more are finished in place
    Deferred def{nullptr, nullptr, nullptr, 0};
    if (PREC == MLS_PREC_MIXED) {
        def.cap = (int)std::min<int64_t>(n, std::max<int64_t>(1024, n / 32));
        MLS_CUDA_TRY(scratch.alloc(&def.sp, (size_t)(def.cap + 1) * sizeof(int32_t)));
        MLS_CUDA_TRY(scratch.alloc(&def.rows, (size_t)def.cap * k * sizeof(int32_t)));
        def.count = def.sp + def.cap;
        MLS_CUDA_TRY(cudaMemsetAsync(def.count, 0, sizeof(int32_t), st));
    }
    MLS_CUDA_TRY(cudaMemsetAsync(grid->work, 0, 8 * sizeof(int), st));
    const RowOut out{nullptr, nullptr, pos};
    const Fin fin{grid->view.pts, bat, k, h, out_xyz, out_n, status, def};
    chain<<<chain_blocks, kChainThreads, 0, st>>>(grid->view, k, grid->work, out, fin, nullptr, nullptr);
    sparse<<<sparse_blocks, kChainThreads, 0, st>>>(grid->view, k, grid->work, out, fin);
    count_launches(2);
    if (PREC == MLS_PREC_MIXED) {
        k_fused_deferred<DEG><<<sms * 2, 128, 0, st>>>(grid->view.pts, k, h, def, out_xyz, out_n, status);
        count_launches(1);
    }
    MLS_CUDA_TRY(cudaGetLastError());
    return MLS_OK;
}

template <int PREC>
int launch_fused_deg(const mls_grid *grid, int k, float h, int degree, float *out_xyz, float *out_n,
                     uint8_t *status, int32_t *pos, cudaStream_t st) {
    switch (degree) {
        case 0:
            return launch_fused<0, PREC>(grid, k, h, out_xyz, out_n, status, pos, st);
        case 1:
            return launch_fused<1, PREC>(grid, k, h, out_xyz, out_n, status, pos, st);
        default:
            return launch_fused<2, PREC>(grid, k, h, out_xyz, out_n, status, pos, st);
    }
}

}  // namespace

int launch_knn_project(const mls_grid *grid, int k, float h, int degree, int precision, float *out_xyz,
                       float *out_n, uint8_t *status, int32_t *pos, cudaStream_t st) {
    if (precision == MLS_PREC_FP32)
        return launch_fused_deg<MLS_PREC_FP32>(grid, k, h, degree, out_xyz, out_n, status, pos, st);
    return launch_fused_deg<MLS_PREC_MIXED>(grid, k, h, degree, out_xyz, out_n, status, pos, st);
}

}  // namespace mls
