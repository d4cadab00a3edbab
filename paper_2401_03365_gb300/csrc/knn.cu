// Exact k nearest neighbours over the grid (the neighbour search of Sec. 2.2,
// read as kNN): one warp per query, queries taken in Morton order.
//
// For a query the warp first picks a level: the base level, or a coarser one
// when the 3x3x3 block of cells around the query holds fewer than k points.
// It then searches that block and, while needed, the next shells of cells
// (Chebyshev radius 2, 3, ...).  The search stops when the current k-th key is
// below a lower bound on the key of every point outside the searched block:
// the squared distance from the query to the block's faces (exact in double),
// shrunk by a relative 2^-20, which covers the rounding of the float key
// (at most about 5 units of 2^-24).  Ties are broken by the lower index, so
// the result is the unique first k of the order (key, index).
//
// The warp keeps the best 32*KPL candidates as a sorted list spread over the
// lanes (entry e = r * 32 + lane in register r), each a 64-bit word
// (key bits << 32 | index), which orders exactly as (key, index) because keys
// are non-negative floats.
#include "grid.cuh"

namespace mls {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kKnnThreads = 256;

// The ranking key: float differences, squares and sums, each rounded to
// nearest, association ((dx^2 + dy^2) + dz^2), never fused.
__device__ __forceinline__ float rank_key(float4 p, float qx, float qy, float qz) {
    float dx = __fsub_rn(p.x, qx);
    float dy = __fsub_rn(p.y, qy);
    float dz = __fsub_rn(p.z, qz);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

template <int KPL>
struct TopK {
    uint64_t e[KPL];
    uint64_t kth;

    __device__ void init() {
#pragma unroll
        for (int r = 0; r < KPL; ++r) e[r] = ~0ull;
        kth = ~0ull;
    }

    // Insert the candidates of the warp (one per lane, ~0 for none) that beat
    // the current k-th entry, one at a time.
    __device__ void offer(uint64_t cand, int k, int lane) {
        unsigned m = __ballot_sync(kFull, cand < kth);
        while (m) {
            int src = __ffs(m) - 1;
            uint64_t c = __shfl_sync(kFull, cand, src);
            int pos = 0;
#pragma unroll
            for (int r = 0; r < KPL; ++r) pos += __popc(__ballot_sync(kFull, e[r] < c));
            uint64_t up[KPL];
#pragma unroll
            for (int r = 0; r < KPL; ++r) up[r] = __shfl_up_sync(kFull, e[r], 1);
#pragma unroll
            for (int r = 1; r < KPL; ++r) {
                uint64_t carry = __shfl_sync(kFull, e[r - 1], 31);
                if (lane == 0) up[r] = carry;
            }
#pragma unroll
            for (int r = 0; r < KPL; ++r) {
                int idx = r * 32 + lane;
                e[r] = idx > pos ? up[r] : (idx == pos ? c : e[r]);
            }
            const int kr = (k - 1) >> 5, kl = (k - 1) & 31;
            uint64_t kv = e[0];
#pragma unroll
            for (int r = 1; r < KPL; ++r)
                if (r == kr) kv = e[r];
            kth = __shfl_sync(kFull, kv, kl);
            m &= ~(1u << src);
            m &= __ballot_sync(kFull, cand < kth);
        }
    }
};

// Range of the cell at level `lev` with integer coordinates c (any may be out
// of the grid): start and count, count 0 when empty or outside.
__device__ __forceinline__ void cell_range(const GridView &g, int lev, int cx, int cy, int cz, int &start,
                                           int &count) {
    start = 0;
    count = 0;
    const int dims = (int)(kAxisCells >> lev);
    if (cx < 0 || cy < 0 || cz < 0 || cx >= dims || cy >= dims || cz >= dims) return;
    const LevelTable &t = g.level[lev];
    int32_t id = lookup_cell(t, morton3((uint32_t)cx, (uint32_t)cy, (uint32_t)cz));
    if (id < 0) return;
    start = __ldg(t.cell_start + id);
    count = __ldg(t.cell_start + id + 1) - start;
}

// Scan the points of up to 32 cells (one per lane) and offer them to the list.
template <int KPL>
__device__ void scan_cells(const GridView &g, int start, int count, float qx, float qy, float qz, int k,
                           int lane, TopK<KPL> &top) {
    int incl = count;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    for (int base = 0; base < total; base += 32) {
        const int e = base + lane;
        int j = 0;    // number of cells whose inclusive count is <= e
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            int v = __shfl_sync(kFull, incl, j + step - 1);
            if (v <= e) j += step;
        }
        const int st_j = __shfl_sync(kFull, start, j & 31);
        const int in_j = __shfl_sync(kFull, incl, j & 31);
        const int ct_j = __shfl_sync(kFull, count, j & 31);
        uint64_t cand = ~0ull;
        if (e < total) {
            float4 p = __ldg(g.pts + st_j + (e - (in_j - ct_j)));
            float key = rank_key(p, qx, qy, qz);
            cand = ((uint64_t)__float_as_uint(key) << 32) | (uint32_t)__float_as_int(p.w);
        }
        top.offer(cand, k, lane);
    }
}

template <int KPL>
__global__ void __launch_bounds__(kKnnThreads) k_knn(GridView g, int k, int32_t *__restrict__ out_idx,
                                                     float *__restrict__ out_key) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (kKnnThreads / 32);
    for (int64_t sp = (blockIdx.x * (int64_t)kKnnThreads + threadIdx.x) >> 5; sp < g.n; sp += warps) {
        const float4 q = __ldg(g.pts + sp);
        const int32_t qi = __float_as_int(q.w);
        uint32_t c0[3];
        double frac[3];
        c0[0] = cell_coord(q.x, g.frame.origin[0], g.frame.inv_s0, &frac[0]);
        c0[1] = cell_coord(q.y, g.frame.origin[1], g.frame.inv_s0, &frac[1]);
        c0[2] = cell_coord(q.z, g.frame.origin[2], g.frame.inv_s0, &frac[2]);

        // level: coarsen while the 27 cells around the query hold fewer than k points
        int lev = g.base_level;
        int start = 0, count = 0;
        const int bx = lane % 3 - 1, by = (lane / 3) % 3 - 1, bz = lane / 9 - 1;
        for (;;) {
            start = count = 0;
            if (lane < 27)
                cell_range(g, lev, (int)(c0[0] >> lev) + bx, (int)(c0[1] >> lev) + by,
                           (int)(c0[2] >> lev) + bz, start, count);
            int tot = warp_sum(count);
            if (tot >= k || lev >= g.top_level) break;
            ++lev;
        }
        TopK<KPL> top;
        top.init();
        scan_cells<KPL>(g, start, count, q.x, q.y, q.z, k, lane, top);

        const int C[3] = {(int)(c0[0] >> lev), (int)(c0[1] >> lev), (int)(c0[2] >> lev)};
        const int dims = (int)(kAxisCells >> lev);
        const double S = ldexp(g.frame.s0, lev);
        double t[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) t[a] = ((double)(c0[a] & ((1u << lev) - 1u)) + frac[a]) / (double)(1u << lev);

        for (int L = 1;; ++L) {
            // lower bound on the distance to any point outside the block of radius L
            double dmin = INFINITY;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (C[a] - L > 0) dmin = fmin(dmin, (L + t[a]) * S);
                if (C[a] + L < dims - 1) dmin = fmin(dmin, (L + 1 - t[a]) * S);
            }
            if (dmin == INFINITY) break;                       // the whole grid is searched
            if (top.kth != ~0ull) {
                double kth_key = (double)__uint_as_float((uint32_t)(top.kth >> 32));
                if (kth_key < dmin * dmin * (1.0 - 0x1p-20)) break;
            }
            // shell of radius L + 1
            const int R = L + 1, m = 2 * R + 1, m3 = m * m * m;
            for (int base = 0; base < m3; base += 32) {
                const int li = base + lane;
                start = count = 0;
                if (li < m3) {
                    const int dx = li % m - R, dy = (li / m) % m - R, dz = li / (m * m) - R;
                    const int cheb = max(abs(dx), max(abs(dy), abs(dz)));
                    if (cheb == R) cell_range(g, lev, C[0] + dx, C[1] + dy, C[2] + dz, start, count);
                }
                if (__ballot_sync(kFull, count > 0))
                    scan_cells<KPL>(g, start, count, q.x, q.y, q.z, k, lane, top);
            }
        }
#pragma unroll
        for (int r = 0; r < KPL; ++r) {
            const int e = r * 32 + lane;
            if (e < k) {
                out_idx[(int64_t)qi * k + e] = (int32_t)(uint32_t)top.e[r];
                if (out_key) out_key[(int64_t)qi * k + e] = __uint_as_float((uint32_t)(top.e[r] >> 32));
            }
        }
    }
}

}  // namespace

int launch_knn(const mls_grid *grid, int k, int32_t *idx, float *key, cudaStream_t st) {
    int64_t n = grid->n;
    int64_t blocks = (n * 32 + kKnnThreads - 1) / kKnnThreads;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t cap = (int64_t)sms * 8 * 16;
    if (blocks > cap) blocks = cap;
    if (k <= 32)
        k_knn<1><<<(int)blocks, kKnnThreads, 0, st>>>(grid->view, k, idx, key);
    else
        k_knn<2><<<(int)blocks, kKnnThreads, 0, st>>>(grid->view, k, idx, key);
    count_launches(1);
    MLS_CUDA_TRY(cudaGetLastError());
    return MLS_OK;
}

}  // namespace mls
