// Grid build (the spatial index of Sec. 2.2, with a space-filling-curve order
// as the paper suggests for unordered clouds): bounding box, level-0 cell
// keys, an LSD radix sort of (key, point index), the sorted float4 points with
// their Morton cell keys, and one hash table of occupied cells per level from
// the base level up.  The sort key is the cell's index along the Hilbert
// curve: like the Morton key it lists every cell of every level as one run of
// consecutive positions (its top 3 l bits name the level-l cell), and
// consecutive cells along it are always face neighbours, so consecutive
// points are closer than in Morton order (the kNN bounds each query from the
// one before it).  The hash tables and the search keep Morton keys.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "grid.cuh"
#include "hilbert.cuh"

namespace mls {

namespace {

struct Misc {
    int bbox[6];                           // ordered ints: min xyz, max xyz
    int nonfinite;
    int pad;
    unsigned long long level_hist[kMaxLevels];
    GridFrame frame;
    uint64_t *cell_key[kMaxLevels];        // device copies of the per-level key arrays
};

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;   // 2048 keys per block
constexpr int kDigitBits = 8;
constexpr int kDigits = 1 << kDigitBits;
constexpr int kKeyBits = 3 * kMortonBits;              // 63

__global__ void k_init_misc(Misc *m) {
    int t = threadIdx.x;
    if (t < 3) {
        m->bbox[t] = 0x7fffffff;                        // +max ordered
        m->bbox[3 + t] = (int)0x80000000;               // -max ordered
    }
    if (t == 0) m->nonfinite = 0;
    if (t < kMaxLevels) m->level_hist[t] = 0;
}

__global__ void k_bbox(const float *__restrict__ xyz, int64_t n, Misc *m) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    int bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float v = xyz[3 * i + a];
            if (!isfinite(v)) bad = 1;
            lo[a] = fminf(lo[a], v);
            hi[a] = fmaxf(hi[a], v);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    }
    bad = __any_sync(0xffffffffu, bad);
    // the block's warps meet in shared memory: one set of global atomics per block
    __shared__ int sb[7];
    if (threadIdx.x < 3) {
        sb[threadIdx.x] = 0x7fffffff;
        sb[3 + threadIdx.x] = (int)0x80000000;
    }
    if (threadIdx.x == 0) sb[6] = 0;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        for (int a = 0; a < 3; ++a) {
            atomicMin(&sb[a], float_to_ordered(lo[a]));
            atomicMax(&sb[3 + a], float_to_ordered(hi[a]));
        }
        if (bad) sb[6] = 1;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        atomicMin(&m->bbox[threadIdx.x], sb[threadIdx.x]);
        atomicMax(&m->bbox[3 + threadIdx.x], sb[3 + threadIdx.x]);
    }
    if (threadIdx.x == 0 && sb[6]) atomicOr(&m->nonfinite, 1);
}

// The level-0 frame: cell side s0 = a power of two with 2^21 cells spanning
// the largest extent plus one cell, origin = bbox min rounded down to a
// multiple of s0 (exact in float), eps from the largest coordinate magnitude.
__global__ void k_frame(Misc *m) {
    if (threadIdx.x != 0 || m->nonfinite) return;
    float lo[3], hi[3], ext = 0.0f;
    for (int a = 0; a < 3; ++a) {
        lo[a] = ordered_to_float(m->bbox[a]);
        hi[a] = ordered_to_float(m->bbox[3 + a]);
        ext = fmaxf(ext, hi[a] - lo[a]);
    }
    // s0 >= ext / (2^21 - 2) (rounded up to a power of two) keeps every
    // point inside the 2^21 cells per axis; 2^-100 floors degenerate extents
    float need = ext / (float)(kAxisCells - 2) * (1.0f + 0x1p-20f);
    int e;
    frexpf(fmaxf(need, 0x1p-100f), &e);
    GridFrame f;
    f.s0 = ldexpf(1.0f, e);
    f.inv_s0 = ldexpf(1.0f, -e);
    float mag = 0.0f;
    for (int a = 0; a < 3; ++a) {
        f.origin[a] = floorf(lo[a] * f.inv_s0) * f.s0;
        mag = fmaxf(mag, fmaxf(fabsf(f.origin[a]), fabsf(f.origin[a] + f.s0 * (float)kAxisCells)));
    }
    int em;
    frexpf(fmaxf(mag, 0x1p-100f), &em);     // mag < 2^em
    f.eps = ldexpf(8.0f, em - 24);           // 8 ulp of values below 2^em
    m->frame = f;
}

// Sort keys: the Hilbert index of each point's level-0 cell, or, for a build
// whose radix passes read only the key bits from 3 `level` up, the index of
// its level-`level` cell on the coarser curve shifted into place: the same
// bits there (the bits below are zero and not read), so the same order.
__global__ void k_keys(const float *__restrict__ xyz, int64_t n, const Misc *__restrict__ m, int level,
                       uint64_t *__restrict__ keys, int32_t *__restrict__ perm) {
    GridFrame f = m->frame;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t c[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) c[a] = cell_coord(xyz[3 * i + a], f.origin[a], f.inv_s0) >> level;
        keys[i] = hilbert3(c[0], c[1], c[2], kMortonBits - level) << (3 * level);
        perm[i] = (int32_t)i;
    }
}

// ---- LSD radix sort of (key, value), 8-bit digits, stable ----------------

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint64_t *__restrict__ keys,
                                                              int64_t n, int shift, int nblocks,
                                                              int32_t *__restrict__ block_hist) {
    __shared__ int hist[kDigits];
    for (int d = threadIdx.x; d < kDigits; d += blockDim.x) hist[d] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        int64_t i = base + it * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&hist[(keys[i] >> shift) & (kDigits - 1)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kDigits; d += blockDim.x)
        block_hist[(int64_t)d * nblocks + blockIdx.x] = hist[d];
}

// One block per digit: exclusive scan over the blocks' counts of that digit;
// the digit's total goes to totals[d].
__global__ void __launch_bounds__(1024) k_radix_scan(int32_t *__restrict__ block_hist, int nblocks,
                                                     int32_t *__restrict__ totals) {
    __shared__ int warp_sums[32];
    __shared__ int carry;
    int32_t *row = block_hist + (int64_t)blockIdx.x * nblocks;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < nblocks; base += 1024) {
        int i = base + threadIdx.x;
        int v = i < nblocks ? row[i] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int s = warp_sums[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            warp_sums[lane] = s;
        }
        __syncthreads();
        int excl = carry + (warp ? warp_sums[warp - 1] : 0) + x - v;
        if (i < nblocks) row[i] = excl;
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_sums[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

// Scatter of one digit pass.  Each warp ranks its 256 keys per digit (stable:
// item order, then lane); the block's keys are then reordered by digit in
// shared memory, so that consecutive threads write consecutive positions of
// one digit's run (coalesced stores instead of one segment per lane).
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const uint64_t *__restrict__ keys_in, const int32_t *__restrict__ vals_in, int64_t n, int shift,
    int nblocks, const int32_t *__restrict__ block_off, const int32_t *__restrict__ totals,
    uint64_t *__restrict__ keys_out, int32_t *__restrict__ vals_out) {
    constexpr int kWarps = kSortThreads / 32;
    __shared__ int wcount[kWarps][kDigits];
    __shared__ int digit_base[kDigits];     // global start of each digit's run
    __shared__ int local_start[kDigits];    // start of each digit's run within the block
    __shared__ uint64_t tile_k[kSortTile];
    __shared__ int32_t tile_v[kSortTile];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kDigits * kWarps; d += blockDim.x) (&wcount[0][0])[d] = 0;
    // exclusive scan of the digit totals (256 entries) by warp 0
    if (warp == 0) {
        int carry = 0;
        for (int c = 0; c < kDigits; c += 32) {
            int v = totals[c + lane], x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            digit_base[c + lane] = carry + x - v;
            carry += __shfl_sync(0xffffffffu, x, 31);
        }
    }
    __syncthreads();
    uint64_t k[kSortItems];
    int32_t v[kSortItems];
    int rank[kSortItems];
    const int64_t bbase = (int64_t)blockIdx.x * kSortTile;
    const int64_t wbase = bbase + (int64_t)warp * 32 * kSortItems;
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        int64_t i = wbase + it * 32 + lane;
        bool ok = i < n;
        k[it] = ok ? keys_in[i] : ~0ull;
        v[it] = ok ? vals_in[i] : 0;
        int d = ok ? (int)((k[it] >> shift) & (kDigits - 1)) : -1;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int before = __popc(peers & lanemask_lt());
        int leader = __ffs(peers) - 1;
        int prev = ok ? wcount[warp][d] : 0;
        rank[it] = prev + before;
        __syncwarp();
        if (ok && lane == leader) wcount[warp][d] = prev + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive scan of its count over the warps, and its total
    for (int d = threadIdx.x; d < kDigits; d += blockDim.x) {
        int s = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            int c = wcount[w][d];
            wcount[w][d] = s;
            s += c;
        }
        local_start[d] = s;
    }
    __syncthreads();
    // exclusive scan of the block's digit totals (warp 0)
    if (warp == 0) {
        int carry = 0;
        for (int c = 0; c < kDigits; c += 32) {
            int v0 = local_start[c + lane], x = v0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            local_start[c + lane] = carry + x - v0;
            carry += __shfl_sync(0xffffffffu, x, 31);
        }
    }
    __syncthreads();
    // the block's keys in digit order
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        int64_t i = wbase + it * 32 + lane;
        if (i >= n) continue;
        int d = (int)((k[it] >> shift) & (kDigits - 1));
        int at = local_start[d] + wcount[warp][d] + rank[it];
        tile_k[at] = k[it];
        tile_v[at] = v[it];
    }
    __syncthreads();
    const int count = (int)min((int64_t)kSortTile, n - bbase);
    for (int t = threadIdx.x; t < count; t += kSortThreads) {
        const uint64_t key = tile_k[t];
        const int d = (int)((key >> shift) & (kDigits - 1));
        const int64_t pos = (int64_t)digit_base[d] + block_off[(int64_t)d * nblocks + blockIdx.x] + (t - local_start[d]);
        keys_out[pos] = key;
        vals_out[pos] = tile_v[t];
    }
}

__global__ void k_gather_pts(const float *__restrict__ xyz, const int32_t *__restrict__ perm,
                             int64_t n, const Misc *__restrict__ m, float4 *__restrict__ pts,
                             uint64_t *__restrict__ mkeys) {
    GridFrame f = m->frame;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        int32_t i = perm[s];
        const float p[3] = {xyz[3 * (int64_t)i], xyz[3 * (int64_t)i + 1], xyz[3 * (int64_t)i + 2]};
        pts[s] = make_float4(p[0], p[1], p[2], __int_as_float(i));
        mkeys[s] = morton3(cell_coord(p[0], f.origin[0], f.inv_s0), cell_coord(p[1], f.origin[1], f.inv_s0),
                           cell_coord(p[2], f.origin[2], f.inv_s0));
    }
}

// Level of the highest key bit in which sorted neighbours s-1 and s differ:
// they share a cell at every level above it.
__device__ inline int split_level(const uint64_t *keys, int64_t s) {
    if (s == 0) return kMaxLevels;     // the first point opens a cell at every level
    uint64_t d = keys[s] ^ keys[s - 1];
    if (d == 0) return -1;
    return (63 - __clzll((long long)d)) / 3;
}

__global__ void k_level_hist(const uint64_t *__restrict__ keys, int64_t n, Misc *m) {
    __shared__ unsigned long long hist[kMaxLevels];
    if (threadIdx.x < kMaxLevels) hist[threadIdx.x] = 0;
    __syncthreads();
    // one shared atomic per distinct level among a warp's points
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); s0 < n; s0 += stride) {
        const int64_t s = s0 + (threadIdx.x & 31) + 1;
        const int l = s < n ? split_level(keys, s) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, l);
        if (l >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[l], (unsigned long long)__popc(peers));
    }
    __syncthreads();
    if (threadIdx.x < kMaxLevels && hist[threadIdx.x]) atomicAdd(&m->level_hist[threadIdx.x], hist[threadIdx.x]);
}

// ---- cell tables for levels base..top --------------------------------------

constexpr int kHeadThreads = 256;

// Per block and level: how many sorted points open a cell at that level.
__global__ void __launch_bounds__(kHeadThreads) k_head_count(const uint64_t *__restrict__ keys,
                                                              int64_t n, int base, int top,
                                                              int nblocks, int32_t *__restrict__ counts) {
    __shared__ int c[kMaxLevels];
    if (threadIdx.x < kMaxLevels) c[threadIdx.x] = 0;
    __syncthreads();
    int64_t s = (int64_t)blockIdx.x * kHeadThreads + threadIdx.x;
    int l = s < n ? split_level(keys, s) : -1;
    for (int lev = base; lev <= top; ++lev) {
        unsigned b = __ballot_sync(0xffffffffu, l >= lev);
        if ((threadIdx.x & 31) == 0 && b) atomicAdd(&c[lev], __popc(b));
    }
    __syncthreads();
    if (threadIdx.x <= top - base) counts[(int64_t)threadIdx.x * nblocks + blockIdx.x] = c[base + threadIdx.x];
}

__global__ void __launch_bounds__(kHeadThreads) k_head_write(const uint64_t *__restrict__ keys,
                                                              const uint64_t *__restrict__ mkeys,
                                                              int64_t n, int base, int top, int nblocks,
                                                              const int32_t *__restrict__ offsets,
                                                              GridView view, uint64_t **cell_key) {
    __shared__ int wsum[kHeadThreads / 32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t s = (int64_t)blockIdx.x * kHeadThreads + threadIdx.x;
    int l = s < n ? split_level(keys, s) : -1;
    uint64_t key = s < n ? mkeys[s] : 0;          // the cell's Morton key, for the hash tables
    for (int lev = base; lev <= top; ++lev) {
        unsigned b = __ballot_sync(0xffffffffu, l >= lev);
        if (lane == 0) wsum[warp] = __popc(b);
        __syncthreads();
        int before = 0;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        if (l >= lev) {
            int ord = offsets[(int64_t)(lev - base) * nblocks + blockIdx.x] + before + __popc(b & lanemask_lt());
            const_cast<int32_t *>(view.level[lev].cell_start)[ord] = (int32_t)s;
            cell_key[lev][ord] = key >> (3 * lev);
        }
        __syncthreads();
    }
}

__global__ void k_hash_insert(GridView view, uint64_t *const *cell_key, int base, int n_total) {
    int lev = base + blockIdx.y;
    const LevelTable &t = view.level[lev];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < t.ncells; c += gridDim.x * blockDim.x) {
        uint64_t key = cell_key[lev][c];
        uint32_t h = hash_key(key) & t.hmask;
        uint64_t *slots = const_cast<uint64_t *>(t.hkeys);
        for (uint32_t probe = 0; probe <= t.hmask; ++probe) {
            unsigned long long prev = atomicCAS((unsigned long long *)(slots + h), (unsigned long long)kEmptyKey,
                                                (unsigned long long)key);
            if (prev == kEmptyKey || prev == key) {
                const_cast<int32_t *>(t.hvals)[h] = c;
                break;
            }
            h = (h + 1) & t.hmask;
        }
        if (c == 0) const_cast<int32_t *>(t.cell_start)[t.ncells] = n_total;
    }
}

template <typename T>
int grow(T **p, size_t count, size_t *cap) {
    if (*p && *cap >= count) return MLS_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    size_t c = count < 1 ? 1 : count;
    MLS_CUDA_TRY(cudaMalloc((void **)p, c * sizeof(T)));
    *cap = c;
    return MLS_OK;
}

int blocks_for(int64_t n, int threads, int per_sm = 16) {
    const int64_t cap = (int64_t)sm_count() * per_sm;
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

}  // namespace

void free_grid_buffers(mls_grid *g) {
    if (g->side) cudaStreamSynchronize(g->side);
    for (cudaEvent_t &e : g->side_ev)
        if (e) {
            cudaEventDestroy(e);
            e = nullptr;
        }
    if (g->side) {
        cudaStreamDestroy(g->side);
        g->side = nullptr;
    }
    cudaFree(g->mkeys);
    cudaFree(g->keys);
    cudaFree(g->keys_alt);
    cudaFree(g->perm);
    cudaFree(g->perm_alt);
    cudaFree(g->pts);
    cudaFree(g->block_hist);
    cudaFree(g->scan_tmp);
    cudaFree(g->misc);
    cudaFree(g->work);
    cudaFreeHost(g->misc_host);
    for (int l = 0; l < kMaxLevels; ++l) {
        cudaFree(g->hkeys[l]);
        cudaFree(g->hvals[l]);
        cudaFree(g->cell_start[l]);
        cudaFree(g->cell_key[l]);
    }
}

int build_grid(mls_grid *g, const float *xyz, int64_t n, float cell_size, int k_hint, cudaStream_t st) {
    g->stream = st;
    g->xyz = xyz;
    g->n = n;
    g->k_hint = k_hint;
    if (g->cap < n) {
        cudaFree(g->keys);
        cudaFree(g->keys_alt);
        cudaFree(g->mkeys);
        cudaFree(g->perm);
        cudaFree(g->perm_alt);
        cudaFree(g->pts);
        g->keys = g->keys_alt = g->mkeys = nullptr;
        g->perm = g->perm_alt = nullptr;
        g->pts = nullptr;
        g->cap = 0;
        MLS_CUDA_TRY(cudaMalloc(&g->keys, n * sizeof(uint64_t)));
        MLS_CUDA_TRY(cudaMalloc(&g->keys_alt, n * sizeof(uint64_t)));
        MLS_CUDA_TRY(cudaMalloc(&g->mkeys, n * sizeof(uint64_t)));
        MLS_CUDA_TRY(cudaMalloc(&g->perm, n * sizeof(int32_t)));
        MLS_CUDA_TRY(cudaMalloc(&g->perm_alt, n * sizeof(int32_t)));
        MLS_CUDA_TRY(cudaMalloc(&g->pts, n * sizeof(float4)));
        g->cap = n;
    }
    {
        int rc0 = grow(&g->work, (size_t)n + 8, &g->work_cap);
        if (rc0) return rc0;
    }
    if (!g->misc) {
        MLS_CUDA_TRY(cudaMalloc(&g->misc, sizeof(Misc)));
        MLS_CUDA_TRY(cudaMallocHost(&g->misc_host, sizeof(Misc)));
    }
    Misc *m = (Misc *)g->misc;
    const int T = 256;
    k_init_misc<<<1, 32, 0, st>>>(m);
    k_bbox<<<blocks_for(n, T), T, 0, st>>>(xyz, n, m);
    k_frame<<<1, 32, 0, st>>>(m);
    MLS_CUDA_TRY(cudaGetLastError());

    // radix sort of the keys' bits from level sort_level up, 8 bits a pass
    // (all 63 bits, 8 passes, on a first build; the search never uses the
    // cells below the base level, so later builds of the handle skip the bits
    // below one level under the last base: points within such a cell keep
    // their input order).  If the cloud turns out to want a finer base than
    // the partial sort resolves (its coarsest allowed level already holds 4x
    // the target occupancy), the keys are sorted again in full.
    int sort_level = cell_size > 0.0f ? 0 : g->sort_level;
    int nblocks = (int)((n + kSortTile - 1) / kSortTile);
    int rc = grow(&g->block_hist, (size_t)nblocks * kDigits, &g->block_hist_cap);
    if (rc) return rc;
    rc = grow(&g->scan_tmp, (size_t)kDigits + 64, &g->scan_tmp_cap);
    if (rc) return rc;
    const Misc *hm = (const Misc *)g->misc_host;
    int64_t cells[kMaxLevels];
    int top = kMaxLevels - 1;
    int base = top;
    for (;;) {
        // (the passes that cover the bits from 3 sort_level up start as low as
        // their width allows: the extra low bits order points within the cells
        // more finely at no cost)
        const int passes = (kKeyBits - 3 * sort_level + kDigitBits - 1) / kDigitBits;
        const int lo_shift = std::max(0, kKeyBits - kDigitBits * passes);     // lowest key bit the passes read
        k_keys<<<blocks_for(n, T), T, 0, st>>>(xyz, n, m, lo_shift / 3, g->keys, g->perm);
        count_launches(1);
        for (int shift = lo_shift; shift < kKeyBits; shift += kDigitBits) {
            k_radix_hist<<<nblocks, kSortThreads, 0, st>>>(g->keys, n, shift, nblocks, g->block_hist);
            k_radix_scan<<<kDigits, 1024, 0, st>>>(g->block_hist, nblocks, g->scan_tmp);
            k_radix_scatter<<<nblocks, kSortThreads, 0, st>>>(g->keys, g->perm, n, shift, nblocks, g->block_hist,
                                                              g->scan_tmp, g->keys_alt, g->perm_alt);
            uint64_t *tk = g->keys;
            g->keys = g->keys_alt;
            g->keys_alt = tk;
            int32_t *tp = g->perm;
            g->perm = g->perm_alt;
            g->perm_alt = tp;
        }
        count_launches(3 * passes + 2);     // the passes, the point gather, the level histogram
        MLS_CUDA_TRY(cudaMemsetAsync(m->level_hist, 0, sizeof(m->level_hist), st));
        k_gather_pts<<<blocks_for(n, T), T, 0, st>>>(xyz, g->perm, n, m, g->pts, g->mkeys);
        k_level_hist<<<blocks_for(n, T), T, 0, st>>>(g->keys, n, m);
        MLS_CUDA_TRY(cudaGetLastError());
        MLS_CUDA_TRY(cudaMemcpyAsync(g->misc_host, m, sizeof(Misc), cudaMemcpyDeviceToHost, st));
        MLS_CUDA_TRY(cudaStreamSynchronize(st));
        if (hm->nonfinite) return set_error(MLS_ERR_NONFINITE, "mls_build_grid: a coordinate is NaN or infinite");

        // unique cells per level: 1 + number of sorted neighbours split at or above it
        unsigned long long above = 0;
        for (int l = kMaxLevels - 1; l >= 0; --l) {
            above += hm->level_hist[l];
            cells[l] = 1 + (int64_t)above;
        }
        base = top;
        if (cell_size > 0.0f) {
            double r = std::log2((double)cell_size / (double)hm->frame.s0);
            base = (int)std::lround(r);
            if (base < 0) base = 0;
            if (base > top) base = top;
            break;
        }
        // finest level whose mean occupancy reaches k_hint / 6 (the cell
        // counts are exact from the sorted level up)
        const double target = k_hint / 6.0 > 1.0 ? k_hint / 6.0 : 1.0;
        for (int l = sort_level; l <= top; ++l)
            if ((double)n / (double)cells[l] >= target) {
                base = l;
                break;
            }
        if (sort_level == 0 || base > sort_level || (double)n / (double)cells[base] < 4.0 * target) break;
        sort_level = 0;
    }
    GridView &v = g->view;
    v.pts = g->pts;
    v.keys = g->mkeys;
    v.frame = hm->frame;
    v.n = (int32_t)n;
    v.base_level = base;
    g->sort_level = base > 0 ? base - 1 : 0;
    v.top_level = top;
    for (int l = 0; l < kMaxLevels; ++l) v.side[l] = std::ldexp(hm->frame.s0, l);
    int nlev = top - base + 1;
    for (int l = 0; l < kMaxLevels; ++l) v.level[l] = LevelTable{};
    for (int l = base; l <= top; ++l) {
        size_t cap = 64;
        while (cap < (size_t)(2 * cells[l])) cap <<= 1;
        if (g->hcap[l] < cap) {
            cudaFree(g->hkeys[l]);
            cudaFree(g->hvals[l]);
            g->hkeys[l] = nullptr;
            g->hvals[l] = nullptr;
            g->hcap[l] = 0;
            MLS_CUDA_TRY(cudaMalloc(&g->hkeys[l], cap * sizeof(uint64_t)));
            MLS_CUDA_TRY(cudaMalloc(&g->hvals[l], cap * sizeof(int32_t)));
            g->hcap[l] = cap;
        }
        size_t need = (size_t)cells[l] + 1;
        if (g->ccap[l] < need) {
            cudaFree(g->cell_key[l]);
            cudaFree(g->cell_start[l]);
            g->cell_key[l] = nullptr;
            g->cell_start[l] = nullptr;
            g->ccap[l] = 0;
            MLS_CUDA_TRY(cudaMalloc(&g->cell_key[l], need * sizeof(uint64_t)));
            MLS_CUDA_TRY(cudaMalloc(&g->cell_start[l], need * sizeof(int32_t)));
            g->ccap[l] = need;
        }
        MLS_CUDA_TRY(cudaMemsetAsync(g->hkeys[l], 0xff, cap * sizeof(uint64_t), st));
        v.level[l].hkeys = g->hkeys[l];
        v.level[l].hvals = g->hvals[l];
        v.level[l].cell_start = g->cell_start[l];
        v.level[l].hmask = (uint32_t)(cap - 1);
        v.level[l].ncells = (int32_t)cells[l];
    }
    // cell starts and keys for every level in two passes over the sorted keys
    int hblocks = (int)((n + kHeadThreads - 1) / kHeadThreads);
    rc = grow(&g->block_hist, (size_t)hblocks * nlev, &g->block_hist_cap);
    if (rc) return rc;
    rc = grow(&g->scan_tmp, (size_t)kDigits + 64, &g->scan_tmp_cap);
    if (rc) return rc;
    uint64_t *host_ptrs[kMaxLevels];
    for (int l = 0; l < kMaxLevels; ++l) host_ptrs[l] = g->cell_key[l];
    uint64_t **dev_ptrs = m->cell_key;
    MLS_CUDA_TRY(cudaMemcpyAsync(dev_ptrs, host_ptrs, sizeof(host_ptrs), cudaMemcpyHostToDevice, st));
    k_head_count<<<hblocks, kHeadThreads, 0, st>>>(g->keys, n, base, top, hblocks, g->block_hist);
    k_radix_scan<<<nlev, 1024, 0, st>>>(g->block_hist, hblocks, g->scan_tmp);
    k_head_write<<<hblocks, kHeadThreads, 0, st>>>(g->keys, g->mkeys, n, base, top, hblocks, g->block_hist, v,
                                                   dev_ptrs);
    dim3 hg(blocks_for(cells[base], T), nlev);
    k_hash_insert<<<hg, T, 0, st>>>(v, dev_ptrs, base, (int)n);
    count_launches(3 + 4);     // init, bbox, frame; head count, scan, head write, hash insert
    MLS_CUDA_TRY(cudaGetLastError());
    return MLS_OK;
}

}  // namespace mls
