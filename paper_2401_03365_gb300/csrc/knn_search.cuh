// Exact k nearest neighbours over the grid (the neighbour search of Sec. 2.2,
// read as kNN).
//
// Order and ties.  The key of candidate p for query q is the float
// fl((fl(dx^2) + fl(dy^2)) + fl(dz^2)), dx = fl(p.x - q.x), never fused; a
// candidate is the 64-bit word (key bits << 32 | point index), and since keys
// are non-negative floats, word order is exactly the order (key, index).  The
// result is the unique first k words.
//
// Work layout.  One warp per query; each warp walks runs of consecutive
// queries in the grid's order (the Hilbert order of the cells).  For every
// query the warp first gets a key bound tau with at least k points at or
// below it:
//   - chained: from each of the two previous queries, with k-th key kappa at
//     distance d, tau = (sqrt(kappa) + d)^2 (triangle inequality), inflated by
//     relative margins of 2^-20 per step, which cover float rounding; the
//     smaller of the two is used when it allows the base level;
//   - otherwise (chunk start, sparse region): the finest level whose 5x5x5
//     cube of cells around the query holds k points; its cells nearest to the
//     query holding 2k points are scanned and tau is the largest key of the
//     first histogram bucket reaching k.
// It then searches the 5x5x5 cube of the finest level whose cells are at least
// half the search radius sqrt(tau) (plus twice the frame's rounding bound
// eps), which then contains the search ball; cells whose box is farther than
// the radius are skipped.  The words with key <= tau (>= k of them, every
// true neighbour among them) are ranked by a 32-bucket counting sort on the
// key and a rank inside each bucket.  If more than 128 survive, tau is
// tightened from the bucket histogram and the search repeated; past that a
// sorted insertion list finishes the query.
//
// The cube's 125 cell ranges (four per lane) are cached in the warp's shared
// memory: queries that follow each other in the grid order mostly share them.
#pragma once

#include <algorithm>

#include "grid.cuh"

namespace mls {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kChunk = 128;         // largest run of consecutive queries per warp chain
constexpr int kMinChunk = 8;        // smallest run, near the end of the queue
constexpr int kCap = 128;           // kept-word capacity for the counting sort
constexpr int kSlots = 4;           // cube cells per lane: 4 x 32 >= 125
constexpr int kMaxSegWords = 64;    // segment-start bitmap: 2048 points per round
constexpr float kGrow = 1.0f + 0x1p-20f;

struct __align__(16) WarpBuf {
    unsigned long long surv[kCap];  // kept words (key bits << 32 | point index)
    unsigned long long tmp[kCap];
    int32_t spos[kCap];             // sorted positions of the kept words
    int32_t tpos[kCap];
    int32_t nb[64];                 // sorted positions of the previous query's neighbours
    unsigned segbits[kMaxSegWords]; // first point of each cell of the current round
    int hist[32];
    int fill[32];
    unsigned binmax[32];
    int nprev;                      // kept words of the last ranked query (in tpos)
    int cell_start[32];             // cells of the current visiting round
    int cell_count[32];
    int cube_start[kSlots * 32];    // the cached cube of cells (struct Cube)
    int cube_count[kSlots * 32];
    float kth;
};

// The ranking key: float differences, squares and sums, each rounded to
// nearest, association ((dx^2 + dy^2) + dz^2), never fused.
__device__ __forceinline__ float rank_key(float4 p, float qx, float qy, float qz) {
    float dx = __fsub_rn(p.x, qx);
    float dy = __fsub_rn(p.y, qy);
    float dz = __fsub_rn(p.z, qz);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

__device__ __forceinline__ unsigned long long pack(float key, float4 p) {
    return ((unsigned long long)__float_as_uint(key) << 32) | (uint32_t)__float_as_int(p.w);
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Offsets of cube cell j (0..124) from the centre cell.
__device__ __forceinline__ void cube_offset(int j, int &dx, int &dy, int &dz) {
    dx = j % 5 - 2;
    dy = (j / 5) % 5 - 2;
    dz = j / 25 - 2;
}

// The 5x5x5 cube of cells around (cx, cy, cz) at level lev: cell j = r * 32 +
// lane is held by this lane in slot r.  M = points in the whole cube.
// The cell ranges live in the warp's shared buffer (slot r of lane t at
// r * 32 + t): kept in registers or local memory they would be spilled and
// written back through L2 on every reload.
struct Cube {
    int lev = -1, cx = 0, cy = 0, cz = 0, M = 0;
    int *st = nullptr, *ct = nullptr;    // this lane's slots: st[r * 32], ct[r * 32]
};

// Looks the 125 cells of the cube around (cx, cy, cz) up in table t (dims
// cells per axis) with the four probes of a lane in flight together, writes
// this lane's slots st[r * 32], ct[r * 32] and returns the cube's point
// count.  Out of line: it runs only when a query's cube differs from the
// previous one, and one body keeps the search kernels' code small.
__device__ __noinline__ int fetch_cube(const LevelTable t, int dims, int cx, int cy, int cz, int *st_out,
                                       int *ct_out, int lane) {
    uint64_t key[kSlots];
    uint32_t h[kSlots];
    bool live[kSlots];
#pragma unroll
    for (int r = 0; r < kSlots; ++r) {
        const int j = r * 32 + lane;
        int dx, dy, dz;
        cube_offset(j, dx, dy, dz);
        const int x = cx + dx, y = cy + dy, z = cz + dz;
        live[r] = j < 125 && x >= 0 && y >= 0 && z >= 0 && x < dims && y < dims && z < dims;
        key[r] = live[r] ? morton3((uint32_t)x, (uint32_t)y, (uint32_t)z) : 0;
        h[r] = hash_key(key[r]) & t.hmask;
    }
    uint64_t slot[kSlots];
#pragma unroll
    for (int r = 0; r < kSlots; ++r) slot[r] = live[r] ? __ldg(t.hkeys + h[r]) : kEmptyKey;
    int id[kSlots];
#pragma unroll
    for (int r = 0; r < kSlots; ++r) {
        id[r] = -1;
        if (!live[r]) continue;
        for (uint32_t probe = 0; probe <= t.hmask; ++probe) {
            if (slot[r] == key[r]) {
                id[r] = __ldg(t.hvals + h[r]);
                break;
            }
            if (slot[r] == kEmptyKey) break;
            h[r] = (h[r] + 1) & t.hmask;
            slot[r] = __ldg(t.hkeys + h[r]);
        }
    }
    int tot = 0;
#pragma unroll
    for (int r = 0; r < kSlots; ++r) {
        int st = 0, ct = 0;
        if (id[r] >= 0) {
            st = __ldg(t.cell_start + id[r]);
            ct = __ldg(t.cell_start + id[r] + 1) - st;
        }
        st_out[r * 32] = st;
        ct_out[r * 32] = ct;
        tot += ct;
    }
    return warp_sum(tot);
}

// The cube of level lev around the query's level-0 cell c0, unless it is the
// one already cached.
__device__ __forceinline__ void load_cube(const GridView &g, int lev, const uint32_t c0[3], Cube &cb, int lane) {
    const int cx = (int)(c0[0] >> lev), cy = (int)(c0[1] >> lev), cz = (int)(c0[2] >> lev);
    if (cb.lev == lev && cb.cx == cx && cb.cy == cy && cb.cz == cz) return;
    cb.lev = lev;
    cb.cx = cx;
    cb.cy = cy;
    cb.cz = cz;
    cb.M = fetch_cube(g.level[lev], (int)(kAxisCells >> lev), cx, cy, cz, cb.st, cb.ct, lane);
}

// Squared distance from q to the box of this lane's cube cell in slot r.
__device__ __forceinline__ float cell_dist2(const GridView &g, const Cube &cb, int r, int lane, float4 q) {
    int dx, dy, dz;
    cube_offset(r * 32 + lane, dx, dy, dz);
    const float S = g.side[cb.lev];
    const float lx = g.frame.origin[0] + (float)(cb.cx + dx) * S;
    const float ly = g.frame.origin[1] + (float)(cb.cy + dy) * S;
    const float lz = g.frame.origin[2] + (float)(cb.cz + dz) * S;
    const float gx = fmaxf(0.f, fmaxf(lx - q.x, q.x - (lx + S)));
    const float gy = fmaxf(0.f, fmaxf(ly - q.y, q.y - (ly + S)));
    const float gz = fmaxf(0.f, fmaxf(lz - q.z, q.z - (lz + S)));
    return gx * gx + gy * gy + gz * gz;
}

// Visits every point of the cube cells with box distance^2 <= lim2, 32 at a
// time (one per lane; `valid` false on idle lanes).  The non-empty selected
// cells are packed onto the lanes (32 per round) and a bitmap of the first
// point of each cell maps a lane's point number to its cell in O(1).
// What the visit of a cube's cells needs from the grid, passed by value to the
// out-of-line scan (a reference to the grid view there would read its fields
// through memory on every call).
struct CellGeom {
    const float4 *pts;
    float S, ox, oy, oz;     // cell side at the cube's level, frame origin
};

__device__ __forceinline__ CellGeom cell_geom(const GridView &g, const Cube &cb) {
    return CellGeom{g.pts, g.side[cb.lev], g.frame.origin[0], g.frame.origin[1], g.frame.origin[2]};
}

template <int U, typename F>
__device__ void for_each_point(const CellGeom &g, const Cube &cb, WarpBuf &wb, float4 q, float lim2, int lane,
                               F &&f) {
    // squared gap from q to the cube's slabs: lane 5 a + t (a < 3, t < 5)
    // holds axis a at cell offset t - 2; a cell's box distance^2 is the sum
    // of its three slabs' gaps (rounding of a few ulps, far inside the
    // 2^-20 margins of lim2)
    float gap2 = 0.f;
    {
        const int ax = lane / 5, t = lane - 5 * ax;
        if (ax < 3) {
            const float S = g.S;
            const int c = ax == 0 ? cb.cx : (ax == 1 ? cb.cy : cb.cz);
            const float qa = ax == 0 ? q.x : (ax == 1 ? q.y : q.z);
            const float o = ax == 0 ? g.ox : (ax == 1 ? g.oy : g.oz);
            const float lo = o + (float)(c + t - 2) * S;
            const float gp = fmaxf(0.f, fmaxf(lo - qa, qa - (lo + S)));
            gap2 = gp * gp;
        }
    }
    bool sel[kSlots];
    int nsel = 0;
#pragma unroll
    for (int r = 0; r < kSlots; ++r) {
        const int j = r * 32 + lane;     // cells past 124 are empty (ct = 0)
        const int jx = j % 5, jy = (j / 5) % 5, jz = min(j / 25, 4);
        const float d2 = (__shfl_sync(kFull, gap2, jx) + __shfl_sync(kFull, gap2, 5 + jy)) +
                         __shfl_sync(kFull, gap2, 10 + jz);
        sel[r] = cb.ct[r * 32] > 0 && d2 <= lim2;
        nsel += sel[r];
    }
    const int incl_sel = warp_incl_scan(nsel, lane);
    const int total_sel = __shfl_sync(kFull, incl_sel, 31);
    for (int round = 0; round < total_sel; round += 32) {
        // cell number `round + lane` of the selection goes to this lane
        int my_start = 0, my_count = 0;
        int c = incl_sel - nsel;       // selection number of this lane's first selected slot
#pragma unroll
        for (int r = 0; r < kSlots; ++r) {
            if (sel[r]) {
                const int dst = c - round;
                // each lane publishes its selected cells through shared memory
                if (dst >= 0 && dst < 32) {
                    wb.cell_start[dst] = cb.st[r * 32];
                    wb.cell_count[dst] = cb.ct[r * 32];
                }
                ++c;
            }
        }
        __syncwarp();
        const int ncell = min(32, total_sel - round);
        if (lane < ncell) {
            my_start = wb.cell_start[lane];
            my_count = wb.cell_count[lane];
        }
        __syncwarp();
        const int incl = warp_incl_scan(my_count, lane);
        const int total = __shfl_sync(kFull, incl, 31);
        const int excl = incl - my_count;
        // bitmap of cell starts (cells are non-empty, so starts are distinct)
        const int words = (total + 31) >> 5;
        for (int w = lane; w < words && w < kMaxSegWords; w += 32) wb.segbits[w] = 0u;
        __syncwarp();
        if (lane < ncell && excl < 32 * kMaxSegWords) atomicOr(&wb.segbits[excl >> 5], 1u << (excl & 31));
        __syncwarp();
        int segbase = 0;     // cells starting before the current batch
        const unsigned le = (2u << lane) - 1u;
        // U rounds of 32 points at a time: their loads are issued together
        for (int base0 = 0; base0 < total; base0 += 32 * U) {
            float4 pt[U];
            int pos[U];
            bool valid[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int base = base0 + 32 * u;
                const int e = base + lane;
                valid[u] = e < total;
                int j = 0;
                unsigned w = 0u;
                if (base < total) {
                    if (total <= 32 * kMaxSegWords) {
                        w = wb.segbits[base >> 5];
                        j = segbase + __popc(w & le) - 1;
                    } else {              // very large rounds: search the inclusive counts
#pragma unroll
                        for (int step = 16; step >= 1; step >>= 1) {
                            int v = __shfl_sync(kFull, incl, j + step - 1);
                            if (v <= e) j += step;
                        }
                    }
                }
                j &= 31;
                const int st = __shfl_sync(kFull, my_start, j);
                const int ex = __shfl_sync(kFull, excl, j);
                segbase += __popc(w);
                pos[u] = valid[u] ? st + (e - ex) : 0;
                pt[u] = __ldg(g.pts + pos[u]);
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (base0 + 32 * u < total) f(pt[u], valid[u], pos[u]);
        }
        __syncwarp();
    }
}

// Key buckets, monotone in the key.  With lo = 0: 32 buckets of width
// 1 / scale from 0 (the last also takes every larger key).  With lo > 0:
// bucket 0 takes the keys below lo and buckets 1-31 split [lo, lo + 31 / scale).
struct Bins {
    float lo, scale;
    __device__ __forceinline__ int operator()(float key) const {
        if (lo > 0.f) return key < lo ? 0 : min(31, 1 + (int)((key - lo) * scale));
        return min(31, (int)(key * scale));
    }
};

// Keeps the visited words with key <= tau: the first kCap (word and sorted
// position) go to the buffers.  Returns the number kept.  With hist, every
// kept key is also counted in the 32 buckets of `bins` with each bucket's
// largest key, for tightening tau when far too many are kept.
// Out of line, one copy for all callers: the query solver around it is
// inlined into the kernels, and a single body keeps the code they share in
// the instruction cache.
template <int U>
__device__ __forceinline__ int scan_keep_body(const CellGeom &g, const Cube &cb, WarpBuf &wb, float4 q, float lim2,
                                              float tau, Bins bins, int lane, bool hist) {
    if (hist) {
        __syncwarp();
        wb.hist[lane] = 0;
        wb.binmax[lane] = 0u;
        __syncwarp();
    }
    int S = 0;
    for_each_point<U>(g, cb, wb, q, lim2, lane, [&](float4 p, bool valid, int pos) {
        const float key = rank_key(p, q.x, q.y, q.z);
        const bool keep = valid && key <= tau;
        const unsigned m = __ballot_sync(kFull, keep);
        if (keep) {
            const int slot = S + __popc(m & lanemask_lt());
            if (slot < kCap) {
                wb.surv[slot] = pack(key, p);
                wb.spos[slot] = pos;
            }
            if (hist) {
                const int bin = bins(key);
                atomicAdd(&wb.hist[bin], 1);
                atomicMax(&wb.binmax[bin], __float_as_uint(key));
            }
        }
        S += __popc(m);
    });
    __syncwarp();
    return S;
}

template <int U>
__device__ __noinline__ int scan_keep(const CellGeom g, const Cube &cb, WarpBuf &wb, float4 q, float lim2,
                                      float tau, Bins bins, int lane, bool hist) {
    return scan_keep_body<U>(g, cb, wb, q, lim2, tau, bins, lane, hist);
}

// Histogram (count and largest key) of the first min(S, kCap) kept words in
// the 32 buckets of `bins`.
__device__ void bucket_hist(WarpBuf &wb, int S, Bins bins, int lane) {
    wb.hist[lane] = 0;
    wb.binmax[lane] = 0u;
    __syncwarp();
    for (int s = lane; s < min(S, kCap); s += 32) {
        const float key = __uint_as_float((uint32_t)(wb.surv[s] >> 32));
        const int bin = bins(key);
        atomicAdd(&wb.hist[bin], 1);
        atomicMax(&wb.binmax[bin], __float_as_uint(key));
    }
    __syncwarp();
}

// Smallest key bound with at least k histogrammed words at or below it: the
// largest key of the buckets up to the one where the running count reaches k
// (that bucket's number in *bstar_out, -1 with the fallback; the running
// count through it in *count_out).
__device__ float tighten(const WarpBuf &wb, int k, int lane, float fallback, int *bstar_out = nullptr,
                         int *count_out = nullptr) {
    const int incl = warp_incl_scan(wb.hist[lane], lane);
    const unsigned reach = __ballot_sync(kFull, incl >= k);
    if (bstar_out) *bstar_out = reach ? __ffs(reach) - 1 : -1;
    if (count_out) *count_out = __shfl_sync(kFull, incl, reach ? __ffs(reach) - 1 : 31);
    if (!reach) return fallback;
    const int bstar = __ffs(reach) - 1;
    unsigned mx = lane <= bstar ? wb.binmax[lane] : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
    return __uint_as_float(mx);
}

// Where a query's row goes: its neighbours' original indices (row = the
// query's original index) and their keys in the same layout, and their
// sorted positions (row = the query's sorted position); any may be NULL.
struct RowOut {
    int32_t *idx;
    float *key;
    int32_t *pos;

    // entry `rank` of the row of query qi (sorted position sp): neighbour
    // with original index i, key `key_`, sorted position p
    __device__ __forceinline__ void put(int32_t qi, int64_t sp, int k, int rank, int32_t i, float key_,
                                        int32_t p) const {
        if (idx) idx[(int64_t)qi * k + rank] = i;
        if (key) key[(int64_t)qi * k + rank] = key_;
        if (pos) pos[sp * k + rank] = p;
    }
};

// Counting sort of the S <= kCap kept words by bucket, then rank inside the
// bucket; the first k go to the output row and their sorted positions to
// wb.nb.  Returns the k-th key.
template <class Out>
__device__ float rank_and_write(WarpBuf &wb, int S, Bins bins, int k, int lane, int32_t qi, int64_t sp,
                                const Out &out) {
    bucket_hist(wb, S, bins, lane);
    const int h = wb.hist[lane];
    wb.fill[lane] = warp_incl_scan(h, lane) - h;
    __syncwarp();
    for (int s = lane; s < S; s += 32) {
        const unsigned long long v = wb.surv[s];
        const int bin = bins(__uint_as_float((uint32_t)(v >> 32)));
        const int at = atomicAdd(&wb.fill[bin], 1);
        wb.tmp[at] = v;
        wb.tpos[at] = wb.spos[s];
    }
    __syncwarp();
    for (int p = lane; p < S; p += 32) {
        const unsigned long long v = wb.tmp[p];
        const float key = __uint_as_float((uint32_t)(v >> 32));
        const int bin = bins(key);
        const int end = wb.fill[bin], beg = end - wb.hist[bin];
        int rank = beg;
        for (int t = beg; t < end; ++t) rank += wb.tmp[t] < v;
        if (rank < k) {
            out.put(qi, sp, k, rank, (int32_t)(uint32_t)v, key, wb.tpos[p]);
            if (rank < 64) wb.nb[rank] = wb.tpos[p];     // the radius rows can be longer than a kNN row
            if (rank == k - 1) wb.kth = key;
        }
    }
    if (lane == 0) wb.nprev = S;
    __syncwarp();
    return wb.kth;
}

// Sorted insertion list over the lanes (entry r * 32 + lane in register r),
// the fallback when too many words share the smallest keys.
template <int KPL>
struct TopK {
    unsigned long long e[KPL];
    int pos[KPL];
    unsigned long long kth;

    __device__ void init() {
#pragma unroll
        for (int r = 0; r < KPL; ++r) {
            e[r] = ~0ull;
            pos[r] = 0;
        }
        kth = ~0ull;
    }

    __device__ void offer(unsigned long long cand, int cpos, int k, int lane) {
        unsigned m = __ballot_sync(kFull, cand < kth);
        while (m) {
            const int src = __ffs(m) - 1;
            const unsigned long long c = __shfl_sync(kFull, cand, src);
            const int cp = __shfl_sync(kFull, cpos, src);
            int at = 0;
#pragma unroll
            for (int r = 0; r < KPL; ++r) at += __popc(__ballot_sync(kFull, e[r] < c));
            unsigned long long up[KPL];
            int upp[KPL];
#pragma unroll
            for (int r = 0; r < KPL; ++r) {
                up[r] = __shfl_up_sync(kFull, e[r], 1);
                upp[r] = __shfl_up_sync(kFull, pos[r], 1);
            }
#pragma unroll
            for (int r = 1; r < KPL; ++r) {
                const unsigned long long carry = __shfl_sync(kFull, e[r - 1], 31);
                const int carryp = __shfl_sync(kFull, pos[r - 1], 31);
                if (lane == 0) {
                    up[r] = carry;
                    upp[r] = carryp;
                }
            }
#pragma unroll
            for (int r = 0; r < KPL; ++r) {
                const int idx = r * 32 + lane;
                if (idx > at) {
                    e[r] = up[r];
                    pos[r] = upp[r];
                } else if (idx == at) {
                    e[r] = c;
                    pos[r] = cp;
                }
            }
            const int kr = (k - 1) >> 5, kl = (k - 1) & 31;
            unsigned long long kv = e[0];
#pragma unroll
            for (int r = 1; r < KPL; ++r)
                if (r == kr) kv = e[r];
            kth = __shfl_sync(kFull, kv, kl);
            m &= ~(1u << src);
            m &= __ballot_sync(kFull, cand < kth);
        }
    }
};

template <int KPL, class Out>
__device__ float insertion_fallback(const CellGeom geo, const Cube &cb, WarpBuf &wb, float4 q, float lim2,
                                    float tau, int k, int lane, int32_t qi, int64_t sp, const Out &out) {
    TopK<KPL> top;
    top.init();
    for_each_point<1>(geo, cb, wb, q, lim2, lane, [&](float4 p, bool valid, int pos) {
        const float key = rank_key(p, q.x, q.y, q.z);
        top.offer(valid && key <= tau ? pack(key, p) : ~0ull, pos, k, lane);
    });
#pragma unroll
    for (int r = 0; r < KPL; ++r) {
        const int e = r * 32 + lane;
        if (e < k) {
            out.put(qi, sp, k, e, (int32_t)(uint32_t)top.e[r], __uint_as_float((uint32_t)(top.e[r] >> 32)),
                    top.pos[r]);
            wb.nb[e] = top.pos[r];
            wb.tpos[e] = top.pos[r];
        }
    }
    if (lane == 0) wb.nprev = k;
    __syncwarp();
    return __uint_as_float((uint32_t)(top.kth >> 32));
}

// Key bound from an earlier query p (its k-th key kappa): its k neighbours
// are within sqrt(kappa) + |q - p| of q.
__device__ __forceinline__ float chain_bound(float4 q, float4 p, float kappa) {
    const float dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
    const float d = sqrtf(dx * dx + dy * dy + dz * dz) * kGrow;
    const float R = (sqrtf(kappa) * kGrow + d) * kGrow;
    return R * R * kGrow * kGrow;
}

// Key bound from the previous query's kept words (wb.nprev of them, sorted
// positions in wb.tpos, its k neighbours among them): the k-th smallest of
// their keys seen from q, to bucket precision (real points, so no margin).
template <int KPL>
__device__ float survivor_bound(const GridView &g, WarpBuf &wb, float4 q, int k, int lane) {
    const int S = wb.nprev;
    float key[kCap / 32];
    float mx = 0.f;
#pragma unroll
    for (int r = 0; r < kCap / 32; ++r) {
        const int e = r * 32 + lane;
        key[r] = e < S ? rank_key(__ldg(g.pts + wb.tpos[e]), q.x, q.y, q.z) : INFINITY;
        if (e < S) mx = fmaxf(mx, key[r]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
    __syncwarp();
    wb.hist[lane] = 0;
    wb.binmax[lane] = 0u;
    __syncwarp();
    const float scale = mx > 0.f ? 32.0f / mx : 0.f;
#pragma unroll
    for (int r = 0; r < kCap / 32; ++r)
        if (r * 32 + lane < S) {
            const int bin = min(31, (int)(key[r] * scale));
            atomicAdd(&wb.hist[bin], 1);
            atomicMax(&wb.binmax[bin], __float_as_uint(key[r]));
        }
    __syncwarp();
    return tighten(wb, k, lane, mx);
}

// Key bound from the previous query's neighbours: the largest of their keys
// seen from q (k real points, so no margin is needed).
template <int KPL>
__device__ __forceinline__ float neighbour_bound(const GridView &g, const WarpBuf &wb, float4 q, int k, int lane) {
    float mx = 0.f;
#pragma unroll
    for (int r = 0; r < KPL; ++r) {
        const int e = r * 32 + lane;
        if (e < k) mx = fmaxf(mx, rank_key(__ldg(g.pts + wb.nb[e]), q.x, q.y, q.z));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
    return mx;
}

// The warp search for one query (lanes over candidates): the query's own key
// bound (from the 5x5x5 cube of the finest level holding k points) unless a
// finite tau_in is given, then the cube search with culling, tightening and,
// as a last resort, the sorted insertion list.  Returns the k-th key.
template <int KPL, int U, class Out>
__device__ __forceinline__ float solve_query(const GridView &g, WarpBuf &wb, Cube &cb, float4 q, int32_t qi,
                                             int64_t sp, const uint32_t c0[3], float tau, int k, int lane,
                                             bool may_defer, const Out &out) {
    const float eps2 = 2.0f * g.frame.eps;
    // fewer than k points have a key below lo (known from a histogram of
    // every key <= tau): later histograms split [lo, tau] only
    float lo = 0.f;
    int bstar = -1;
    bool full_hist = false;
    if (!(tau < INFINITY)) {
        // fresh bound: coarsen until the cube holds k points, then take the
        // cells nearest to the query that hold 2k of them
        int lev = g.base_level;
        for (;; ++lev) {
            load_cube(g, lev, c0, cb, lane);
            if (cb.M >= k || lev >= g.top_level) break;
        }
        // a sparse neighbourhood (a cube above the base level) is left to
        // the pass that shares such queries among all warps
        if (may_defer && lev > g.base_level) return NAN;
        const float S = g.side[lev];
        // count-weighted histogram of cell distances over [0, 3S)
        __syncwarp();
        wb.hist[lane] = 0;
        __syncwarp();
        const float dscale = 32.0f / (3.0f * S);
#pragma unroll
        for (int r = 0; r < kSlots; ++r)
            if (cb.ct[r * 32] > 0)
                atomicAdd(&wb.hist[min(31, (int)(sqrtf(cell_dist2(g, cb, r, lane, q)) * dscale))], cb.ct[r * 32]);
        __syncwarp();
        const int need = min(2 * k, cb.M);
        const unsigned ok = __ballot_sync(kFull, warp_incl_scan(wb.hist[lane], lane) >= need);
        __syncwarp();
        // bucket 31 also holds every farther cell: then take them all
        const bool all = __ffs(ok) >= 32;
        const float rstar = (float)(__ffs(ok)) / dscale;
        const float lim = (rstar + eps2) * kGrow;
        const float lim2 = all ? INFINITY : lim * lim;
        // every visited point lies within lim + sqrt(3) S of q (any cube point
        // within 3 sqrt(3) S < 5.2 S): bucket all their keys over [0, hi]
        const float far = ((all ? 5.2f * S : lim) + 1.7320509f * S + eps2) * kGrow * kGrow;
        const float hi = far * far * kGrow;
        const Bins fb{0.f, hi > 0.f ? 32.0f / hi : 0.f};
        scan_keep<U>(cell_geom(g, cb), cb, wb, q, lim2, INFINITY, fb, lane, true);
        int below = 0;
        tau = tighten(wb, k, lane, hi, nullptr, &below);
        // the visited points alone put more than 2 kCap keys at or below tau:
        // a plain search would overflow, so the first one takes the histogram;
        // so does every deferred (sparse) query, whose first search usually
        // overflows and costs tens of thousands of candidates
        full_hist = below > 2 * kCap || !may_defer;
    }
    for (int iter = 0;; ++iter) {
        // finest level whose cube (radius two cells) holds the search ball
        const float reach = sqrtf(tau) * kGrow * kGrow + eps2;
        int lev = g.base_level;
        while (lev < g.top_level && !(2.0f * g.side[lev] > reach)) ++lev;
        load_cube(g, lev, c0, cb, lane);
        const float lim = (reach + eps2) * kGrow;
        const float lim2 = lim * lim;
        // ranking buckets over [0, tau]; tightening buckets over [lo, tau]
        const Bins rb{0.f, tau > 0.f ? 32.0f / tau : 0.f};
        const Bins tb = lo > 0.f ? Bins{lo, tau > lo ? 31.0f / (tau - lo) : 0.f} : rb;
        const int S = scan_keep<U>(cell_geom(g, cb), cb, wb, q, lim2, tau, tb, lane, full_hist);
        if (S >= k && S <= kCap) return rank_and_write(wb, S, rb, k, lane, qi, sp, out);
        if (S < k) {            // cannot happen for a valid bound: search everything
            tau = INFINITY;
            full_hist = false;
            continue;
        }
        if (iter >= 8) return insertion_fallback<KPL>(cell_geom(g, cb), cb, wb, q, lim2, tau, k, lane, qi, sp, out);
        if (full_hist) {        // buckets over every kept word: each round cuts ~32x
            tau = tighten(wb, k, lane, tau, &bstar);
            // the buckets before the k-th key's hold fewer than k keys
            const int first = lo > 0.f ? 1 : 0;     // first bucket of [lo, tau]
            if (bstar > first && tb.scale > 0.f) lo = tb.lo + (float)(bstar - first) / tb.scale;
            if (!(lo < tau)) lo = 0.f;              // a rounding tie at the edge: start over from 0
            full_hist = false;
        } else if (S <= 2 * kCap) {
            // a mild overflow: the first kCap kept words (real points) bound it
            bucket_hist(wb, S, rb, lane);
            tau = tighten(wb, k, lane, tau);
        } else {
            full_hist = true;   // rescan with buckets over all kept words
        }
    }
}

// ---- chains: one query per warp -----------------------------------------
//
// A warp takes runs of consecutive queries from a global counter: 128 at a
// time while many remain, fewer (down to 8) as the queue drains, so that the
// warps finish together.  The bound for a query comes from the query before
// it: the k-th smallest key,
// seen from the new query, of the points that query kept (its k neighbours
// among them), and the triangle bound from the query before that.  A fresh
// bound is computed when there is no earlier query, or the bound is more than
// 9 times the previous query's own k-th key or reaches past four base cells.
// Queries in sparse regions (their fresh bound needs a level above the base)
// are appended to a list and solved afterwards by k_knn_sparse, where
// all warps share them: they cost far more than the rest and would otherwise
// leave a few warps running long after the others.
//
// work[1]: deferred count; work[2]: next deferred; work[4..5]: next query
// (64-bit); work[8 ...]: sorted positions of the deferred queries.

constexpr int kChainThreads = 256;
constexpr int kChainWarps = kChainThreads / 32;

__device__ __forceinline__ int warp_take(int *counter, int lane) {
    int v = 0;
    if (lane == 0) v = atomicAdd(counter, 1);
    return __shfl_sync(kFull, v, 0);
}

// What a chain does with its finished queries.  PlainRows: nothing beyond
// the row outputs (the kNN alone).  A policy provides the launch bound
// kBlocksPerSm, start (once per warp, with the warp's global number),
// rows (the output object for the next finished query), done (the query at
// sorted position sp got its row) and finish (the warp has no more queries).
struct PlainRows {
    // Five blocks per SM (the shared buffers allow five): the kernel is bound
    // by instruction issue and latency, and more resident warps hide more of
    // the latter.
    static constexpr int kBlocksPerSm = 5;
    __device__ __forceinline__ void start(int64_t, int) {}
    __device__ __forceinline__ const RowOut &rows(const RowOut &out) const { return out; }
    __device__ __forceinline__ void done(int64_t, int) {}
    __device__ __forceinline__ void finish(int) {}
};

// SKIP: the queries flagged in skip[] are listed in iso (the work-list
// layout: count iso[1], next iso[2], sorted positions from iso[8]).  Every
// warp takes them first, one at a time, each searched in full (never
// deferred), and then the runs of the queue, stepping over the flagged
// queries (the chain's bounds hold between any two queries).  The listed
// queries are the costly ones: taken first by all warps, the longest of them
// end well before the queue does.
template <int KPL, class Fin, bool SKIP = false>
__global__ void __launch_bounds__(kChainThreads, Fin::kBlocksPerSm) k_knn_chain(GridView g, int k,
                                                                                int *__restrict__ work, RowOut out,
                                                                                Fin fin,
                                                                                const uint8_t *__restrict__ skip,
                                                                                int *__restrict__ iso) {
    __shared__ WarpBuf bufs[kChainWarps];
    const int lane = threadIdx.x & 31;
    WarpBuf &wb = bufs[threadIdx.x >> 5];
    const int64_t n_warps = (int64_t)gridDim.x * kChainWarps;
    unsigned long long *next_query = reinterpret_cast<unsigned long long *>(&work[4]);
    const float big = 16.0f * g.side[g.base_level] * g.side[g.base_level];
    Cube cb;
    cb.st = wb.cube_start + lane;
    cb.ct = wb.cube_count + lane;
    fin.start((blockIdx.x * (int64_t)kChainThreads + threadIdx.x) >> 5, lane);
    const int n_iso = SKIP ? iso[1] : 0;
    bool from_iso = SKIP && n_iso > 0;
    for (;;) {
        long long first = 0, len = 0;
        if (from_iso) {
            const int i = warp_take(&iso[2], lane);
            if (i < n_iso) {
                first = iso[8 + i];
                len = 1;
            } else {
                from_iso = false;
            }
        }
        if (!from_iso) {
            // run length from a racy read of the queue: any length is
            // correct, since every run is reserved by its own atomic add
            if (lane == 0) {
                const long long left = g.n - (long long)*(volatile unsigned long long *)next_query;
                len = min((long long)kChunk, max((long long)kMinChunk, left / (2 * n_warps)));
                first = (long long)atomicAdd(next_query, (unsigned long long)len);
            }
            first = __shfl_sync(kFull, first, 0);
            len = __shfl_sync(kFull, len, 0);
            if (first >= g.n) break;
        }
        // the previous query (its kept points in wb, k-th key k1, position
        // p1) and the one before it (position p2, k-th key k2)
        int n_prev = 0;
        float4 p1 = make_float4(0.f, 0.f, 0.f, 0.f), p2 = p1;
        float k1 = 0.f, k2 = 0.f;
        const int64_t end = min((int64_t)g.n, (int64_t)(first + len));
        for (int64_t sp = first; sp < end; ++sp) {
            if (SKIP && !from_iso && __ldg(skip + sp)) continue;
            const float4 q = __ldg(g.pts + sp);
            const uint64_t key0 = __ldg(g.keys + sp);
            const uint32_t c0[3] = {compact3(key0), compact3(key0 >> 1), compact3(key0 >> 2)};
            float tau = INFINITY;
            if (n_prev >= 1) tau = survivor_bound<KPL>(g, wb, q, k, lane);
            if (n_prev >= 2) tau = fminf(tau, chain_bound(q, p2, k2));
            // a bound far above the previous query's, or reaching past four
            // base cells, would search a large region: start afresh instead
            if (n_prev == 0 || tau > 9.0f * k1 || tau > big) tau = INFINITY;
            const float kth = solve_query<KPL, 1>(g, wb, cb, q, __float_as_int(q.w), sp, c0, tau, k, lane, !from_iso,
                                                  fin.rows(out));
            if (isnan(kth)) {
                if (lane == 0) work[8 + atomicAdd(&work[1], 1)] = (int)sp;
                n_prev = 0;
                continue;
            }
            fin.done(sp, lane);
            p2 = p1;
            k2 = k1;
            p1 = q;
            k1 = kth;
            n_prev = min(n_prev + 1, 2);
        }
    }
    fin.finish(lane);
}

// The sparse queries scan many candidates each, with few warps left to hide
// memory latency at the end of the pass: their candidate loads go four
// rounds of 32 at a time, and four blocks per SM stay resident (64 registers).
constexpr int kSparseRounds = 4;

template <int KPL, class Fin>
__global__ void __launch_bounds__(kChainThreads, 4) k_knn_sparse(GridView g, int k, int *__restrict__ work,
                                                                 RowOut out, Fin fin) {
    __shared__ WarpBuf bufs[kChainWarps];
    const int lane = threadIdx.x & 31;
    WarpBuf &wb = bufs[threadIdx.x >> 5];
    const int count = work[1];
    Cube cb;
    cb.st = wb.cube_start + lane;
    cb.ct = wb.cube_count + lane;
    fin.start((blockIdx.x * (int64_t)kChainThreads + threadIdx.x) >> 5, lane);
    for (int i = warp_take(&work[2], lane); i < count; i = warp_take(&work[2], lane)) {
        const int64_t sp = work[8 + i];
        const float4 q = __ldg(g.pts + sp);
        const uint64_t key0 = __ldg(g.keys + sp);
        const uint32_t c0[3] = {compact3(key0), compact3(key0 >> 1), compact3(key0 >> 2)};
        solve_query<KPL, kSparseRounds>(g, wb, cb, q, __float_as_int(q.w), sp, c0, INFINITY, k, lane, false,
                                        fin.rows(out));
        fin.done(sp, lane);
    }
    fin.finish(lane);
}

}  // namespace

}  // namespace mls
