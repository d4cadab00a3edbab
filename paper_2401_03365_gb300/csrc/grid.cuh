// Uniform-grid spatial index: device view and host-side owner.
#pragma once

#include "common.cuh"

namespace mls {

constexpr uint64_t kEmptyKey = ~0ull;   // Morton keys use 63 bits, so never a key

// Hash of a cell key (splitmix64 finaliser).
__host__ __device__ inline uint32_t hash_key(uint64_t k) {
    k ^= k >> 30;
    k *= 0xbf58476d1ce4e5b9ull;
    k ^= k >> 27;
    k *= 0x94d049bb133111ebull;
    k ^= k >> 31;
    return (uint32_t)k;
}

// Occupied cells of one level: an open-addressing table from the cell's key
// (level-0 key >> 3 * level) to its id, and the sorted range of each cell.
struct LevelTable {
    const uint64_t *hkeys;     // capacity slots, kEmptyKey when free
    const int32_t *hvals;      // cell id of each slot
    const int32_t *cell_start; // ncells + 1 sorted positions
    uint32_t hmask;            // capacity - 1 (capacity is a power of two)
    int32_t ncells;
};

// Everything a query kernel needs, passed by value.
struct GridView {
    const float4 *pts;         // sorted points: x, y, z, original index (int bits)
    const uint64_t *keys;      // level-0 Morton cell keys of the sorted points
    GridFrame frame;
    int32_t n;
    int32_t base_level;        // first level with a table
    int32_t top_level;         // last level (a single cell covers the cloud)
    float side[kMaxLevels];    // cell side per level, s0 * 2^level (exact)
    LevelTable level[kMaxLevels];
};

// Cell id of `key` at a level, or -1 when the cell is empty.
__device__ inline int32_t lookup_cell(const LevelTable &t, uint64_t key) {
    uint32_t h = hash_key(key) & t.hmask;
    for (uint32_t probe = 0; probe <= t.hmask; ++probe) {
        uint64_t k = __ldg(t.hkeys + h);
        if (k == key) return __ldg(t.hvals + h);
        if (k == kEmptyKey) return -1;
        h = (h + 1) & t.hmask;
    }
    return -1;
}

}  // namespace mls

// Host-side owner of the device buffers (opaque to C callers).
struct mls_grid {
    int device = -1;
    cudaStream_t stream = nullptr;
    int64_t n = 0, cap = 0;
    int k_hint = 0;
    const float *xyz = nullptr;
    // sort buffers and sorted data
    uint64_t *keys = nullptr, *keys_alt = nullptr;   // sort keys (Hilbert order of the level-0 cells)
    uint64_t *mkeys = nullptr;                       // Morton keys of the cells, in sorted order
    int32_t *perm = nullptr, *perm_alt = nullptr;
    float4 *pts = nullptr;
    int32_t *block_hist = nullptr;
    size_t block_hist_cap = 0;
    int32_t *scan_tmp = nullptr;
    size_t scan_tmp_cap = 0;
    // small device scratch: bbox, flags, level histogram, frame
    void *misc = nullptr;
    // kNN work list: counters and the deferred queries (n + 8 ints)
    int *work = nullptr;
    size_t work_cap = 0;
    void *misc_host = nullptr;   // pinned mirror
    // per-level tables
    uint64_t *hkeys[mls::kMaxLevels] = {};
    int32_t *hvals[mls::kMaxLevels] = {};
    int32_t *cell_start[mls::kMaxLevels] = {};
    uint64_t *cell_key[mls::kMaxLevels] = {};
    size_t hcap[mls::kMaxLevels] = {};
    size_t ccap[mls::kMaxLevels] = {};
    mls::GridView view{};
    // The next build orders the keys only by their bits at and above this
    // level (the cells finer than it are never searched): one level below
    // the base level of the last build; 0 (the whole key) at first.
    int sort_level = 0;
    // side stream (high priority) and events of the pipelined kNN and
    // projection, created on first use
    mutable cudaStream_t side = nullptr;
    mutable cudaEvent_t side_ev[2] = {nullptr, nullptr};
};
