// Device helpers shared by the kernels of libmls (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mls.h"

namespace mls {

constexpr int kWarp = 32;
// A warp's 32 neighbour rows staged transposed in shared memory: entry j of
// lane t at j * kRowStride + t.  A stride of 33 words puts the staging
// writes (lanes over j, one row at a time) and the reads (lanes over t) in
// 32 different banks; a stride of 32 made every staging write a 32-way bank
// conflict.
constexpr int kRowStride = 33;
constexpr int kMortonBits = 21;                  // bits per axis of a level-0 cell coordinate
constexpr uint32_t kAxisCells = 1u << kMortonBits;
constexpr int kMaxLevels = kMortonBits + 1;      // level L: cell side s0 * 2^L, L = 0..21

// Records the thread's last error message; returns `code`.
int set_error(int code, const char *fmt, ...);

// Clears the thread's last error message (every entry point starts so).
void clear_error();

// Adds to the process-wide count of kernel launches.
void count_launches(int n);

// Stream-ordered scratch from the library's per-device pool (scratch.cu);
// release with cudaFreeAsync on the same stream.
cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t st);

// Number of SMs of the current device (queried once per device); grids of
// grid-stride kernels are sized as multiples of it.
int sm_count();

// Scratch buffers of one call, freed together (cudaFreeAsync on the call's
// stream) when the set goes out of scope, on every exit path.
class ScratchSet {
  public:
    explicit ScratchSet(cudaStream_t st) : st_(st) {}
    ScratchSet(const ScratchSet &) = delete;
    ScratchSet &operator=(const ScratchSet &) = delete;
    ~ScratchSet() {
        for (int i = 0; i < n_; ++i) cudaFreeAsync(p_[i], st_);
    }
    template <class T>
    cudaError_t alloc(T **out, size_t bytes) {
        *out = nullptr;
        if (n_ == kMax) return cudaErrorInvalidValue;
        void *q = nullptr;
        const cudaError_t e = scratch_alloc(&q, bytes, st_);
        if (e != cudaSuccess) return e;
        p_[n_++] = q;
        *out = static_cast<T *>(q);
        return cudaSuccess;
    }

  private:
    static constexpr int kMax = 16;
    cudaStream_t st_;
    void *p_[kMax] = {};
    int n_ = 0;
};

#define MLS_CUDA_TRY(expr)                                                              \
    do {                                                                                \
        cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return ::mls::set_error(e_ == cudaErrorMemoryAllocation ? MLS_ERR_OOM       \
                                                                     : MLS_ERR_CUDA,    \
                                    "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_),    \
                                    __FILE__, __LINE__);                                \
    } while (0)

// Spread the low 21 bits of v so that bit b lands on bit 3b.
__host__ __device__ inline uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// Morton key: x on bit 0 of every triple, y on bit 1, z on bit 2.
__host__ __device__ inline uint64_t morton3(uint32_t cx, uint32_t cy, uint32_t cz) {
    return spread3(cx) | (spread3(cy) << 1) | (spread3(cz) << 2);
}

// Inverse of spread3: gather bits 0, 3, 6, ... into the low 21 bits.
__host__ __device__ inline uint32_t compact3(uint64_t x) {
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
    x = (x ^ (x >> 32)) & 0x1fffffull;
    return (uint32_t)x;
}

// Geometry of the level-0 grid, in float: cell side s0 (a power of two) and an
// origin that is a multiple of s0 (so both are exact floats), plus `eps`, a
// bound on how far float rounding can put a point outside the cell it is
// filed under, or move a computed distance from a point to a cell face: eight
// units in the last place of the largest coordinate magnitude of the domain.
struct GridFrame {
    float origin[3];
    float s0;
    float inv_s0;
    float eps;
};

// Level-0 cell coordinate of a coordinate value (clamped to the grid).
__device__ inline uint32_t cell_coord(float x, float origin, float inv_s0) {
    float g = floorf((x - origin) * inv_s0);
    g = fminf(fmaxf(g, 0.0f), (float)(kAxisCells - 1));
    return (uint32_t)g;
}

// Ordered-integer view of a float for atomic min / max.
__device__ inline int float_to_ordered(float f) {
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ inline float ordered_to_float(int i) {
    return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff);
}

__device__ inline unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ inline T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace mls
