// Device-wide exclusive prefix sums of int32 and int64 (three passes: block
// scans, a scan of the block totals, and the carry-in add), and the stream
// compaction built on them.
#include <algorithm>

#include "common.cuh"

namespace mls {

namespace {

constexpr int kScanThreads = 1024;

template <typename T>
__device__ __forceinline__ T block_incl_scan(T v, T *warp_tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) warp_tot[warp] = v;
    __syncthreads();
    if (warp == 0) {
        T t = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    return v + (warp ? warp_tot[warp - 1] : 0);
}

template <typename TI, typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(const TI *__restrict__ in, int64_t n_in,
                                                              T *__restrict__ out, int64_t n, T *__restrict__ sums) {
    __shared__ T warp_tot[32];
    const int64_t i = blockIdx.x * (int64_t)kScanThreads + threadIdx.x;
    const T v = i < n_in ? (T)in[i] : T(0);
    const T incl = block_incl_scan<T>(v, warp_tot);
    if (i < n) out[i] = incl - v;
    if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = incl;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(T *__restrict__ sums, int64_t m) {
    __shared__ T warp_tot[32];
    __shared__ T carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < m; base += kScanThreads) {
        const int64_t i = base + threadIdx.x;
        const T v = i < m ? sums[i] : T(0);
        const T incl = block_incl_scan<T>(v, warp_tot);
        const T c = carry;
        if (i < m) sums[i] = c + incl - v;
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) carry = c + incl;
        __syncthreads();
    }
}

template <typename T>
__global__ void k_scan_add(T *__restrict__ out, int64_t n, const T *__restrict__ sums) {
    const int64_t i = blockIdx.x * (int64_t)kScanThreads + threadIdx.x;
    if (i < n) out[i] += sums[blockIdx.x];
}

// Flag of the entries to keep: (status & mask) == 0.
__global__ void k_keep_flags(const uint8_t *__restrict__ status, int64_t n, int mask, int32_t *__restrict__ flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = (status[i] & mask) == 0;
}

__global__ void k_keep_scatter(const int32_t *__restrict__ flag, const int32_t *__restrict__ pos, int64_t n,
                               int32_t *__restrict__ kept, int64_t *__restrict__ num) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (flag[i]) kept[pos[i]] = (int32_t)i;
        if (i == n - 1) *num = (int64_t)pos[i] + flag[i];
    }
}

// n outputs over the first n_in <= n inputs (the rest count as zero).
template <typename TI, typename T>
int scan_impl(const TI *in, int64_t n_in, T *out, int64_t n, cudaStream_t st) {
    const int64_t blocks = (n + kScanThreads - 1) / kScanThreads;
    ScratchSet scratch(st);
    T *sums = nullptr;
    MLS_CUDA_TRY(scratch.alloc(&sums, (size_t)blocks * sizeof(T)));
    k_scan_blocks<TI, T><<<(unsigned)blocks, kScanThreads, 0, st>>>(in, n_in, out, n, sums);
    k_scan_sums<T><<<1, kScanThreads, 0, st>>>(sums, blocks);
    k_scan_add<T><<<(unsigned)blocks, kScanThreads, 0, st>>>(out, n, sums);
    count_launches(3);
    MLS_CUDA_TRY(cudaGetLastError());
    return MLS_OK;
}

}  // namespace

int device_exclusive_scan(const int32_t *in, int32_t *out, int64_t n, cudaStream_t st) {
    return scan_impl<int32_t, int32_t>(in, n, out, n, st);
}

// out[i] = sum of in[0 .. i), widened to int64; n + 1 outputs (the last the total).
int device_exclusive_scan64(const int32_t *in, int64_t *out, int64_t n, cudaStream_t st) {
    return scan_impl<int32_t, int64_t>(in, n, out, n + 1, st);
}

int device_compact(const uint8_t *status, int64_t n, int mask, int32_t *kept, int64_t *num, cudaStream_t st) {
    ScratchSet scratch(st);
    int32_t *flag = nullptr;
    MLS_CUDA_TRY(scratch.alloc(&flag, (size_t)(2 * n) * sizeof(int32_t)));
    int32_t *pos = flag + n;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 16);
    k_keep_flags<<<grid, 256, 0, st>>>(status, n, mask, flag);
    int rc = device_exclusive_scan(flag, pos, n, st);
    if (rc != MLS_OK) return rc;
    k_keep_scatter<<<grid, 256, 0, st>>>(flag, pos, n, kept, num);
    count_launches(2);
    MLS_CUDA_TRY(cudaGetLastError());
    return MLS_OK;
}

}  // namespace mls
