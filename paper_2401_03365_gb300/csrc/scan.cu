// Device-wide exclusive prefix sum of int32 (three passes: block scans, a
// scan of the block totals, and the carry-in add).
#include "common.cuh"

namespace mls {

namespace {

constexpr int kScanThreads = 1024;

__device__ __forceinline__ int block_incl_scan(int v, int *warp_tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) warp_tot[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int t = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    return v + (warp ? warp_tot[warp - 1] : 0);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(const int32_t *__restrict__ in, int32_t *__restrict__ out,
                                                              int64_t n, int32_t *__restrict__ sums) {
    __shared__ int warp_tot[32];
    const int64_t i = blockIdx.x * (int64_t)kScanThreads + threadIdx.x;
    const int v = i < n ? in[i] : 0;
    const int incl = block_incl_scan(v, warp_tot);
    if (i < n) out[i] = incl - v;
    if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = incl;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(int32_t *__restrict__ sums, int64_t m) {
    __shared__ int warp_tot[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < m; base += kScanThreads) {
        const int64_t i = base + threadIdx.x;
        const int v = i < m ? sums[i] : 0;
        const int incl = block_incl_scan(v, warp_tot);
        const int c = carry;
        if (i < m) sums[i] = c + incl - v;
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) carry = c + incl;
        __syncthreads();
    }
}

__global__ void k_scan_add(int32_t *__restrict__ out, int64_t n, const int32_t *__restrict__ sums) {
    const int64_t i = blockIdx.x * (int64_t)kScanThreads + threadIdx.x;
    if (i < n) out[i] += sums[blockIdx.x];
}

}  // namespace

int device_exclusive_scan(const int32_t *in, int32_t *out, int64_t n, cudaStream_t st) {
    const int64_t blocks = (n + kScanThreads - 1) / kScanThreads;
    int32_t *sums = nullptr;
    MLS_CUDA_TRY(scratch_alloc((void **)&sums, (size_t)blocks * sizeof(int32_t), st));
    k_scan_blocks<<<(unsigned)blocks, kScanThreads, 0, st>>>(in, out, n, sums);
    k_scan_sums<<<1, kScanThreads, 0, st>>>(sums, blocks);
    k_scan_add<<<(unsigned)blocks, kScanThreads, 0, st>>>(out, n, sums);
    count_launches(3);
    MLS_CUDA_TRY(cudaGetLastError());
    MLS_CUDA_TRY(cudaFreeAsync(sums, st));
    return MLS_OK;
}

}  // namespace mls
