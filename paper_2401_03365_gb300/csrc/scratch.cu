// Stream-ordered scratch memory of the library.
//
// The per-call buffers of the projection and its adjoint (up to ~1 GB per
// million points in the backward) come from a memory pool of the library's
// own, one per device, whose release threshold is unbounded: memory freed at
// the end of a call stays mapped for the next one.  The device's default pool
// would hand it back to the system at every synchronisation and map it again
// on the next allocation, which costs milliseconds per call on large clouds.
// mls_release_scratch() returns the unused part to the system.
#include <atomic>
#include <cstdint>
#include <mutex>

#include "common.cuh"

namespace mls {

namespace {
constexpr int kMaxDevices = 64;
cudaMemPool_t g_pools[kMaxDevices] = {};
std::mutex g_pool_mutex;

cudaError_t pool_for_current(cudaMemPool_t *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = UINT64_MAX;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        g_pools[dev] = pool;
    }
    *out = g_pools[dev];
    return cudaSuccess;
}
}  // namespace

int sm_count() {
    static std::atomic<int> counts[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 1;
    int c = counts[dev].load(std::memory_order_relaxed);
    if (c == 0) {
        if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c < 1) return 1;
        counts[dev].store(c, std::memory_order_relaxed);
    }
    return c;
}

cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t st) {
    cudaMemPool_t pool = nullptr;
    cudaError_t e = pool_for_current(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes < 1 ? 1 : bytes, pool, st);
}

}  // namespace mls

extern "C" int mls_release_scratch(void) {
    std::lock_guard<std::mutex> lock(mls::g_pool_mutex);
    for (int d = 0; d < mls::kMaxDevices; ++d) {
        if (!mls::g_pools[d]) continue;
        int cur = 0;
        MLS_CUDA_TRY(cudaGetDevice(&cur));
        MLS_CUDA_TRY(cudaSetDevice(d));
        const cudaError_t e1 = cudaDeviceSynchronize();
        const cudaError_t e2 = cudaMemPoolTrimTo(mls::g_pools[d], 0);
        MLS_CUDA_TRY(cudaSetDevice(cur));
        MLS_CUDA_TRY(e1);
        MLS_CUDA_TRY(e2);
    }
    return MLS_OK;
}
