// Batched MLS projection: many independent clouds of uneven size and k in
// one persistent launch (the per-point loop of Algorithm 1 run over the
// union of the clouds), its CUDA-graph capture, and the autotuner that picks
// the launch shape.
//
// Work is cut into tiles of tile_pts consecutive (grid-ordered) points of
// one cloud.  A persistent grid (SMs x resident blocks) takes tiles from one
// atomic counter; tiles are numbered cloud by cloud in decreasing order of k
// (then of size), so the most expensive tiles start first and the cheap ones
// fill the tail.  Within a tile a block handles blockDim / G points per round,
// G lanes per point (project_point), `rounds` rounds per tile.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "project_point.cuh"

struct mls_batch {
    int device = 0;
    int sms = 0;
    int B = 0;
    int64_t total = 0;
    int k_max = 0;
    std::vector<int64_t> off;      // B + 1 point offsets
    std::vector<int32_t> k;        // per cloud
    std::vector<int32_t> seq;      // processing order of the clouds
    // device memory: one block of small arrays, the float4 copy of the points
    void *dsmall = nullptr;
    float4 *xyz4 = nullptr;
    int64_t *d_pt_off = nullptr;   // B + 1
    int64_t *d_idx_off = nullptr;  // B + 1
    int32_t *d_k = nullptr;        // B
    int32_t *d_seq = nullptr;      // B
    int32_t *d_tile_off = nullptr; // B + 1, in processing order
    unsigned *d_counter = nullptr;
    // launch shape
    int lanes = 1, threads = 128, rounds = 1;
    int ntiles = 0;
    // captured graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_kernels = 0;
    // autotuner record: (lanes, threads, rounds, ms)
    std::vector<int32_t> tune_cfg;
    std::vector<float> tune_ms;
};

namespace mls {

namespace {

constexpr int kBatchMaxThreads = 256;

struct BatchArgs {
    const float4 *xyz4;
    const int32_t *idx;
    const int32_t *order;
    const float *h;
    const int64_t *pt_off;
    const int64_t *idx_off;
    const int32_t *k;
    const int32_t *seq;
    const int32_t *tile_off;
    unsigned *counter;
    float *out_xyz;
    float *out_n;
    uint8_t *status;
    int B;
    int ntiles;
    int G;
    int tile_pts;
    int k_max;
};

__global__ void k_batch_pack(const float *__restrict__ xyz, int64_t n, float4 *__restrict__ xyz4) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        xyz4[i] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], 0.f);
}

template <int DEG, int PREC>
__global__ void __launch_bounds__(kBatchMaxThreads, 4) k_project_batched(BatchArgs a) {
    extern __shared__ int32_t rows[];
    __shared__ int s_tile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int G = a.G;
    const int sub = lane & (G - 1);
    const int grp = threadIdx.x / G;
    const int ppr = blockDim.x / G;
    int32_t *my_rows = rows + warp * a.k_max * kRowStride;
    for (;;) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(a.counter, 1u);
        __syncthreads();
        const int t = s_tile;
        __syncthreads();
        if (t >= a.ntiles) return;
        // the cloud holding tile t: last c with tile_off[c] <= t
        int lo = 0, hi = a.B;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(a.tile_off + mid) <= t) lo = mid;
            else hi = mid;
        }
        const int b = __ldg(a.seq + lo);
        const int64_t p0 = __ldg(a.pt_off + b);
        const int64_t nb = __ldg(a.pt_off + b + 1) - p0;
        const int k = __ldg(a.k + b);
        const float h = __ldg(a.h + b);
        const int64_t start = (int64_t)(t - __ldg(a.tile_off + lo)) * a.tile_pts;
        const int64_t end = min(start + (int64_t)a.tile_pts, nb);
        const float4 *x4 = a.xyz4 + p0;
        const int32_t *idx = a.idx + __ldg(a.idx_off + b);
        const int32_t *ord = a.order ? a.order + p0 : nullptr;
        for (int64_t base = start; base < end; base += ppr) {
            float out[3], nf[3];
            uint8_t st;
            int64_t i;
            bool write;
            if (G == 1) {
                // one lane per point; the warp's 32 rows staged transposed
                // in shared memory with coalesced loads
                const int64_t wbase = base + warp * 32;
                if (wbase >= end) continue;
                const int64_t slot = wbase + lane;
                i = slot < end ? (ord ? (int64_t)__ldg(ord + slot) : slot) : -1;
                const int nrows = (int)min((int64_t)32, end - wbase);
                __syncwarp();
#pragma unroll 8
                for (int r = 0; r < 32; ++r) {
                    const int64_t i_r = __shfl_sync(0xffffffffu, i, r);
                    if (r < nrows)
                        for (int c = lane; c < k; c += 32) my_rows[c * kRowStride + r] = __ldg(idx + i_r * k + c);
                }
                __syncwarp();
                if (slot >= end) continue;
                const float4 r4 = __ldg(x4 + i);
                st = project_point<DEG, PREC>(
                    x4, [&](int j) { return my_rows[j * kRowStride + lane]; }, k, 0, 1, h, r4.x, r4.y, r4.z, out, nf);
                write = true;
            } else {
                // G lanes per point: the whole warp runs the shuffles, lanes
                // past the tile's end work on its last point and write nothing
                if (base + (warp * 32) / G >= end) continue;
                const int64_t slot = base + grp;
                write = slot < end && sub == 0;
                const int64_t sc = slot < end ? slot : end - 1;
                i = ord ? (int64_t)__ldg(ord + sc) : sc;
                const int32_t *row = idx + i * k;
                const float4 r4 = __ldg(x4 + i);
                st = project_point<DEG, PREC>(
                    x4, [&](int j) { return __ldg(row + j); }, k, sub, G, h, r4.x, r4.y, r4.z, out, nf);
            }
            if (write) {
                const int64_t o = p0 + i;
                a.out_xyz[3 * o] = out[0];
                a.out_xyz[3 * o + 1] = out[1];
                a.out_xyz[3 * o + 2] = out[2];
                if (a.out_n) {
                    a.out_n[3 * o] = nf[0];
                    a.out_n[3 * o + 1] = nf[1];
                    a.out_n[3 * o + 2] = nf[2];
                }
                if (a.status) a.status[o] = st;
            }
        }
    }
}

using BatchKernel = void (*)(BatchArgs);

BatchKernel batch_kernel(int degree, int precision) {
    const bool mixed = precision == MLS_PREC_MIXED;
    switch (degree) {
        case 0:
            return mixed ? k_project_batched<0, MLS_PREC_MIXED> : k_project_batched<0, MLS_PREC_FP32>;
        case 1:
            return mixed ? k_project_batched<1, MLS_PREC_MIXED> : k_project_batched<1, MLS_PREC_FP32>;
        default:
            return mixed ? k_project_batched<2, MLS_PREC_MIXED> : k_project_batched<2, MLS_PREC_FP32>;
    }
}

bool valid_shape(int lanes, int threads, int rounds) {
    if (lanes < 1 || lanes > 32 || (lanes & (lanes - 1))) return false;
    if (threads < 32 || threads > kBatchMaxThreads || threads % 32) return false;
    return rounds >= 1 && rounds <= 64;
}

size_t batch_smem(const mls_batch *b) {
    return b->lanes == 1 ? (size_t)b->k_max * kRowStride * sizeof(int32_t) * (b->threads / 32) : 0;
}

// Tile offsets for the current shape, uploaded synchronously.
int set_shape(mls_batch *b, int lanes, int threads, int rounds) {
    const int64_t tile_pts = (int64_t)(threads / lanes) * rounds;
    std::vector<int32_t> tile_off(b->B + 1, 0);
    int64_t acc = 0;
    for (int c = 0; c < b->B; ++c) {
        tile_off[c] = (int32_t)acc;
        const int cl = b->seq[c];
        acc += (b->off[cl + 1] - b->off[cl] + tile_pts - 1) / tile_pts;
    }
    tile_off[b->B] = (int32_t)acc;
    if (acc > 0x7fffffffLL) return set_error(MLS_ERR_TOO_LARGE, "mls_batch: %lld tiles", (long long)acc);
    MLS_CUDA_TRY(cudaMemcpy(b->d_tile_off, tile_off.data(), tile_off.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice));
    b->lanes = lanes;
    b->threads = threads;
    b->rounds = rounds;
    b->ntiles = (int)acc;
    return MLS_OK;
}

int check_launch(const mls_batch *b, const float *xyz, const int32_t *idx, const float *h, int degree,
                 int precision, const float *out_xyz, const char *fn) {
    if (!b) return set_error(MLS_ERR_INVALID_ARG, "%s: null batch", fn);
    if (!xyz || !idx || !h || !out_xyz) return set_error(MLS_ERR_INVALID_ARG, "%s: null pointer", fn);
    if (degree < 0 || degree > 2)
        return set_error(MLS_ERR_UNSUPPORTED_DEGREE, "%s: degree = %d not in {0, 1, 2}", fn, degree);
    if (precision != MLS_PREC_FP32 && precision != MLS_PREC_MIXED)
        return set_error(MLS_ERR_INVALID_ARG, "%s: precision = %d (FP32 or mixed)", fn, precision);
    if ((const void *)out_xyz == (const void *)xyz) return set_error(MLS_ERR_INVALID_ARG, "%s: output aliases the input", fn);
    return MLS_OK;
}

int batch_launch(mls_batch *b, const float *xyz, const int32_t *idx, const int32_t *order, const float *h,
                 int degree, int precision, float *out_xyz, float *out_n, uint8_t *status, cudaStream_t st) {
    const BatchKernel kern = batch_kernel(degree, precision);
    const size_t smem = batch_smem(b);
    MLS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    MLS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, b->threads, smem));
    if (per_sm < 1) return set_error(MLS_ERR_INVALID_ARG, "mls_project_batched: shape does not fit an SM");
    const int blocks = (int)std::min<int64_t>((int64_t)b->sms * per_sm, std::max(b->ntiles, 1));
    MLS_CUDA_TRY(cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned), st));
    k_batch_pack<<<(int)std::min<int64_t>((b->total + 255) / 256, (int64_t)b->sms * 16), 256, 0, st>>>(
        xyz, b->total, b->xyz4);
    BatchArgs a;
    a.xyz4 = b->xyz4;
    a.idx = idx;
    a.order = order;
    a.h = h;
    a.pt_off = b->d_pt_off;
    a.idx_off = b->d_idx_off;
    a.k = b->d_k;
    a.seq = b->d_seq;
    a.tile_off = b->d_tile_off;
    a.counter = b->d_counter;
    a.out_xyz = out_xyz;
    a.out_n = out_n;
    a.status = status;
    a.B = b->B;
    a.ntiles = b->ntiles;
    a.G = b->lanes;
    a.tile_pts = (b->threads / b->lanes) * b->rounds;
    a.k_max = b->k_max;
    kern<<<blocks, b->threads, smem, st>>>(a);
    count_launches(2);
    MLS_CUDA_TRY(cudaGetLastError());
    return MLS_OK;
}

void drop_graph(mls_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_kernels = 0;
}

// Candidate launch shapes of the autotuner: lanes per point x threads per
// block x rounds per tile.
constexpr int kTuneLanes[] = {1, 2, 4, 8};
constexpr int kTuneThreads[] = {64, 128, 256};
constexpr int kTuneRounds[] = {1, 4};

}  // namespace

}  // namespace mls

extern "C" {

int mls_batch_create(int batch, const int64_t *h_offsets, const int32_t *h_k, mls_batch **out) {
    using mls::set_error;
    if (!out) return set_error(MLS_ERR_INVALID_ARG, "mls_batch_create: null out");
    *out = nullptr;
    if (batch < 1 || !h_offsets || !h_k)
        return set_error(MLS_ERR_INVALID_ARG, "mls_batch_create: batch = %d, offsets and k required", batch);
    if (h_offsets[0] != 0) return set_error(MLS_ERR_INVALID_ARG, "mls_batch_create: offsets[0] = %lld != 0",
                                            (long long)h_offsets[0]);
    int k_max = 0;
    for (int c = 0; c < batch; ++c) {
        const int64_t n = h_offsets[c + 1] - h_offsets[c];
        if (n < 1) return set_error(MLS_ERR_INVALID_ARG, "mls_batch_create: cloud %d has %lld points", c, (long long)n);
        if (n > 0x7fffffffLL) return set_error(MLS_ERR_TOO_LARGE, "mls_batch_create: cloud %d has %lld points", c,
                                               (long long)n);
        if (h_k[c] < 1 || h_k[c] > MLS_MAX_K || h_k[c] > n)
            return set_error(MLS_ERR_K_TOO_LARGE, "mls_batch_create: cloud %d: k = %d not in [1, min(%d, n)]", c,
                             h_k[c], MLS_MAX_K);
        k_max = std::max(k_max, (int)h_k[c]);
    }
    const int64_t total = h_offsets[batch];
    if (total > 0x7fffffffLL) return set_error(MLS_ERR_TOO_LARGE, "mls_batch_create: %lld points in all",
                                               (long long)total);
    mls_batch *b = new mls_batch();
    b->B = batch;
    b->total = total;
    b->k_max = k_max;
    b->off.assign(h_offsets, h_offsets + batch + 1);
    b->k.assign(h_k, h_k + batch);
    b->seq.resize(batch);
    std::iota(b->seq.begin(), b->seq.end(), 0);
    std::stable_sort(b->seq.begin(), b->seq.end(), [b](int x, int y) {
        if (b->k[x] != b->k[y]) return b->k[x] > b->k[y];
        return b->off[x + 1] - b->off[x] > b->off[y + 1] - b->off[y];
    });
    std::vector<int64_t> idx_off(batch + 1, 0);
    for (int c = 0; c < batch; ++c) idx_off[c + 1] = idx_off[c] + (b->off[c + 1] - b->off[c]) * b->k[c];
    auto fail = [b](int rc) {
        mls_batch_destroy(b);
        return rc;
    };
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    const size_t bytes = (size_t)(batch + 1) * 16 + (size_t)batch * 8 + (size_t)(batch + 1) * 4 + 64;
    if (e == cudaSuccess) e = cudaMalloc(&b->dsmall, bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->xyz4, (size_t)total * sizeof(float4));
    if (e != cudaSuccess)
        return fail(set_error(e == cudaErrorMemoryAllocation ? MLS_ERR_OOM : MLS_ERR_CUDA, "mls_batch_create: %s",
                              cudaGetErrorString(e)));
    char *p = (char *)b->dsmall;
    b->d_pt_off = (int64_t *)p;
    p += (size_t)(batch + 1) * 8;
    b->d_idx_off = (int64_t *)p;
    p += (size_t)(batch + 1) * 8;
    b->d_k = (int32_t *)p;
    p += (size_t)batch * 4;
    b->d_seq = (int32_t *)p;
    p += (size_t)batch * 4;
    b->d_tile_off = (int32_t *)p;
    p += (size_t)(batch + 1) * 4;
    b->d_counter = (unsigned *)(((uintptr_t)p + 15) & ~(uintptr_t)15);
    e = cudaMemcpy(b->d_pt_off, b->off.data(), (batch + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_idx_off, idx_off.data(), (batch + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_k, b->k.data(), batch * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_seq, b->seq.data(), batch * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(set_error(MLS_ERR_CUDA, "mls_batch_create: %s", cudaGetErrorString(e)));
    const int rc = mls::set_shape(b, 1, 128, 1);
    if (rc != MLS_OK) return fail(rc);
    *out = b;
    return MLS_OK;
}

void mls_batch_destroy(mls_batch *b) {
    if (!b) return;
    cudaDeviceSynchronize();
    mls::drop_graph(b);
    if (b->xyz4) cudaFree(b->xyz4);
    if (b->dsmall) cudaFree(b->dsmall);
    delete b;
}

int64_t mls_batch_total(const mls_batch *b) { return b ? b->total : -1; }

int64_t mls_batch_idx_offset(const mls_batch *b, int cloud) {
    if (!b || cloud < 0 || cloud > b->B) return -1;
    int64_t acc = 0;
    for (int c = 0; c < cloud; ++c) acc += (b->off[c + 1] - b->off[c]) * b->k[c];
    return acc;
}

int mls_batch_set_shape(mls_batch *b, int lanes_per_point, int threads, int rounds) {
    if (!b) return mls::set_error(MLS_ERR_INVALID_ARG, "mls_batch_set_shape: null batch");
    if (!mls::valid_shape(lanes_per_point, threads, rounds))
        return mls::set_error(MLS_ERR_INVALID_ARG, "mls_batch_set_shape: lanes %d, threads %d, rounds %d",
                              lanes_per_point, threads, rounds);
    if (lanes_per_point == b->lanes && threads == b->threads && rounds == b->rounds) return MLS_OK;
    mls::drop_graph(b);
    return mls::set_shape(b, lanes_per_point, threads, rounds);
}

int mls_batch_get_shape(const mls_batch *b, int *lanes_per_point, int *threads, int *rounds) {
    if (!b || !lanes_per_point || !threads || !rounds)
        return mls::set_error(MLS_ERR_INVALID_ARG, "mls_batch_get_shape: null argument");
    *lanes_per_point = b->lanes;
    *threads = b->threads;
    *rounds = b->rounds;
    return MLS_OK;
}

int mls_project_batched(mls_batch *b, const float *d_xyz, const int32_t *d_idx, const int32_t *d_order,
                        const float *d_h, int degree, int precision, float *d_out_xyz, float *d_out_normal,
                        uint8_t *d_status, mls_stream stream) {
    const int rc = mls::check_launch(b, d_xyz, d_idx, d_h, degree, precision, d_out_xyz, "mls_project_batched");
    if (rc != MLS_OK) return rc;
    return mls::batch_launch(b, d_xyz, d_idx, d_order, d_h, degree, precision, d_out_xyz, d_out_normal, d_status,
                             (cudaStream_t)stream);
}

int mls_batch_capture(mls_batch *b, const float *d_xyz, const int32_t *d_idx, const int32_t *d_order,
                      const float *d_h, int degree, int precision, float *d_out_xyz, float *d_out_normal,
                      uint8_t *d_status) {
    int rc = mls::check_launch(b, d_xyz, d_idx, d_h, degree, precision, d_out_xyz, "mls_batch_capture");
    if (rc != MLS_OK) return rc;
    mls::drop_graph(b);
    cudaStream_t cs = nullptr;
    MLS_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return mls::set_error(MLS_ERR_CUDA, "mls_batch_capture: %s", cudaGetErrorString(e));
    }
    const int64_t before = mls_kernel_launches();
    rc = mls::batch_launch(b, d_xyz, d_idx, d_order, d_h, degree, precision, d_out_xyz, d_out_normal, d_status, cs);
    const int kernels = (int)(mls_kernel_launches() - before);
    mls::count_launches(-kernels);            // captured, not run
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (rc != MLS_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return rc != MLS_OK ? rc : mls::set_error(MLS_ERR_CUDA, "mls_batch_capture: %s", cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        b->exec = nullptr;
        return mls::set_error(MLS_ERR_CUDA, "mls_batch_capture: instantiate: %s", cudaGetErrorString(e));
    }
    b->graph = g;
    b->graph_kernels = kernels;
    return MLS_OK;
}

int mls_batch_replay(mls_batch *b, mls_stream stream) {
    if (!b || !b->exec) return mls::set_error(MLS_ERR_INVALID_ARG, "mls_batch_replay: nothing captured");
    MLS_CUDA_TRY(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    mls::count_launches(b->graph_kernels);
    return MLS_OK;
}

int mls_batch_autotune(mls_batch *b, const float *d_xyz, const int32_t *d_idx, const int32_t *d_order,
                       const float *d_h, int degree, int precision, float *d_out_xyz, float *d_out_normal,
                       uint8_t *d_status, int reps, mls_stream stream) {
    int rc = mls::check_launch(b, d_xyz, d_idx, d_h, degree, precision, d_out_xyz, "mls_batch_autotune");
    if (rc != MLS_OK) return rc;
    if (reps < 1 || reps > 100) return mls::set_error(MLS_ERR_INVALID_ARG, "mls_batch_autotune: reps = %d", reps);
    cudaStream_t st = (cudaStream_t)stream;
    mls::drop_graph(b);
    b->tune_cfg.clear();
    b->tune_ms.clear();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MLS_CUDA_TRY(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return mls::set_error(MLS_ERR_CUDA, "mls_batch_autotune: %s", cudaGetErrorString(ce));
    }
    float best = INFINITY;
    int best_cfg[3] = {1, 128, 1};
    for (int G : mls::kTuneLanes)
        for (int T : mls::kTuneThreads)
            for (int R : mls::kTuneRounds) {
                if (rc != MLS_OK) break;
                rc = mls::set_shape(b, G, T, R);
                // one untimed run, then the fastest of `reps`
                float cfg_ms = INFINITY;
                for (int r = 0; rc == MLS_OK && r <= reps; ++r) {
                    if (r > 0 && cudaEventRecord(e0, st) != cudaSuccess) {
                        rc = mls::set_error(MLS_ERR_CUDA, "mls_batch_autotune: event record failed");
                        break;
                    }
                    rc = mls::batch_launch(b, d_xyz, d_idx, d_order, d_h, degree, precision, d_out_xyz,
                                           d_out_normal, d_status, st);
                    if (rc != MLS_OK || r == 0) continue;
                    float ms = 0.f;
                    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                        rc = mls::set_error(MLS_ERR_CUDA, "mls_batch_autotune: event timing failed");
                        break;
                    }
                    cfg_ms = std::min(cfg_ms, ms);
                }
                if (rc != MLS_OK) break;
                b->tune_cfg.insert(b->tune_cfg.end(), {G, T, R});
                b->tune_ms.push_back(cfg_ms);
                if (cfg_ms < best) {
                    best = cfg_ms;
                    best_cfg[0] = G;
                    best_cfg[1] = T;
                    best_cfg[2] = R;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != MLS_OK) return rc;
    rc = mls::set_shape(b, best_cfg[0], best_cfg[1], best_cfg[2]);
    if (rc != MLS_OK) return rc;
    // leave the outputs of the chosen shape in place
    return mls::batch_launch(b, d_xyz, d_idx, d_order, d_h, degree, precision, d_out_xyz, d_out_normal, d_status, st);
}

int mls_batch_tune_results(const mls_batch *b, int capacity, int32_t *shapes, float *ms) {
    if (!b) return mls::set_error(MLS_ERR_INVALID_ARG, "mls_batch_tune_results: null batch");
    const int n = (int)b->tune_ms.size();
    for (int i = 0; i < std::min(n, capacity); ++i) {
        if (shapes) std::memcpy(shapes + 3 * i, b->tune_cfg.data() + 3 * i, 3 * sizeof(int32_t));
        if (ms) ms[i] = b->tune_ms[i];
    }
    return n;
}

}  // extern "C"
