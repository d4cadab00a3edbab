// C ABI of libmls: argument validation, the grid handle, error reporting.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>

#include "grid.cuh"

namespace mls {

int build_grid(mls_grid *g, const float *xyz, int64_t n, float cell_size, int k_hint, cudaStream_t st);
void free_grid_buffers(mls_grid *g);
int launch_knn(const mls_grid *grid, int k, int32_t *idx, float *key, int32_t *pos, cudaStream_t st);
int launch_project_sorted(const float4 *pts, int64_t n, const int32_t *pos, int k, float h, int degree,
                          int precision, float *out_xyz, float *out_n, uint8_t *status, float *state,
                          cudaStream_t st);
int launch_knn_project_sorted(const mls_grid *g, int k, float h, int degree, int precision, int32_t *pos,
                              float *out_xyz, float *out_n, uint8_t *status, float *state, int32_t *offsets,
                              cudaStream_t st);
int launch_knn_project(const mls_grid *grid, int k, float h, int degree, int precision, float *out_xyz,
                       float *out_n, uint8_t *status, int32_t *pos, cudaStream_t st);
int launch_points_in_boxes(const mls_grid *grid, const float *boxes, int64_t m, uint8_t *mask, cudaStream_t st);
int launch_backward_sorted(const float4 *pts, const int32_t *order, int64_t n, const int32_t *rows, int k, float h,
                           int degree, int precision, const float *gp, const float *gn, float *grad_xyz,
                           float *grad_h, const float *state, const int32_t *offsets, cudaStream_t st);
int launch_project(const float *xyz, int64_t n, const int32_t *idx, int k, float h, int degree, int precision,
                   const int32_t *order, float *out_xyz, float *out_n, uint8_t *status, cudaStream_t st);
int launch_radius(const mls_grid *grid, float R2, int32_t *count, const int64_t *offsets, int32_t *rows,
                  float *keys, int *overflow, cudaStream_t st);
int launch_project_rows(const float *xyz, int64_t n, const int64_t *off, const int32_t *rows, float h, int degree,
                        int precision, int min_nb, const int32_t *order, float *out_xyz, float *out_n,
                        uint8_t *status, cudaStream_t st);
int device_exclusive_scan64(const int32_t *in, int64_t *out, int64_t n, cudaStream_t st);
int device_compact(const uint8_t *status, int64_t n, int mask, int32_t *kept, int64_t *num, cudaStream_t st);
int launch_project_levin(const float *xyz, int64_t n, const int32_t *idx, int k, float h, int degree,
                         int precision, int max_iter, float tol, const int32_t *order, float *out_xyz,
                         float *out_n, uint8_t *status, cudaStream_t st);
int launch_backward(const float *xyz, int64_t n, const int32_t *idx, int k, float h, int degree, int precision,
                    const int32_t *order, const float *gp, const float *gn, float *grad_xyz, float *grad_h,
                    cudaStream_t st);

namespace {
thread_local char g_last_error[512] = "";
std::atomic<int64_t> g_launches{0};

// Mean neighbour distance excluding self, accumulated in FP64 in a fixed
// order (a grid-stride loop of a fixed grid, then fixed trees), so the
// result does not change from run to run.  The grid is a constant, not a
// multiple of the device's SM count, so that the summation order, and with
// it the result, is also the same on every device.
constexpr int kMeanBlocks = 1216;
constexpr int kMeanThreads = 256;

__global__ void __launch_bounds__(kMeanThreads) k_mean_dist(const float *__restrict__ xyz, int64_t n,
                                                            const int32_t *__restrict__ idx, int k,
                                                            double *__restrict__ part_sum,
                                                            unsigned long long *__restrict__ part_cnt) {
    __shared__ double ssum[kMeanThreads / 32];
    __shared__ unsigned long long scnt[kMeanThreads / 32];
    double sum = 0.0;
    unsigned long long cnt = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * k;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / k, j = idx[e];
        if (j == i) continue;
        double d2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            double d = (double)xyz[3 * j + a] - (double)xyz[3 * i + a];
            d2 += d * d;
        }
        sum += sqrt(d2);
        ++cnt;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) {
        ssum[threadIdx.x >> 5] = sum;
        scnt[threadIdx.x >> 5] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        unsigned long long c = 0;
        for (int w = 0; w < kMeanThreads / 32; ++w) {
            t += ssum[w];
            c += scnt[w];
        }
        part_sum[blockIdx.x] = t;
        part_cnt[blockIdx.x] = c;
    }
}

__global__ void __launch_bounds__(1024) k_mean_finish(const double *__restrict__ part_sum,
                                                      const unsigned long long *__restrict__ part_cnt,
                                                      double *__restrict__ out) {
    __shared__ double red[1024];
    __shared__ unsigned long long redc[1024];
    double t = 0.0;
    unsigned long long c = 0;
    for (int b = threadIdx.x; b < kMeanBlocks; b += 1024) {
        t += part_sum[b];
        c += part_cnt[b];
    }
    red[threadIdx.x] = t;
    redc[threadIdx.x] = c;
    __syncthreads();
    for (int s = 512; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red[threadIdx.x] += red[threadIdx.x + s];
            redc[threadIdx.x] += redc[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = redc[0] ? red[0] / (double)redc[0] : 0.0;
}

}  // namespace

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void clear_error() { g_last_error[0] = 0; }

int set_error(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
    return code;
}

}  // namespace mls

using mls::set_error;

extern "C" {

const char *mls_last_error(void) { return mls::g_last_error; }

int64_t mls_kernel_launches(void) { return mls::g_launches.load(std::memory_order_relaxed); }

const char *mls_status_str(int code) {
    switch (code) {
        case MLS_OK: return "ok";
        case MLS_ERR_INVALID_ARG: return "invalid argument";
        case MLS_ERR_K_TOO_LARGE: return "k too large";
        case MLS_ERR_UNSUPPORTED_DEGREE: return "unsupported degree";
        case MLS_ERR_CUDA: return "CUDA error";
        case MLS_ERR_OOM: return "out of device memory";
        case MLS_ERR_TIMEOUT: return "device wait timed out";
        case MLS_ERR_NONFINITE: return "non-finite coordinate";
        case MLS_ERR_TOO_LARGE: return "too many points";
        default: return "unknown status";
    }
}

int mls_build_grid(const float *d_xyz, int64_t n, float cell_size, int k_hint, mls_stream stream,
                   mls_grid **inout) {
    mls::g_last_error[0] = 0;
    if (!d_xyz || !inout) return set_error(MLS_ERR_INVALID_ARG, "mls_build_grid: null pointer");
    if (n < 1) return set_error(MLS_ERR_INVALID_ARG, "mls_build_grid: n = %lld < 1", (long long)n);
    if (n > 0x7fffffffLL) return set_error(MLS_ERR_TOO_LARGE, "mls_build_grid: n = %lld", (long long)n);
    if (k_hint < 1 || k_hint > MLS_MAX_K)
        return set_error(MLS_ERR_K_TOO_LARGE, "mls_build_grid: k_hint = %d not in [1, %d]", k_hint, MLS_MAX_K);
    if (std::isnan(cell_size)) return set_error(MLS_ERR_INVALID_ARG, "mls_build_grid: cell_size is NaN");
    mls_grid *g = *inout;
    bool fresh = false;
    if (!g) {
        g = new (std::nothrow) mls_grid();
        if (!g) return set_error(MLS_ERR_OOM, "mls_build_grid: host allocation failed");
        fresh = true;
        cudaGetDevice(&g->device);
    }
    int rc = mls::build_grid(g, d_xyz, n, cell_size, k_hint, (cudaStream_t)stream);
    if (rc != MLS_OK) {
        if (fresh) {
            mls::free_grid_buffers(g);
            delete g;
        } else {
            g->n = 0;   // unusable until rebuilt
        }
        return rc;
    }
    *inout = g;
    return MLS_OK;
}

void mls_grid_destroy(mls_grid *g) {
    if (!g) return;
    if (g->stream) cudaStreamSynchronize(g->stream);
    mls::free_grid_buffers(g);
    delete g;
}

int64_t mls_grid_size(const mls_grid *g) { return g ? g->n : -1; }

const int32_t *mls_grid_order(const mls_grid *g) { return g && g->n > 0 ? g->perm : nullptr; }

int mls_knn(const mls_grid *g, int k, int32_t *d_idx, float *d_key, mls_stream stream) {
    mls::g_last_error[0] = 0;
    if (!g || !d_idx) return set_error(MLS_ERR_INVALID_ARG, "mls_knn: null pointer");
    if (g->n < 1) return set_error(MLS_ERR_INVALID_ARG, "mls_knn: grid is empty (failed build?)");
    if (k < 1 || k > MLS_MAX_K || k > g->n)
        return set_error(MLS_ERR_K_TOO_LARGE, "mls_knn: k = %d not in [1, min(%d, n = %lld)]", k, MLS_MAX_K,
                         (long long)g->n);
    return mls::launch_knn(g, k, d_idx, d_key, nullptr, (cudaStream_t)stream);
}

int mls_knn_sorted(const mls_grid *g, int k, int32_t *d_pos, int32_t *d_idx, float *d_key, mls_stream stream) {
    mls::g_last_error[0] = 0;
    if (!g || !d_pos) return set_error(MLS_ERR_INVALID_ARG, "mls_knn_sorted: null pointer");
    if (g->n < 1) return set_error(MLS_ERR_INVALID_ARG, "mls_knn_sorted: grid is empty (failed build?)");
    if (k < 1 || k > MLS_MAX_K || k > g->n)
        return set_error(MLS_ERR_K_TOO_LARGE, "mls_knn_sorted: k = %d not in [1, min(%d, n = %lld)]", k, MLS_MAX_K,
                         (long long)g->n);
    return mls::launch_knn(g, k, d_idx, d_key, d_pos, (cudaStream_t)stream);
}

int mls_project_sorted(const mls_grid *g, const int32_t *d_pos, int k, float h, int degree, int precision,
                       float *d_out_xyz, float *d_out_normal, uint8_t *d_status, float *d_state,
                       mls_stream stream) {
    mls::g_last_error[0] = 0;
    if (!g || !d_pos || !d_out_xyz) return set_error(MLS_ERR_INVALID_ARG, "mls_project_sorted: null pointer");
    if (g->n < 1) return set_error(MLS_ERR_INVALID_ARG, "mls_project_sorted: grid is empty (failed build?)");
    if (k < 1 || k > MLS_MAX_K || k > g->n)
        return set_error(MLS_ERR_K_TOO_LARGE, "mls_project_sorted: k = %d not in [1, min(%d, n)]", k, MLS_MAX_K);
    if (!(h > 0.0f) || !std::isfinite(h))
        return set_error(MLS_ERR_INVALID_ARG, "mls_project_sorted: h = %g must be finite and > 0", (double)h);
    if (degree < 0 || degree > 2)
        return set_error(MLS_ERR_UNSUPPORTED_DEGREE, "mls_project_sorted: degree = %d not in {0, 1, 2}", degree);
    if (precision != MLS_PREC_FP32 && precision != MLS_PREC_MIXED)
        return set_error(MLS_ERR_INVALID_ARG, "mls_project_sorted: precision = %d (FP32 or mixed)", precision);
    if ((const void *)d_out_xyz == (const void *)g->xyz)
        return set_error(MLS_ERR_INVALID_ARG, "mls_project_sorted: output aliases the grid's points");
    return mls::launch_project_sorted(g->view.pts, g->n, d_pos, k, h, degree, precision, d_out_xyz, d_out_normal,
                                      d_status, d_state, (cudaStream_t)stream);
}

int mls_knn_project(const mls_grid *g, int k, float h, int degree, int precision, float *d_out_xyz,
                    float *d_out_normal, uint8_t *d_status, int32_t *d_pos, mls_stream stream) {
    mls::g_last_error[0] = 0;
    if (!g || !d_out_xyz) return set_error(MLS_ERR_INVALID_ARG, "mls_knn_project: null pointer");
    if (g->n < 1) return set_error(MLS_ERR_INVALID_ARG, "mls_knn_project: grid is empty (failed build?)");
    if (k < 1 || k > MLS_MAX_K_FUSED || k > g->n)
        return set_error(MLS_ERR_K_TOO_LARGE, "mls_knn_project: k = %d not in [1, min(%d, n = %lld)]", k,
                         MLS_MAX_K_FUSED, (long long)g->n);
    if (!(h > 0.0f) || !std::isfinite(h))
        return set_error(MLS_ERR_INVALID_ARG, "mls_knn_project: h = %g must be finite and > 0", (double)h);
    if (degree < 0 || degree > 2)
        return set_error(MLS_ERR_UNSUPPORTED_DEGREE, "mls_knn_project: degree = %d not in {0, 1, 2}", degree);
    if (precision != MLS_PREC_FP32 && precision != MLS_PREC_MIXED)
        return set_error(MLS_ERR_INVALID_ARG, "mls_knn_project: precision = %d (FP32 or mixed)", precision);
    if ((const void *)d_out_xyz == (const void *)g->xyz)
        return set_error(MLS_ERR_INVALID_ARG, "mls_knn_project: output aliases the grid's points");
    return mls::launch_knn_project(g, k, h, degree, precision, d_out_xyz, d_out_normal, d_status, d_pos,
                                   (cudaStream_t)stream);
}

int mls_knn_project_sorted(const mls_grid *g, int k, float h, int degree, int precision, int32_t *d_pos,
                           float *d_out_xyz, float *d_out_normal, uint8_t *d_status, float *d_state,
                           int32_t *d_offsets, mls_stream stream) {
    mls::g_last_error[0] = 0;
    if (!g || !d_pos || !d_out_xyz) return set_error(MLS_ERR_INVALID_ARG, "mls_knn_project_sorted: null pointer");
    if (g->n < 1) return set_error(MLS_ERR_INVALID_ARG, "mls_knn_project_sorted: grid is empty (failed build?)");
    if (k < 1 || k > MLS_MAX_K || k > g->n)
        return set_error(MLS_ERR_K_TOO_LARGE, "mls_knn_project_sorted: k = %d not in [1, min(%d, n = %lld)]", k,
                         MLS_MAX_K, (long long)g->n);
    if (!(h > 0.0f) || !std::isfinite(h))
        return set_error(MLS_ERR_INVALID_ARG, "mls_knn_project_sorted: h = %g must be finite and > 0", (double)h);
    if (degree < 0 || degree > 2)
        return set_error(MLS_ERR_UNSUPPORTED_DEGREE, "mls_knn_project_sorted: degree = %d not in {0, 1, 2}", degree);
    if (precision != MLS_PREC_FP32 && precision != MLS_PREC_MIXED)
        return set_error(MLS_ERR_INVALID_ARG, "mls_knn_project_sorted: precision = %d (FP32 or mixed)", precision);
    if ((const void *)d_out_xyz == (const void *)g->xyz)
        return set_error(MLS_ERR_INVALID_ARG, "mls_knn_project_sorted: output aliases the grid's points");
    if (d_offsets && g->n > 0x7fffffffLL / MLS_MAX_K)
        return set_error(MLS_ERR_TOO_LARGE, "mls_knn_project_sorted: n = %lld too large for the offsets",
                         (long long)g->n);
    return mls::launch_knn_project_sorted(g, k, h, degree, precision, d_pos, d_out_xyz, d_out_normal, d_status,
                                          d_state, d_offsets, (cudaStream_t)stream);
}

int64_t mls_knn_deferred(const mls_grid *g, mls_stream stream) {
    mls::g_last_error[0] = 0;
    if (!g || !g->work) return set_error(MLS_ERR_INVALID_ARG, "mls_knn_deferred: no kNN on this grid");
    int head[4] = {0, 0, 0, 0};
    cudaStream_t st = (cudaStream_t)stream;
    MLS_CUDA_TRY(cudaMemcpyAsync(head, g->work, sizeof(head), cudaMemcpyDeviceToHost, st));
    MLS_CUDA_TRY(cudaStreamSynchronize(st));
    return (int64_t)head[1] + head[3];     // handed to the second pass + isolated
}

int mls_project(const float *d_xyz, int64_t n, const int32_t *d_idx, int k, float h, int degree, int precision,
                const int32_t *d_order, float *d_out_xyz, float *d_out_normal, uint8_t *d_status,
                mls_stream stream) {
    mls::g_last_error[0] = 0;
    if (!d_xyz || !d_idx || !d_out_xyz) return set_error(MLS_ERR_INVALID_ARG, "mls_project: null pointer");
    if (n < 1) return set_error(MLS_ERR_INVALID_ARG, "mls_project: n = %lld < 1", (long long)n);
    if (n > 0x7fffffffLL) return set_error(MLS_ERR_TOO_LARGE, "mls_project: n = %lld", (long long)n);
    if (k < 1 || k > MLS_MAX_K || k > n)
        return set_error(MLS_ERR_K_TOO_LARGE, "mls_project: k = %d not in [1, min(%d, n)]", k, MLS_MAX_K);
    if (!(h > 0.0f) || !std::isfinite(h))
        return set_error(MLS_ERR_INVALID_ARG, "mls_project: h = %g must be finite and > 0", (double)h);
    if (degree < 0 || degree > 2)
        return set_error(MLS_ERR_UNSUPPORTED_DEGREE, "mls_project: degree = %d not in {0, 1, 2}", degree);
    if (precision < MLS_PREC_FP32 || precision > MLS_PREC_FP64)
        return set_error(MLS_ERR_INVALID_ARG, "mls_project: precision = %d", precision);
    if ((const void *)d_out_xyz == (const void *)d_xyz)
        return set_error(MLS_ERR_INVALID_ARG, "mls_project: output aliases the input");
    return mls::launch_project(d_xyz, n, d_idx, k, h, degree, precision, d_order, d_out_xyz, d_out_normal,
                               d_status, (cudaStream_t)stream);
}

static int check_radius(const mls_grid *g, float R, const char *fn) {
    if (!g || g->n < 1) return set_error(MLS_ERR_INVALID_ARG, "%s: empty or null grid", fn);
    if (!(R >= 0.0f) || !std::isfinite(R)) return set_error(MLS_ERR_INVALID_ARG, "%s: R = %g", fn, (double)R);
    return MLS_OK;
}

int mls_radius_count(const mls_grid *g, float R, int32_t *d_count, int64_t *d_offsets, mls_stream stream) {
    mls::g_last_error[0] = 0;
    int rc = check_radius(g, R, "mls_radius_count");
    if (rc != MLS_OK) return rc;
    if (!d_count) return set_error(MLS_ERR_INVALID_ARG, "mls_radius_count: null count");
    cudaStream_t st = (cudaStream_t)stream;
    rc = mls::launch_radius(g, R * R, d_count, nullptr, nullptr, nullptr, nullptr, st);
    if (rc != MLS_OK || !d_offsets) return rc;
    return mls::device_exclusive_scan64(d_count, d_offsets, g->n, st);
}

int mls_radius_rows(const mls_grid *g, float R, const int64_t *d_offsets, int32_t *d_rows, float *d_keys,
                    mls_stream stream) {
    mls::g_last_error[0] = 0;
    int rc = check_radius(g, R, "mls_radius_rows");
    if (rc != MLS_OK) return rc;
    if (!d_offsets || !d_rows) return set_error(MLS_ERR_INVALID_ARG, "mls_radius_rows: null pointer");
    cudaStream_t st = (cudaStream_t)stream;
    mls::ScratchSet scratch(st);
    int *overflow = nullptr;
    MLS_CUDA_TRY(scratch.alloc(&overflow, sizeof(int)));
    MLS_CUDA_TRY(cudaMemsetAsync(overflow, 0, sizeof(int), st));
    rc = mls::launch_radius(g, R * R, nullptr, d_offsets, d_rows, d_keys, overflow, st);
    int worst = 0;
    if (rc == MLS_OK) {
        cudaError_t e = cudaMemcpyAsync(&worst, overflow, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = set_error(MLS_ERR_CUDA, "mls_radius_rows: %s", cudaGetErrorString(e));
    }
    if (rc != MLS_OK) return rc;
    if (worst > 0)
        return set_error(MLS_ERR_K_TOO_LARGE, "mls_radius_rows: a neighbourhood holds %d points, more than %d",
                         worst, MLS_MAX_RADIUS_NB);
    return MLS_OK;
}

int mls_project_rows(const float *d_xyz, int64_t n, const int64_t *d_offsets, const int32_t *d_rows, float h,
                     int degree, int precision, int min_neighbors, const int32_t *d_order, float *d_out_xyz,
                     float *d_out_normal, uint8_t *d_status, mls_stream stream) {
    mls::g_last_error[0] = 0;
    if (!d_xyz || !d_offsets || !d_rows || !d_out_xyz)
        return set_error(MLS_ERR_INVALID_ARG, "mls_project_rows: null pointer");
    if (n < 1) return set_error(MLS_ERR_INVALID_ARG, "mls_project_rows: n = %lld < 1", (long long)n);
    if (n > 0x7fffffffLL) return set_error(MLS_ERR_TOO_LARGE, "mls_project_rows: n = %lld", (long long)n);
    if (!(h > 0.0f) || !std::isfinite(h))
        return set_error(MLS_ERR_INVALID_ARG, "mls_project_rows: h = %g must be finite and > 0", (double)h);
    if (degree < 0 || degree > 2)
        return set_error(MLS_ERR_UNSUPPORTED_DEGREE, "mls_project_rows: degree = %d not in {0, 1, 2}", degree);
    if (precision != MLS_PREC_FP32 && precision != MLS_PREC_MIXED)
        return set_error(MLS_ERR_INVALID_ARG, "mls_project_rows: precision = %d (FP32 or mixed)", precision);
    if (min_neighbors < 0) return set_error(MLS_ERR_INVALID_ARG, "mls_project_rows: min_neighbors = %d", min_neighbors);
    if ((const void *)d_out_xyz == (const void *)d_xyz)
        return set_error(MLS_ERR_INVALID_ARG, "mls_project_rows: output aliases the input");
    return mls::launch_project_rows(d_xyz, n, d_offsets, d_rows, h, degree, precision, min_neighbors, d_order,
                                    d_out_xyz, d_out_normal, d_status, (cudaStream_t)stream);
}

int mls_compact(const uint8_t *d_status, int64_t n, int mask, int32_t *d_kept, int64_t *d_num_kept,
                mls_stream stream) {
    mls::g_last_error[0] = 0;
    if (!d_status || !d_kept || !d_num_kept) return set_error(MLS_ERR_INVALID_ARG, "mls_compact: null pointer");
    if (n < 1 || n > 0x7fffffffLL) return set_error(MLS_ERR_INVALID_ARG, "mls_compact: n = %lld", (long long)n);
    return mls::device_compact(d_status, n, mask, d_kept, d_num_kept, (cudaStream_t)stream);
}

int mls_project_levin(const float *d_xyz, int64_t n, const int32_t *d_idx, int k, float h, int degree,
                      int precision, int max_iter, float tol, const int32_t *d_order, float *d_out_xyz,
                      float *d_out_normal, uint8_t *d_status, mls_stream stream) {
    mls::g_last_error[0] = 0;
    if (!d_xyz || !d_idx || !d_out_xyz) return set_error(MLS_ERR_INVALID_ARG, "mls_project_levin: null pointer");
    if (n < 1) return set_error(MLS_ERR_INVALID_ARG, "mls_project_levin: n = %lld < 1", (long long)n);
    if (n > 0x7fffffffLL) return set_error(MLS_ERR_TOO_LARGE, "mls_project_levin: n = %lld", (long long)n);
    if (k < 1 || k > MLS_MAX_K || k > n)
        return set_error(MLS_ERR_K_TOO_LARGE, "mls_project_levin: k = %d not in [1, min(%d, n)]", k, MLS_MAX_K);
    if (!(h > 0.0f) || !std::isfinite(h))
        return set_error(MLS_ERR_INVALID_ARG, "mls_project_levin: h = %g must be finite and > 0", (double)h);
    if (degree < 0 || degree > 2)
        return set_error(MLS_ERR_UNSUPPORTED_DEGREE, "mls_project_levin: degree = %d not in {0, 1, 2}", degree);
    if (precision != MLS_PREC_FP32 && precision != MLS_PREC_MIXED)
        return set_error(MLS_ERR_INVALID_ARG, "mls_project_levin: precision = %d (FP32 or mixed)", precision);
    if (max_iter < 1 || max_iter > 64)
        return set_error(MLS_ERR_INVALID_ARG, "mls_project_levin: max_iter = %d not in [1, 64]", max_iter);
    if (!(tol > 0.0f) || !std::isfinite(tol))
        return set_error(MLS_ERR_INVALID_ARG, "mls_project_levin: tol = %g must be finite and > 0", (double)tol);
    if ((const void *)d_out_xyz == (const void *)d_xyz)
        return set_error(MLS_ERR_INVALID_ARG, "mls_project_levin: output aliases the input");
    return mls::launch_project_levin(d_xyz, n, d_idx, k, h, degree, precision, max_iter, tol, d_order, d_out_xyz,
                                     d_out_normal, d_status, (cudaStream_t)stream);
}

int mls_project_backward(const float *d_xyz, int64_t n, const int32_t *d_idx, int k, float h, int degree,
                         int precision, const int32_t *d_order, const float *d_grad_out_xyz,
                         const float *d_grad_out_normal, float *d_grad_xyz, float *d_grad_h, mls_stream stream) {
    mls::g_last_error[0] = 0;
    if (!d_xyz || !d_idx || !d_grad_out_xyz || !d_grad_xyz || !d_grad_h)
        return set_error(MLS_ERR_INVALID_ARG, "mls_project_backward: null pointer");
    if (n < 1) return set_error(MLS_ERR_INVALID_ARG, "mls_project_backward: n = %lld < 1", (long long)n);
    if (n > 0x7fffffffLL / MLS_MAX_K)
        return set_error(MLS_ERR_TOO_LARGE, "mls_project_backward: n = %lld", (long long)n);
    if (k < 1 || k > MLS_MAX_K || k > n)
        return set_error(MLS_ERR_K_TOO_LARGE, "mls_project_backward: k = %d not in [1, min(%d, n)]", k, MLS_MAX_K);
    if (!(h > 0.0f) || !std::isfinite(h))
        return set_error(MLS_ERR_INVALID_ARG, "mls_project_backward: h = %g must be finite and > 0", (double)h);
    if (degree < 0 || degree > 2)
        return set_error(MLS_ERR_UNSUPPORTED_DEGREE, "mls_project_backward: degree = %d", degree);
    if (precision < MLS_PREC_FP32 || precision > MLS_PREC_FP64)
        return set_error(MLS_ERR_INVALID_ARG, "mls_project_backward: precision = %d", precision);
    if ((const void *)d_grad_xyz == (const void *)d_xyz || (const void *)d_grad_xyz == (const void *)d_grad_out_xyz)
        return set_error(MLS_ERR_INVALID_ARG, "mls_project_backward: output aliases an input");
    return mls::launch_backward(d_xyz, n, d_idx, k, h, degree, precision, d_order, d_grad_out_xyz,
                                d_grad_out_normal, d_grad_xyz, d_grad_h, (cudaStream_t)stream);
}

int mls_project_backward_sorted(const mls_grid *g, const int32_t *d_pos, int k, float h, int degree, int precision,
                                const float *d_grad_out_xyz, const float *d_grad_out_normal, float *d_grad_xyz,
                                float *d_grad_h, const float *d_state, const int32_t *d_offsets,
                                mls_stream stream) {
    mls::g_last_error[0] = 0;
    if (!g || !d_pos || !d_grad_out_xyz || !d_grad_xyz || !d_grad_h)
        return set_error(MLS_ERR_INVALID_ARG, "mls_project_backward_sorted: null pointer");
    if (g->n < 1) return set_error(MLS_ERR_INVALID_ARG, "mls_project_backward_sorted: grid is empty (failed build?)");
    if (g->n > 0x7fffffffLL / MLS_MAX_K)
        return set_error(MLS_ERR_TOO_LARGE, "mls_project_backward_sorted: n = %lld", (long long)g->n);
    if (k < 1 || k > MLS_MAX_K || k > g->n)
        return set_error(MLS_ERR_K_TOO_LARGE, "mls_project_backward_sorted: k = %d not in [1, min(%d, n)]", k,
                         MLS_MAX_K);
    if (!(h > 0.0f) || !std::isfinite(h))
        return set_error(MLS_ERR_INVALID_ARG, "mls_project_backward_sorted: h = %g must be finite and > 0", (double)h);
    if (degree < 0 || degree > 2)
        return set_error(MLS_ERR_UNSUPPORTED_DEGREE, "mls_project_backward_sorted: degree = %d", degree);
    if (precision != MLS_PREC_FP32 && precision != MLS_PREC_MIXED)
        return set_error(MLS_ERR_INVALID_ARG, "mls_project_backward_sorted: precision = %d (FP32 or mixed)",
                         precision);
    if ((const void *)d_grad_xyz == (const void *)g->xyz || (const void *)d_grad_xyz == (const void *)d_grad_out_xyz)
        return set_error(MLS_ERR_INVALID_ARG, "mls_project_backward_sorted: output aliases an input");
    return mls::launch_backward_sorted(g->view.pts, g->perm, g->n, d_pos, k, h, degree, precision, d_grad_out_xyz,
                                       d_grad_out_normal, d_grad_xyz, d_grad_h, d_state, d_offsets,
                                       (cudaStream_t)stream);
}

int mls_points_in_boxes(const mls_grid *g, const float *d_boxes, int64_t m, uint8_t *d_mask, mls_stream stream) {
    mls::g_last_error[0] = 0;
    if (!g || !d_mask || (m > 0 && !d_boxes))
        return set_error(MLS_ERR_INVALID_ARG, "mls_points_in_boxes: null pointer");
    if (g->n < 1) return set_error(MLS_ERR_INVALID_ARG, "mls_points_in_boxes: grid is empty (failed build?)");
    if (m < 0) return set_error(MLS_ERR_INVALID_ARG, "mls_points_in_boxes: m = %lld < 0", (long long)m);
    return mls::launch_points_in_boxes(g, d_boxes, m, d_mask, (cudaStream_t)stream);
}

int mls_mean_knn_dist(const float *d_xyz, int64_t n, const int32_t *d_idx, int k, double *d_out,
                      mls_stream stream) {
    mls::g_last_error[0] = 0;
    if (!d_xyz || !d_idx || !d_out) return set_error(MLS_ERR_INVALID_ARG, "mls_mean_knn_dist: null pointer");
    if (n < 1 || k < 1 || k > MLS_MAX_K) return set_error(MLS_ERR_INVALID_ARG, "mls_mean_knn_dist: n or k");
    cudaStream_t st = (cudaStream_t)stream;
    mls::ScratchSet scratch(st);
    double *part = nullptr;
    MLS_CUDA_TRY(scratch.alloc(&part, 2 * mls::kMeanBlocks * sizeof(double)));
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(part + mls::kMeanBlocks);
    mls::k_mean_dist<<<mls::kMeanBlocks, mls::kMeanThreads, 0, st>>>(d_xyz, n, d_idx, k, part, cnt);
    mls::k_mean_finish<<<1, 1024, 0, st>>>(part, cnt, d_out);
    mls::count_launches(2);
    MLS_CUDA_TRY(cudaGetLastError());
    return MLS_OK;
}

}  // extern "C"
