// The single-cloud MLS projection kernels (Sec. 1.4, Eq. 1; Algorithm 1):
// weighted plane, origin q on it, local height polynomial, projection onto
// the polynomial.  One thread per point (each point is independent, as the
// paper's information graph shows), so the per-point 3x3 eigensolve and 6x6
// solve run on every lane at once; the per-point arithmetic is
// project_point (project_point.cuh).  The FP64 form is a plain restatement in
// double, kept as the slow comparison path.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <mutex>

#include "grid.cuh"
#include "project_point.cuh"

namespace mls {

namespace {

constexpr int kProjThreads = 128;

// Copy of the points as float4 (w = 0): one 16-byte load per neighbour gather.
__global__ void k_pack_xyz4(const float *__restrict__ xyz, int64_t n, float4 *__restrict__ xyz4) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        xyz4[i] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], 0.f);
}

// FP32 / mixed projection, one thread per point.  The warp first copies its
// 32 neighbour rows into shared memory with coalesced loads (stored
// transposed, entry j of lane t at j * kRowStride + t), then every lane runs
// project_point on its own point.  Eight blocks per SM (64 registers): the
// kernel waits on its neighbour gathers, and the extra warps hide that
// latency (measured 11 % faster than five blocks at 88 registers).
// With DEFER (the mixed form with scratch available), a point that needs an
// FP64 step is not finished here: its slot goes to deferred[] (count in
// *n_deferred) for k_project_deferred, so that the warps of this kernel never
// wait on FP64 arithmetic (GB300's FP64 rate is a small fraction of FP32).
// With SORTED, xyz4 is the grid's sorted copy of the points (w = the point's
// original index bits), slot s is sorted position s, idx holds the rows of
// sorted positions by sorted position, and each result goes to the point's
// original index.  With STATE (SORTED only) each point's fit state goes to
// state[c * n + slot] (FitState).  With SKIP, slots with skip[slot] != 0 are
// left alone (their rows are not written yet).
template <int DEG, int PREC, bool LEVIN = false, bool DEFER = false, bool SORTED = false, bool STATE = false,
          bool SKIP = false>
__global__ void __launch_bounds__(kProjThreads, LEVIN ? 5 : 8) k_project(const float4 *__restrict__ xyz4, int64_t n,
                                                          const int32_t *__restrict__ idx, int k, float h,
                                                          const int32_t *__restrict__ order,
                                                          float *__restrict__ out_xyz, float *__restrict__ out_n,
                                                          uint8_t *__restrict__ status, int max_iter,
                                                          float tol, int32_t *__restrict__ deferred,
                                                          int32_t *__restrict__ n_deferred,
                                                          float *__restrict__ state = nullptr,
                                                          const uint8_t *__restrict__ skip = nullptr) {
    extern __shared__ int32_t rows[];
    const int lane = threadIdx.x & 31;
    int32_t *my_rows = rows + (threadIdx.x >> 5) * k * kRowStride;
    const int64_t slot = blockIdx.x * (int64_t)kProjThreads + threadIdx.x;
    const int64_t warp_base = slot - lane;
    const int64_t i = slot < n ? (order ? (int64_t)__ldg(order + slot) : slot) : -1;
    const int nrows = (int)min((int64_t)32, n - warp_base);
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
        const int64_t i_r = __shfl_sync(0xffffffffu, i, r);
        if (r < nrows)
            for (int c = lane; c < k; c += 32) my_rows[c * kRowStride + r] = __ldg(idx + i_r * k + c);
    }
    __syncwarp();
    if (slot >= n) return;
    if (SKIP && __ldg(skip + slot)) return;
    const float4 r4 = __ldg(xyz4 + i);
    float out[3], nf[3];
    const uint8_t st = project_point<DEG, PREC, LEVIN, DEFER, STATE>(
        xyz4, [&](int j) { return my_rows[j * kRowStride + lane]; }, k, 0, 1, h, r4.x, r4.y, r4.z, out, nf, max_iter, tol,
        STATE ? state + slot : nullptr, n);
    if (DEFER && st == kDeferFP64) {
        deferred[atomicAdd(n_deferred, 1)] = (int32_t)slot;
        return;
    }
    const int64_t o = SORTED ? (int64_t)__float_as_int(r4.w) : i;
    out_xyz[3 * o] = out[0];
    out_xyz[3 * o + 1] = out[1];
    out_xyz[3 * o + 2] = out[2];
    if (out_n) {
        out_n[3 * o] = nf[0];
        out_n[3 * o + 1] = nf[1];
        out_n[3 * o + 2] = nf[2];
    }
    if (status) status[o] = st;
}

// The deferred points of the mixed form, one thread each: the same routine
// with its FP64 steps, rows read from global memory (same values and order
// as the first pass, so the results are those of a single pass).  SORTED and
// STATE as in k_project.
template <int DEG, bool SORTED = false, bool STATE = false, int PREC = MLS_PREC_MIXED>
__global__ void __launch_bounds__(kProjThreads) k_project_deferred(const float4 *__restrict__ xyz4, int64_t n,
                                                                  const int32_t *__restrict__ idx, int k, float h,
                                                                  const int32_t *__restrict__ order,
                                                                  const int32_t *__restrict__ deferred,
                                                                  const int32_t *__restrict__ n_deferred,
                                                                  float *__restrict__ out_xyz,
                                                                  float *__restrict__ out_n,
                                                                  uint8_t *__restrict__ status,
                                                                  float *__restrict__ state = nullptr) {
    const int count = *n_deferred;
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < count; d += gridDim.x * blockDim.x) {
        const int64_t slot = deferred[d];
        const int64_t i = order ? (int64_t)__ldg(order + slot) : slot;
        const int32_t *row = idx + i * k;
        const float4 r4 = __ldg(xyz4 + i);
        float out[3], nf[3];
        const uint8_t st = project_point<DEG, PREC, false, false, STATE>(
            xyz4, [&](int j) { return __ldg(row + j); }, k, 0, 1, h, r4.x, r4.y, r4.z, out, nf, 1, 0.f,
            STATE ? state + slot : nullptr, n);
        const int64_t o = SORTED ? (int64_t)__float_as_int(r4.w) : i;
        out_xyz[3 * o] = out[0];
        out_xyz[3 * o + 1] = out[1];
        out_xyz[3 * o + 2] = out[2];
        if (out_n) {
            out_n[3 * o] = nf[0];
            out_n[3 * o + 1] = nf[1];
            out_n[3 * o + 2] = nf[2];
        }
        if (status) status[o] = st;
    }
}

// Variable neighbourhoods (CSR rows, e.g. the radius-R sets of Sec. 1.4),
// one thread per point, rows read straight from global memory.  A point with
// fewer than min_nb other points in its row is an outlier (Sec. 3.3): not
// projected, status MLS_PT_OUTLIER, output = the point, normal = 0.  A row of
// fewer than twice as many points as the basis has coefficients is fitted at
// the next lower degree that has enough (status MLS_PT_DEGREE_REDUCED).
template <int DEG, int PREC>
__global__ void __launch_bounds__(kProjThreads, 8) k_project_rows(const float4 *__restrict__ xyz4, int64_t n,
                                                               const int64_t *__restrict__ off,
                                                               const int32_t *__restrict__ rows, float h,
                                                               int min_nb, const int32_t *__restrict__ order,
                                                               float *__restrict__ out_xyz,
                                                               float *__restrict__ out_n,
                                                               uint8_t *__restrict__ status) {
    const int64_t slot = blockIdx.x * (int64_t)kProjThreads + threadIdx.x;
    if (slot >= n) return;
    const int64_t i = order ? (int64_t)__ldg(order + slot) : slot;
    const int64_t b = __ldg(off + i);
    const int k = (int)(__ldg(off + i + 1) - b);
    const float4 r4 = __ldg(xyz4 + i);
    float out[3] = {r4.x, r4.y, r4.z}, nf[3] = {0.f, 0.f, 0.f};
    uint8_t st = MLS_PT_OUTLIER;
    const auto row = [&](int j) { return __ldg(rows + b + j); };
    if (k - 1 >= min_nb) {
        // the highest degree whose basis has at most k / 2 coefficients
        // (6, 3, 1): a smaller neighbourhood would be interpolated, not
        // smoothed, and a quadratic over 4-6 points can throw the point far
        if (DEG == 2 && k >= 12)
            st = project_point<DEG, PREC>(xyz4, row, k, 0, 1, h, r4.x, r4.y, r4.z, out, nf);
        else if (DEG >= 1 && k >= 6)
            st = project_point<1, PREC>(xyz4, row, k, 0, 1, h, r4.x, r4.y, r4.z, out, nf) |
                 (DEG > 1 ? MLS_PT_DEGREE_REDUCED : 0);
        else
            st = project_point<0, PREC>(xyz4, row, k, 0, 1, h, r4.x, r4.y, r4.z, out, nf) |
                 (DEG > 0 ? MLS_PT_DEGREE_REDUCED : 0);
    }
    out_xyz[3 * i] = out[0];
    out_xyz[3 * i + 1] = out[1];
    out_xyz[3 * i + 2] = out[2];
    if (out_n) {
        out_n[3 * i] = nf[0];
        out_n[3 * i + 1] = nf[1];
        out_n[3 * i + 2] = nf[2];
    }
    if (status) status[i] = st;
}

// The plain FP64 form: the same three passes, every quantity in double,
// neighbours re-read from global memory in each pass.
template <int DEG>
__global__ void __launch_bounds__(kProjThreads) k_project_fp64(const float *__restrict__ xyz, int64_t n,
                                                               const int32_t *__restrict__ idx, int k, float h,
                                                               const int32_t *__restrict__ order,
                                                               float *__restrict__ out_xyz,
                                                               float *__restrict__ out_n,
                                                               uint8_t *__restrict__ status) {
    const int64_t slot = blockIdx.x * (int64_t)kProjThreads + threadIdx.x;
    if (slot >= n) return;
    const int64_t i = order ? (int64_t)order[slot] : slot;
    const double r[3] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
    const int32_t *row = idx + i * k;
    const double hd = (double)h, inv_h2 = 1.0 / (hd * hd);
    double W = 0, m[3] = {0, 0, 0}, D2 = 0;
    for (int j = 0; j < k; ++j) {
        const int64_t p = __ldg(row + j);
        double d[3], dd = 0;
        for (int a = 0; a < 3; ++a) {
            d[a] = (double)__ldg(xyz + 3 * p + a) - r[a];
            dd += d[a] * d[a];
        }
        D2 = fmax(D2, dd);
        const double w = exp(-dd * inv_h2);
        W += w;
        for (int a = 0; a < 3; ++a) m[a] += w * d[a];
    }
    for (int a = 0; a < 3; ++a) m[a] /= W;
    double C[6] = {0, 0, 0, 0, 0, 0};
    for (int j = 0; j < k; ++j) {
        const int64_t p = __ldg(row + j);
        double d[3], dd = 0;
        for (int a = 0; a < 3; ++a) {
            d[a] = (double)__ldg(xyz + 3 * p + a) - r[a];
            dd += d[a] * d[a];
        }
        const double w = exp(-dd * inv_h2);
        const double e[3] = {d[0] - m[0], d[1] - m[1], d[2] - m[2]};
        C[0] += w * e[0] * e[0];
        C[1] += w * e[0] * e[1];
        C[2] += w * e[0] * e[2];
        C[3] += w * e[1] * e[1];
        C[4] += w * e[1] * e[2];
        C[5] += w * e[2] * e[2];
    }
    double nrm[3], e1[3], e2[3], lam[3];
    uint8_t st = (uint8_t)frame_from<double>(C, nrm, e1, e2, lam);
    if (!(lam[2] > (double)kMinSpread * W * D2)) st = MLS_PT_PLANE_DEGENERATE;
    double out[3] = {r[0], r[1], r[2]};
    if (!st) {
        constexpr int M = Basis<DEG>::M;
        const double ofs = nrm[0] * m[0] + nrm[1] * m[1] + nrm[2] * m[2];
        double A[M][M], b[M], L[M][M], x[M];
        for (int a = 0; a < M; ++a) {
            b[a] = 0;
            for (int c = 0; c < M; ++c) A[a][c] = 0;
        }
        for (int j = 0; j < k; ++j) {
            const int64_t p = __ldg(row + j);
            double d[3], dd = 0;
            for (int a = 0; a < 3; ++a) {
                d[a] = (double)__ldg(xyz + 3 * p + a) - r[a];
                dd += d[a] * d[a];
            }
            const double w = exp(-dd * inv_h2);
            const double u = (e1[0] * d[0] + e1[1] * d[1] + e1[2] * d[2]) / hd;
            const double v = (e2[0] * d[0] + e2[1] * d[1] + e2[2] * d[2]) / hd;
            const double f = nrm[0] * d[0] + nrm[1] * d[1] + nrm[2] * d[2] - ofs;
            double phi[6] = {1.0, u, v, u * u, u * v, v * v};
            for (int a = 0; a < M; ++a) {
                b[a] += w * phi[a] * f;
                for (int c = 0; c < M; ++c) A[a][c] += w * phi[a] * phi[c];
            }
        }
        double pmin, pmax, invd[M];
        double a0 = 0;
        if (cholesky<double, M>(A, L, invd, 1e-12, pmin, pmax)) {
            chol_solve<double, M>(L, invd, b, x);
            a0 = x[0];
        } else {
            st |= MLS_PT_POLY_SINGULAR;
        }
        const double s = ofs + a0;
        for (int a = 0; a < 3; ++a) out[a] = r[a] + s * nrm[a];
    }
    for (int a = 0; a < 3; ++a) {
        out_xyz[3 * i + a] = (float)out[a];
        if (out_n) out_n[3 * i + a] = (float)nrm[a];
    }
    if (status) status[i] = st;
}

template <int DEG>
int launch_deg(const float *xyz, int64_t n, const int32_t *idx, int k, float h, int precision,
               const int32_t *order, float *out_xyz, float *out_n, uint8_t *status, cudaStream_t st) {
    const int blocks = (int)((n + kProjThreads - 1) / kProjThreads);
    if (precision == MLS_PREC_FP64) {
        k_project_fp64<DEG><<<blocks, kProjThreads, 0, st>>>(xyz, n, idx, k, h, order, out_xyz, out_n, status);
        count_launches(1);
    } else {
        // a stream-ordered scratch copy of the points as float4
        ScratchSet scratch(st);
        float4 *xyz4 = nullptr;
        MLS_CUDA_TRY(scratch.alloc(&xyz4, (size_t)n * sizeof(float4)));
        k_pack_xyz4<<<(int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 16), 256, 0, st>>>(xyz, n, xyz4);
        const size_t smem = (size_t)k * kRowStride * sizeof(int32_t) * (kProjThreads / 32);
        if (precision == MLS_PREC_MIXED) {
            // FP64 points deferred to a second, compact pass
            int32_t *deferred = nullptr;
            MLS_CUDA_TRY(scratch.alloc(&deferred, (size_t)(n + 1) * sizeof(int32_t)));
            int32_t *n_deferred = deferred + n;
            MLS_CUDA_TRY(cudaMemsetAsync(n_deferred, 0, sizeof(int32_t), st));
            auto kern = k_project<DEG, MLS_PREC_MIXED, false, true>;
            MLS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            kern<<<blocks, kProjThreads, smem, st>>>(xyz4, n, idx, k, h, order, out_xyz, out_n, status, 1, 0.f,
                                                     deferred, n_deferred, nullptr, nullptr);
            k_project_deferred<DEG><<<sm_count() * 2, kProjThreads, 0, st>>>(xyz4, n, idx, k, h, order, deferred, n_deferred,
                                                                     out_xyz, out_n, status);
            count_launches(3);
        } else {
            auto kern = k_project<DEG, MLS_PREC_FP32>;
            MLS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            kern<<<blocks, kProjThreads, smem, st>>>(xyz4, n, idx, k, h, order, out_xyz, out_n, status, 1, 0.f,
                                                     nullptr, nullptr, nullptr, nullptr);
            count_launches(2);
        }
    }
    MLS_CUDA_TRY(cudaGetLastError());
    return MLS_OK;
}

}  // namespace

int launch_project(const float *xyz, int64_t n, const int32_t *idx, int k, float h, int degree, int precision,
                   const int32_t *order, float *out_xyz, float *out_n, uint8_t *status, cudaStream_t st) {
    switch (degree) {
        case 0:
            return launch_deg<0>(xyz, n, idx, k, h, precision, order, out_xyz, out_n, status, st);
        case 1:
            return launch_deg<1>(xyz, n, idx, k, h, precision, order, out_xyz, out_n, status, st);
        default:
            return launch_deg<2>(xyz, n, idx, k, h, precision, order, out_xyz, out_n, status, st);
    }
}

namespace {

// The projection over the grid's sorted points and rows of sorted positions.
// (Two lanes per point, as the batched kernel's autotuner prefers, measured
// slower here: 0.63 ms against 0.56 ms on the 2M-point torus.)
template <int DEG, bool STATE>
int launch_sorted_deg(const float4 *pts, int64_t n, const int32_t *pos, int k, float h, int precision,
                      float *out_xyz, float *out_n, uint8_t *status, float *state, cudaStream_t st) {
    const int blocks = (int)((n + kProjThreads - 1) / kProjThreads);
    const size_t smem = (size_t)k * kRowStride * sizeof(int32_t) * (kProjThreads / 32);
    if (precision == MLS_PREC_MIXED) {
        ScratchSet scratch(st);
        int32_t *deferred = nullptr;
        MLS_CUDA_TRY(scratch.alloc(&deferred, (size_t)(n + 1) * sizeof(int32_t)));
        int32_t *n_deferred = deferred + n;
        MLS_CUDA_TRY(cudaMemsetAsync(n_deferred, 0, sizeof(int32_t), st));
        auto kern = k_project<DEG, MLS_PREC_MIXED, false, true, true, STATE>;
        MLS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<blocks, kProjThreads, smem, st>>>(pts, n, pos, k, h, nullptr, out_xyz, out_n, status, 1, 0.f,
                                                 deferred, n_deferred, state, nullptr);
        k_project_deferred<DEG, true, STATE><<<sm_count() * 2, kProjThreads, 0, st>>>(
            pts, n, pos, k, h, nullptr, deferred, n_deferred, out_xyz, out_n, status, state);
        count_launches(2);
    } else {
        auto kern = k_project<DEG, MLS_PREC_FP32, false, false, true, STATE>;
        MLS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<blocks, kProjThreads, smem, st>>>(pts, n, pos, k, h, nullptr, out_xyz, out_n, status, 1, 0.f,
                                                 nullptr, nullptr, state, nullptr);
        count_launches(1);
    }
    MLS_CUDA_TRY(cudaGetLastError());
    return MLS_OK;
}

}  // namespace

int launch_project_sorted(const float4 *pts, int64_t n, const int32_t *pos, int k, float h, int degree,
                          int precision, float *out_xyz, float *out_n, uint8_t *status, float *state,
                          cudaStream_t st) {
    if (state) {
        switch (degree) {
            case 0: return launch_sorted_deg<0, true>(pts, n, pos, k, h, precision, out_xyz, out_n, status, state, st);
            case 1: return launch_sorted_deg<1, true>(pts, n, pos, k, h, precision, out_xyz, out_n, status, state, st);
            default: return launch_sorted_deg<2, true>(pts, n, pos, k, h, precision, out_xyz, out_n, status, state, st);
        }
    }
    switch (degree) {
        case 0: return launch_sorted_deg<0, false>(pts, n, pos, k, h, precision, out_xyz, out_n, status, nullptr, st);
        case 1: return launch_sorted_deg<1, false>(pts, n, pos, k, h, precision, out_xyz, out_n, status, nullptr, st);
        default: return launch_sorted_deg<2, false>(pts, n, pos, k, h, precision, out_xyz, out_n, status, nullptr, st);
    }
}

int launch_project_rows(const float *xyz, int64_t n, const int64_t *off, const int32_t *rows, float h, int degree,
                        int precision, int min_nb, const int32_t *order, float *out_xyz, float *out_n,
                        uint8_t *status, cudaStream_t st) {
    ScratchSet scratch(st);
    float4 *xyz4 = nullptr;
    MLS_CUDA_TRY(scratch.alloc(&xyz4, (size_t)n * sizeof(float4)));
    k_pack_xyz4<<<(int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 16), 256, 0, st>>>(xyz, n, xyz4);
    const int blocks = (int)((n + kProjThreads - 1) / kProjThreads);
    const bool mixed = precision == MLS_PREC_MIXED;
    switch (degree) {
        case 0:
            (mixed ? k_project_rows<0, MLS_PREC_MIXED> : k_project_rows<0, MLS_PREC_FP32>)<<<blocks, kProjThreads, 0, st>>>(
                xyz4, n, off, rows, h, min_nb, order, out_xyz, out_n, status);
            break;
        case 1:
            (mixed ? k_project_rows<1, MLS_PREC_MIXED> : k_project_rows<1, MLS_PREC_FP32>)<<<blocks, kProjThreads, 0, st>>>(
                xyz4, n, off, rows, h, min_nb, order, out_xyz, out_n, status);
            break;
        default:
            (mixed ? k_project_rows<2, MLS_PREC_MIXED> : k_project_rows<2, MLS_PREC_FP32>)<<<blocks, kProjThreads, 0, st>>>(
                xyz4, n, off, rows, h, min_nb, order, out_xyz, out_n, status);
            break;
    }
    count_launches(2);
    MLS_CUDA_TRY(cudaGetLastError());
    return MLS_OK;
}

namespace {

// The form with the weights about q (Sec. 1.4, Eq. 1): FP32 or mixed.
template <int DEG>
int launch_levin_deg(const float *xyz, int64_t n, const int32_t *idx, int k, float h, int precision, int max_iter,
                     float tol, const int32_t *order, float *out_xyz, float *out_n, uint8_t *status,
                     cudaStream_t st) {
    const int blocks = (int)((n + kProjThreads - 1) / kProjThreads);
    ScratchSet scratch(st);
    float4 *xyz4 = nullptr;
    MLS_CUDA_TRY(scratch.alloc(&xyz4, (size_t)n * sizeof(float4)));
    k_pack_xyz4<<<(int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 16), 256, 0, st>>>(xyz, n, xyz4);
    const size_t smem = (size_t)k * kRowStride * sizeof(int32_t) * (kProjThreads / 32);
    if (precision == MLS_PREC_MIXED) {
        auto kern = k_project<DEG, MLS_PREC_MIXED, true>;
        MLS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<blocks, kProjThreads, smem, st>>>(xyz4, n, idx, k, h, order, out_xyz, out_n, status, max_iter, tol,
                                                 nullptr, nullptr, nullptr, nullptr);
    } else {
        auto kern = k_project<DEG, MLS_PREC_FP32, true>;
        MLS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<blocks, kProjThreads, smem, st>>>(xyz4, n, idx, k, h, order, out_xyz, out_n, status, max_iter, tol,
                                                 nullptr, nullptr, nullptr, nullptr);
    }
    count_launches(2);
    MLS_CUDA_TRY(cudaGetLastError());
    return MLS_OK;
}

}  // namespace

int launch_project_levin(const float *xyz, int64_t n, const int32_t *idx, int k, float h, int degree,
                         int precision, int max_iter, float tol, const int32_t *order, float *out_xyz,
                         float *out_n, uint8_t *status, cudaStream_t st) {
    switch (degree) {
        case 0:
            return launch_levin_deg<0>(xyz, n, idx, k, h, precision, max_iter, tol, order, out_xyz, out_n, status, st);
        case 1:
            return launch_levin_deg<1>(xyz, n, idx, k, h, precision, max_iter, tol, order, out_xyz, out_n, status, st);
        default:
            return launch_levin_deg<2>(xyz, n, idx, k, h, precision, max_iter, tol, order, out_xyz, out_n, status, st);
    }
}

// ---- mls_project_noalloc --------------------------------------------------
//
// The same kernels as mls_project, with the float4 copy of the points kept in
// a file-scope device array instead of stream-ordered scratch.  The array is
// a host-side stand-in in host code: its device address is looked up with the
// device current and passed to the kernels -- on every call made outside a
// stream capture (so a device reset in between cannot leave a stale address),
// from the per-device cache of the last look-up during a capture.

namespace {

__device__ __align__(256) float4 g_noalloc_xyz4[MLS_NOALLOC_MAX_POINTS];

constexpr int kMaxDevices = 64;
float4 *g_noalloc_addr[kMaxDevices] = {};
std::mutex g_noalloc_mutex;

int noalloc_scratch(cudaStream_t st, float4 **out) {
    int dev = 0;
    MLS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(MLS_ERR_CUDA, "mls_project_noalloc: device %d", dev);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    MLS_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev] || cap == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        MLS_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_xyz4));
        g_noalloc_addr[dev] = (float4 *)p;
    }
    *out = g_noalloc_addr[dev];
    return MLS_OK;
}

template <int DEG>
int launch_noalloc(const float *xyz, int64_t n, const int32_t *idx, int k, float h, int precision,
                   const int32_t *order, float *out_xyz, float *out_n, uint8_t *status, cudaStream_t st) {
    const int blocks = (int)((n + kProjThreads - 1) / kProjThreads);
    if (precision == MLS_PREC_FP64) {
        k_project_fp64<DEG><<<blocks, kProjThreads, 0, st>>>(xyz, n, idx, k, h, order, out_xyz, out_n, status);
        count_launches(1);
    } else {
        float4 *xyz4 = nullptr;
        int rc = noalloc_scratch(st, &xyz4);
        if (rc != MLS_OK) return rc;
        k_pack_xyz4<<<(int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 16), 256, 0, st>>>(xyz, n, xyz4);
        const size_t smem = (size_t)k * kRowStride * sizeof(int32_t) * (kProjThreads / 32);
        if (precision == MLS_PREC_MIXED) {
            auto kern = k_project<DEG, MLS_PREC_MIXED>;
            MLS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            kern<<<blocks, kProjThreads, smem, st>>>(xyz4, n, idx, k, h, order, out_xyz, out_n, status, 1, 0.f,
                                                     nullptr, nullptr, nullptr, nullptr);
        } else {
            auto kern = k_project<DEG, MLS_PREC_FP32>;
            MLS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            kern<<<blocks, kProjThreads, smem, st>>>(xyz4, n, idx, k, h, order, out_xyz, out_n, status, 1, 0.f,
                                                     nullptr, nullptr, nullptr, nullptr);
        }
        count_launches(2);
    }
    MLS_CUDA_TRY(cudaGetLastError());
    return MLS_OK;
}

}  // namespace

}  // namespace mls

extern "C" int mls_project_noalloc(const float *d_xyz, int64_t n, const int32_t *d_idx, int k, float h, int degree,
                                   int precision, const int32_t *d_order, float *d_out_xyz, float *d_out_normal,
                                   uint8_t *d_status, mls_stream stream) {
    using mls::set_error;
    mls::clear_error();
    if (!d_xyz || !d_idx || !d_out_xyz) return set_error(MLS_ERR_INVALID_ARG, "mls_project_noalloc: null pointer");
    if (n < 1) return set_error(MLS_ERR_INVALID_ARG, "mls_project_noalloc: n = %lld < 1", (long long)n);
    if (n > MLS_NOALLOC_MAX_POINTS)
        return set_error(MLS_ERR_TOO_LARGE,
                         "mls_project_noalloc: n = %lld exceeds its fixed scratch of %d points; use mls_project",
                         (long long)n, MLS_NOALLOC_MAX_POINTS);
    if (k < 1 || k > MLS_MAX_K || k > n)
        return set_error(MLS_ERR_K_TOO_LARGE, "mls_project_noalloc: k = %d not in [1, min(%d, n)]", k, MLS_MAX_K);
    if (!(h > 0.0f) || !std::isfinite(h))
        return set_error(MLS_ERR_INVALID_ARG, "mls_project_noalloc: h = %g must be finite and > 0", (double)h);
    if (degree < 0 || degree > 2)
        return set_error(MLS_ERR_UNSUPPORTED_DEGREE, "mls_project_noalloc: degree = %d not in {0, 1, 2}", degree);
    if (precision < MLS_PREC_FP32 || precision > MLS_PREC_FP64)
        return set_error(MLS_ERR_INVALID_ARG, "mls_project_noalloc: precision = %d", precision);
    if ((const void *)d_out_xyz == (const void *)d_xyz)
        return set_error(MLS_ERR_INVALID_ARG, "mls_project_noalloc: output aliases the input");
    cudaStream_t st = (cudaStream_t)stream;
    switch (degree) {
        case 0:
            return mls::launch_noalloc<0>(d_xyz, n, d_idx, k, h, precision, d_order, d_out_xyz, d_out_normal, d_status, st);
        case 1:
            return mls::launch_noalloc<1>(d_xyz, n, d_idx, k, h, precision, d_order, d_out_xyz, d_out_normal, d_status, st);
        default:
            return mls::launch_noalloc<2>(d_xyz, n, d_idx, k, h, precision, d_order, d_out_xyz, d_out_normal, d_status, st);
    }
}

namespace mls {

int launch_knn_chain_pass(const mls_grid *grid, int k, int32_t *idx, float *key, int32_t *pos, cudaStream_t st,
                          const uint8_t *skip, int *iso, int blocks_per_sm, bool reset);
int launch_knn_sparse_pass(const mls_grid *grid, int k, int32_t *idx, float *key, int32_t *pos, cudaStream_t st,
                           int blocks_per_sm);
int launch_knn_isolated(const mls_grid *grid, uint8_t *skip, int *iso, int32_t *list, int32_t *count,
                        cudaStream_t st);
bool knn_isolates(const mls_grid *grid);
int launch_backward_offsets(const int32_t *rows, int64_t n, int k, int32_t *off, cudaStream_t st);

namespace {

// The queries the kNN's chain pass left to its sparse pass (the grid's work
// list): flagged in skip[] and appended to the list of slots projected last.
__global__ void k_mark_sparse(const int *__restrict__ work, uint8_t *__restrict__ skip, int32_t *__restrict__ list,
                              int32_t *__restrict__ count) {
    const int m = work[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const int32_t sp = work[8 + i];
        skip[sp] = 1;
        list[atomicAdd(count, 1)] = sp;
    }
}

// The kNN and the projection, pipelined, on the caller's stream and a
// high-priority stream of the grid's own.  From a few hundred thousand
// points, the isolated queries (outliers alone in a cell two base cells wide,
// whose searches climb to coarse levels and scan many points) are listed
// first; the chain pass's warps take them before their runs, so that their
// long searches end under the chain pass instead of after it.  Then the sparse pass over the queries the chain pass
// left runs on the side stream while the projection of every point whose row
// the chain pass wrote runs on the caller's stream beside it; last, the
// isolated and sparse points, and in the mixed form the points that need an
// FP64 step, are projected from one list.  The same rows and the same per-point arithmetic
// as mls_knn_sorted followed by mls_project_sorted.  With `offsets`, the
// adjoint's bucket offsets are counted from the finished rows on the side
// stream too, beside the projection's tail.
template <int DEG, int PREC, bool STATE>
int knn_project_pipelined(const mls_grid *g, int k, float h, int32_t *pos, float *out_xyz, float *out_n,
                          uint8_t *status, float *state, int32_t *offsets, cudaStream_t st) {
    const int64_t n = g->n;
    if (!g->side) {
        int least = 0, greatest = 0;
        MLS_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        MLS_CUDA_TRY(cudaStreamCreateWithPriority(&g->side, cudaStreamNonBlocking, greatest));
        MLS_CUDA_TRY(cudaEventCreateWithFlags(&g->side_ev[0], cudaEventDisableTiming));
        MLS_CUDA_TRY(cudaEventCreateWithFlags(&g->side_ev[1], cudaEventDisableTiming));
    }
    ScratchSet scratch(st);     // freed on st, after it has waited for the side stream
    uint8_t *skip = nullptr;
    int32_t *list = nullptr;
    int *iso = nullptr;         // the isolated queries, in the kNN's work-list layout
    const bool isolate = knn_isolates(g);
    MLS_CUDA_TRY(scratch.alloc(&skip, (size_t)n));
    MLS_CUDA_TRY(scratch.alloc(&list, (size_t)(n + 1) * sizeof(int32_t)));
    if (isolate) MLS_CUDA_TRY(scratch.alloc(&iso, (size_t)(n + 8) * sizeof(int)));
    int32_t *count = list + n;
    if (!isolate) MLS_CUDA_TRY(cudaMemsetAsync(skip, 0, (size_t)n, st));
    MLS_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(int32_t), st));
    const int blocks = (int)((n + kProjThreads - 1) / kProjThreads);
    const size_t smem = (size_t)k * kRowStride * sizeof(int32_t) * (kProjThreads / 32);
    constexpr bool DEFER = PREC == MLS_PREC_MIXED;
    auto kern = k_project<DEG, PREC, false, DEFER, true, STATE, true>;
    MLS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int rc = isolate ? launch_knn_isolated(g, skip, iso, list, count, st) : MLS_OK;
    if (rc == MLS_OK)
        rc = isolate ? launch_knn_chain_pass(g, k, nullptr, nullptr, pos, st, skip, iso, 0, false)
                     : launch_knn_chain_pass(g, k, nullptr, nullptr, pos, st, nullptr, nullptr, 0, true);
    if (rc != MLS_OK) return rc;
    k_mark_sparse<<<sm_count(), 256, 0, st>>>(g->work, skip, list, count);
    MLS_CUDA_TRY(cudaEventRecord(g->side_ev[0], st));
    MLS_CUDA_TRY(cudaStreamWaitEvent(g->side, g->side_ev[0], 0));
    // a full wave of sparse blocks (fewer, leaving room for the projection
    // from the start, measured slower: the sparse pass is the longer path)
    rc = launch_knn_sparse_pass(g, k, nullptr, nullptr, pos, g->side, 0);
    if (rc == MLS_OK && offsets) rc = launch_backward_offsets(pos, n, k, offsets, g->side);
    MLS_CUDA_TRY(cudaEventRecord(g->side_ev[1], g->side));
    if (rc != MLS_OK) {     // the caller's stream still waits for what went to the side stream
        cudaStreamWaitEvent(st, g->side_ev[1], 0);
        return rc;
    }
    kern<<<blocks, kProjThreads, smem, st>>>(g->view.pts, n, pos, k, h, nullptr, out_xyz, out_n, status, 1, 0.f,
                                             list, count, state, skip);
    MLS_CUDA_TRY(cudaStreamWaitEvent(st, g->side_ev[1], 0));
    k_project_deferred<DEG, true, STATE, PREC><<<sm_count() * 2, kProjThreads, 0, st>>>(
        g->view.pts, n, pos, k, h, nullptr, list, count, out_xyz, out_n, status, state);
    count_launches(3);
    MLS_CUDA_TRY(cudaGetLastError());
    return MLS_OK;
}

template <int PREC, bool STATE>
int knn_project_deg(const mls_grid *g, int k, float h, int degree, int32_t *pos, float *out_xyz, float *out_n,
                    uint8_t *status, float *state, int32_t *offsets, cudaStream_t st) {
    switch (degree) {
        case 0: return knn_project_pipelined<0, PREC, STATE>(g, k, h, pos, out_xyz, out_n, status, state, offsets, st);
        case 1: return knn_project_pipelined<1, PREC, STATE>(g, k, h, pos, out_xyz, out_n, status, state, offsets, st);
        default: return knn_project_pipelined<2, PREC, STATE>(g, k, h, pos, out_xyz, out_n, status, state, offsets, st);
    }
}

}  // namespace

int launch_knn_project_sorted(const mls_grid *g, int k, float h, int degree, int precision, int32_t *pos,
                              float *out_xyz, float *out_n, uint8_t *status, float *state, int32_t *offsets,
                              cudaStream_t st) {
    if (precision == MLS_PREC_FP32)
        return state ? knn_project_deg<MLS_PREC_FP32, true>(g, k, h, degree, pos, out_xyz, out_n, status, state,
                                                            offsets, st)
                     : knn_project_deg<MLS_PREC_FP32, false>(g, k, h, degree, pos, out_xyz, out_n, status, state,
                                                             offsets, st);
    return state ? knn_project_deg<MLS_PREC_MIXED, true>(g, k, h, degree, pos, out_xyz, out_n, status, state, offsets,
                                                         st)
                 : knn_project_deg<MLS_PREC_MIXED, false>(g, k, h, degree, pos, out_xyz, out_n, status, state,
                                                          offsets, st);
}

}  // namespace mls
