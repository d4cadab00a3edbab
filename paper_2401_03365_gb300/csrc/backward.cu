// Adjoint of the MLS projection (not in the paper): gradients of
// L = sum_i <gp_i, p'_i> + <gn_i, n_i> with respect to every input
// coordinate and the bandwidth h, neighbour rows and the normal's sign held
// fixed.  The reverse pass follows the forward of Sec. 1.4 / Algorithm 1
// backwards: projection p' = r + (<n, m> + a0) n; height fit a = A^-1 b
// (b-bar = z = A^-1 e_0 a0-bar, A-bar = -z a^T); local coordinates; the frame,
// through the eigenvector derivative dn = sum_b e_b (e_b^T dC n) / (l0 - l_b)
// with the tangent vectors tilted with n (their spin within the plane leaves
// g(0, 0) unchanged, the basis being rotation invariant); the covariance
// C = sum w e e^T about the centroid; the centroid m = sum w d / W; the
// Gaussian weights.
//
// One thread per point recomputes its forward quantities (no frame is
// stored) and writes the gradient it sends to each of its k neighbours into
// an edge buffer, and the gradient of its own position separately.  A
// reverse adjacency (edges bucketed by target point, each bucket ordered by
// edge number) then sums them in a fixed order: results do not depend on
// scheduling.
#include <algorithm>
#include <climits>

#include "solve.cuh"

namespace mls {

int device_exclusive_scan(const int32_t *in, int32_t *out, int64_t n, cudaStream_t st);

namespace {

constexpr int kBwdThreads = 128;
constexpr float kBwdGapFlag = 1e-3f;
constexpr float kBwdCondFlag = 1e5f;

__global__ void k_pack4(const float *__restrict__ xyz, int64_t n, float4 *__restrict__ xyz4) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        xyz4[i] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], 0.f);
}

template <typename T, int M>
__device__ bool factor_and_solve(const T A[M][M], const T b[M], const T e0bar, T a[M], T z[M], T &cond) {
    T L[M][M], pmin, pmax;
    if (!cholesky<T, M>(A, L, T(1e-12), pmin, pmax)) return false;
    cond = (pmax / pmin) * (pmax / pmin);
    chol_solve<T, M>(L, b, a);
    T rhs[M];
#pragma unroll
    for (int r = 0; r < M; ++r) rhs[r] = r == 0 ? e0bar : T(0);
    chol_solve<T, M>(L, rhs, z);
    return true;
}

// Basis values phi(u, v) of the requested degree.
template <int DEG>
__device__ __forceinline__ void basis(float u, float v, float phi[6]) {
    phi[0] = 1.f;
    if (DEG >= 1) {
        phi[1] = u;
        phi[2] = v;
    }
    if (DEG >= 2) {
        phi[3] = u * u;
        phi[4] = u * v;
        phi[5] = v * v;
    }
}

template <int DEG, int PREC>
__global__ void __launch_bounds__(kBwdThreads) k_backward_point(
    const float4 *__restrict__ xyz4, int64_t n, const int32_t *__restrict__ idx, int k, float h,
    const int32_t *__restrict__ order, const float *__restrict__ gout_xyz, const float *__restrict__ gout_n,
    float *__restrict__ edge_grad, float *__restrict__ self_grad, double *__restrict__ h_part) {
    constexpr int M = Basis<DEG>::M;
    extern __shared__ int32_t rows[];
    __shared__ double hred[kBwdThreads / 32];
    const int lane = threadIdx.x & 31;
    int32_t *my_rows = rows + (threadIdx.x >> 5) * k * 32;
    const int64_t slot = blockIdx.x * (int64_t)kBwdThreads + threadIdx.x;
    const int64_t warp_base = slot - lane;
    const int64_t i = slot < n ? (order ? (int64_t)__ldg(order + slot) : slot) : -1;
    const int nrows = (int)min((int64_t)32, n - warp_base);
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
        const int64_t i_r = __shfl_sync(0xffffffffu, i, r);
        if (r < nrows)
            for (int c = lane; c < k; c += 32) my_rows[c * 32 + r] = __ldg(idx + i_r * k + c);
    }
    __syncwarp();
    float hbar = 0.f;
    if (slot < n) {
        const float4 r4 = __ldg(xyz4 + i);
        const float rx = r4.x, ry = r4.y, rz = r4.z;
        const float h2 = h * h, ih = 1.f / h;
        const float neg_scale = -1.4426950408889634f / h2;
        // ---- forward recompute: weights, centroid offset, covariance ----
        float W = 0.f, m[3] = {0.f, 0.f, 0.f};
        float C[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int j = 0; j < k; ++j) {
            const float4 p = __ldg(xyz4 + my_rows[j * 32 + lane]);
            const float d[3] = {p.x - rx, p.y - ry, p.z - rz};
            const float w = exp2f(fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2])) * neg_scale);
            const float Wn = W + w, c = __fdividef(w, Wn);
            float e[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                e[a] = d[a] - m[a];
                m[a] = fmaf(e[a], c, m[a]);
            }
            const float f = W * c;
            C[0] = fmaf(f * e[0], e[0], C[0]);
            C[1] = fmaf(f * e[0], e[1], C[1]);
            C[2] = fmaf(f * e[0], e[2], C[2]);
            C[3] = fmaf(f * e[1], e[1], C[3]);
            C[4] = fmaf(f * e[1], e[2], C[4]);
            C[5] = fmaf(f * e[2], e[2], C[5]);
            W = Wn;
        }
        float nv[3], e1[3], e2[3], lam[3];
        int flag = frame_from<float>(C, nv, e1, e2, lam);
        if (PREC == MLS_PREC_MIXED && (!(lam[2] > 0.f) || (lam[1] - lam[0]) < kBwdGapFlag * lam[2])) {
            double Cd[6], nd[3], e1d[3], e2d[3], ld[3];
#pragma unroll
            for (int c = 0; c < 6; ++c) Cd[c] = (double)C[c];
            flag = frame_from<double>(Cd, nd, e1d, e2d, ld);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                nv[a] = (float)nd[a];
                e1[a] = (float)e1d[a];
                e2[a] = (float)e2d[a];
                lam[a] = (float)ld[a];
            }
        }
        const float gp[3] = {gout_xyz[3 * i], gout_xyz[3 * i + 1], gout_xyz[3 * i + 2]};
        float rbar[3] = {gp[0], gp[1], gp[2]};
        if (flag & MLS_PT_PLANE_DEGENERATE) {
            // p' = r and the normal is taken as constant: nothing reaches the neighbours
            for (int j = 0; j < k; ++j)
#pragma unroll
                for (int a = 0; a < 3; ++a) edge_grad[(i * k + j) * 3 + a] = 0.f;
        } else {
            const float gn[3] = {gout_n ? gout_n[3 * i] : 0.f, gout_n ? gout_n[3 * i + 1] : 0.f,
                                 gout_n ? gout_n[3 * i + 2] : 0.f};
            const float ofs = nv[0] * m[0] + nv[1] * m[1] + nv[2] * m[2];
            // ---- height-fit moments and the two solves ----
            float mom[15], rhs[6];
#pragma unroll
            for (int c = 0; c < 15; ++c) mom[c] = 0.f;
#pragma unroll
            for (int c = 0; c < 6; ++c) rhs[c] = 0.f;
            for (int j = 0; j < k; ++j) {
                const float4 p = __ldg(xyz4 + my_rows[j * 32 + lane]);
                const float d[3] = {p.x - rx, p.y - ry, p.z - rz};
                const float w = exp2f(fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2])) * neg_scale);
                const float u = (e1[0] * d[0] + e1[1] * d[1] + e1[2] * d[2]) * ih;
                const float v = (e2[0] * d[0] + e2[1] * d[1] + e2[2] * d[2]) * ih;
                const float f = nv[0] * d[0] + nv[1] * d[1] + nv[2] * d[2] - ofs;
                float phi[6];
                basis<DEG>(u, v, phi);
                // moments sum w u^a v^b for a + b <= 2 DEG, in degree blocks
                const float pw[5][5] = {{1.f, v, v * v, v * v * v, v * v * v * v}, {u, u * v, u * v * v, u * v * v * v, 0.f},
                                        {u * u, u * u * v, u * u * v * v, 0.f, 0.f}, {u * u * u, u * u * u * v, 0.f, 0.f, 0.f},
                                        {u * u * u * u, 0.f, 0.f, 0.f, 0.f}};
#pragma unroll
                for (int dg = 0; dg <= 2 * DEG; ++dg)
#pragma unroll
                    for (int bb = 0; bb <= dg; ++bb) mom[dg * (dg + 1) / 2 + bb] = fmaf(w, pw[dg - bb][bb], mom[dg * (dg + 1) / 2 + bb]);
#pragma unroll
                for (int c = 0; c < M; ++c) rhs[c] = fmaf(w * f, phi[c], rhs[c]);
            }
            const float s0bar = gp[0] * nv[0] + gp[1] * nv[1] + gp[2] * nv[2];
            float a[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, z[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            bool ok;
            {
                float A[M][M], b[M], cond = 0.f;
                assemble<float, DEG>(mom, A);
#pragma unroll
                for (int c = 0; c < M; ++c) b[c] = rhs[c];
                float af[M], zf[M];
                ok = factor_and_solve<float, M>(A, b, s0bar, af, zf, cond);
                if (PREC == MLS_PREC_MIXED && (!ok || !(cond < kBwdCondFlag))) {
                    double Ad[M][M], bd[M], ad[M], zd[M], condd;
                    assemble<double, DEG>(mom, Ad);
#pragma unroll
                    for (int c = 0; c < M; ++c) bd[c] = (double)rhs[c];
                    ok = factor_and_solve<double, M>(Ad, bd, (double)s0bar, ad, zd, condd);
#pragma unroll
                    for (int c = 0; c < M; ++c) {
                        af[c] = (float)ad[c];
                        zf[c] = (float)zd[c];
                    }
                }
                if (ok) {
#pragma unroll
                    for (int c = 0; c < M; ++c) {
                        a[c] = af[c];
                        z[c] = zf[c];
                    }
                }
            }
            // ---- reverse: projection, polynomial (global part) ----
            const float s = ofs + a[0];
            float nbar[3], e1bar[3] = {0.f, 0.f, 0.f}, e2bar[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int c = 0; c < 3; ++c) nbar[c] = s * gp[c] + gn[c];
            float ofsbar = s0bar;
            if (ok) {
                for (int j = 0; j < k; ++j) {
                    const float4 p = __ldg(xyz4 + my_rows[j * 32 + lane]);
                    const float d[3] = {p.x - rx, p.y - ry, p.z - rz};
                    const float w = exp2f(fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2])) * neg_scale);
                    const float u = (e1[0] * d[0] + e1[1] * d[1] + e1[2] * d[2]) * ih;
                    const float v = (e2[0] * d[0] + e2[1] * d[1] + e2[2] * d[2]) * ih;
                    const float f = nv[0] * d[0] + nv[1] * d[1] + nv[2] * d[2] - ofs;
                    float phi[6];
                    basis<DEG>(u, v, phi);
                    float g = 0.f, zeta = 0.f;
#pragma unroll
                    for (int c = 0; c < M; ++c) {
                        g = fmaf(phi[c], a[c], g);
                        zeta = fmaf(phi[c], z[c], zeta);
                    }
                    const float res = f - g, fbar = w * zeta;
                    float phibar[6];
#pragma unroll
                    for (int c = 0; c < M; ++c) phibar[c] = w * (res * z[c] - zeta * a[c]);
                    float ubar = 0.f, vbar = 0.f;
                    if (DEG >= 1) {
                        ubar = phibar[1];
                        vbar = phibar[2];
                    }
                    if (DEG >= 2) {
                        ubar += 2.f * u * phibar[3] + v * phibar[4];
                        vbar += u * phibar[4] + 2.f * v * phibar[5];
                    }
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        e1bar[c] = fmaf(ubar * ih, d[c], e1bar[c]);
                        e2bar[c] = fmaf(vbar * ih, d[c], e2bar[c]);
                        nbar[c] = fmaf(fbar, d[c], nbar[c]);
                    }
                    hbar -= (ubar * u + vbar * v) * ih;
                    ofsbar -= fbar;
                }
            }
            // ---- ofs = <n, m>; frame (eigenvector derivative, tilt only) ----
            float mbar[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                nbar[c] = fmaf(ofsbar, m[c], nbar[c]);
                mbar[c] = ofsbar * nv[c];
            }
            float Cb[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
            {
                const float *eb[2] = {e1, e2};
                const float *ebb[2] = {e1bar, e2bar};
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const float gam = (nbar[0] * eb[t][0] + nbar[1] * eb[t][1] + nbar[2] * eb[t][2] -
                                       (ebb[t][0] * nv[0] + ebb[t][1] * nv[1] + ebb[t][2] * nv[2])) /
                                      (lam[0] - lam[t + 1]);
#pragma unroll
                    for (int x = 0; x < 3; ++x)
#pragma unroll
                        for (int y = 0; y < 3; ++y) Cb[x][y] += 0.5f * gam * (eb[t][x] * nv[y] + nv[x] * eb[t][y]);
                }
            }
            // ---- per neighbour: everything that reaches d_j ----
            const float iW = 1.f / W;
            for (int j = 0; j < k; ++j) {
                const float4 p = __ldg(xyz4 + my_rows[j * 32 + lane]);
                const float d[3] = {p.x - rx, p.y - ry, p.z - rz};
                const float dd = fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2]));
                const float w = exp2f(dd * neg_scale);
                float dbar[3] = {0.f, 0.f, 0.f}, wbar = 0.f;
                if (ok) {
                    const float u = (e1[0] * d[0] + e1[1] * d[1] + e1[2] * d[2]) * ih;
                    const float v = (e2[0] * d[0] + e2[1] * d[1] + e2[2] * d[2]) * ih;
                    const float f = nv[0] * d[0] + nv[1] * d[1] + nv[2] * d[2] - ofs;
                    float phi[6];
                    basis<DEG>(u, v, phi);
                    float g = 0.f, zeta = 0.f;
#pragma unroll
                    for (int c = 0; c < M; ++c) {
                        g = fmaf(phi[c], a[c], g);
                        zeta = fmaf(phi[c], z[c], zeta);
                    }
                    const float res = f - g, fbar = w * zeta;
                    float phibar[6];
#pragma unroll
                    for (int c = 0; c < M; ++c) phibar[c] = w * (res * z[c] - zeta * a[c]);
                    float ubar = 0.f, vbar = 0.f;
                    if (DEG >= 1) {
                        ubar = phibar[1];
                        vbar = phibar[2];
                    }
                    if (DEG >= 2) {
                        ubar += 2.f * u * phibar[3] + v * phibar[4];
                        vbar += u * phibar[4] + 2.f * v * phibar[5];
                    }
                    wbar += zeta * res;
#pragma unroll
                    for (int c = 0; c < 3; ++c) dbar[c] = ubar * ih * e1[c] + vbar * ih * e2[c] + fbar * nv[c];
                }
                // covariance about the centroid: C = sum w e e^T, e = d - m
                const float e[3] = {d[0] - m[0], d[1] - m[1], d[2] - m[2]};
                float Ce[3];
#pragma unroll
                for (int x = 0; x < 3; ++x) Ce[x] = Cb[x][0] * e[0] + Cb[x][1] * e[1] + Cb[x][2] * e[2];
                wbar += e[0] * Ce[0] + e[1] * Ce[1] + e[2] * Ce[2];
                // centroid m = sum w d / W
                wbar += (mbar[0] * e[0] + mbar[1] * e[1] + mbar[2] * e[2]) * iW;
                const float wb = wbar * w;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    dbar[c] += 2.f * w * Ce[c] + w * mbar[c] * iW;
                    // weight w = exp(-|d|^2 / h^2)
                    dbar[c] -= 2.f * wb * d[c] / h2;
                    rbar[c] -= dbar[c];
                    edge_grad[(i * k + j) * 3 + c] = dbar[c];
                }
                hbar += 2.f * wb * dd / (h2 * h);
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) self_grad[3 * i + c] = rbar[c];
    }
    // dL/dh of the block, reduced in a fixed order
    double hb = (double)hbar;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) hb += __shfl_xor_sync(0xffffffffu, hb, o);
    if (lane == 0) hred[threadIdx.x >> 5] = hb;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kBwdThreads / 32; ++w) t += hred[w];
        h_part[blockIdx.x] = t;
    }
}

__global__ void k_edge_count(const int32_t *__restrict__ idx, int64_t ne, int32_t *__restrict__ cnt) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[idx[e]], 1);
}

__global__ void k_edge_fill(const int32_t *__restrict__ idx, int64_t ne, const int32_t *__restrict__ off,
                            int32_t *__restrict__ fill, int32_t *__restrict__ ent) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = idx[e];
        ent[off[p] + atomicAdd(&fill[p], 1)] = (int32_t)e;
    }
}

// Sum of the edges that point at p plus p's own term, one warp per target:
// the bucket's edge numbers are sorted (bitonic network over 64 slots, two per
// lane) and summed by a fixed tree over the sorted order, so the result does
// not depend on the order in which the edges were bucketed.  Buckets above 64
// entries (rare hubs) are sorted in place and summed by one lane.
__device__ __forceinline__ void cswap(int &a, int &b, bool up) {
    if ((a > b) == up) {
        const int t = a;
        a = b;
        b = t;
    }
}

__global__ void k_gather(int64_t n, const int32_t *__restrict__ off, int32_t *__restrict__ ent,
                         const float *__restrict__ edge_grad, const float *__restrict__ self_grad,
                         float *__restrict__ grad) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; p < n; p += warps) {
        const int32_t b = off[p], m = off[p + 1] - b;
        float g[3] = {0.f, 0.f, 0.f};
        if (m <= 64) {
            int v0 = 2 * lane < m ? ent[b + 2 * lane] : INT_MAX;
            int v1 = 2 * lane + 1 < m ? ent[b + 2 * lane + 1] : INT_MAX;
            // element e = 2 lane + r
#pragma unroll
            for (int kk = 2; kk <= 64; kk <<= 1) {
#pragma unroll
                for (int j = kk >> 1; j > 0; j >>= 1) {
                    const bool up = ((2 * lane) & kk) == 0;
                    if (j == 1) {
                        cswap(v0, v1, up);
                    } else {
                        const int pl = j >> 1;
                        const int o0 = __shfl_xor_sync(0xffffffffu, v0, pl);
                        const int o1 = __shfl_xor_sync(0xffffffffu, v1, pl);
                        const bool lower = (lane & pl) == 0;
                        v0 = (lower == up) ? min(v0, o0) : max(v0, o0);
                        v1 = (lower == up) ? min(v1, o1) : max(v1, o1);
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float a0 = v0 != INT_MAX ? edge_grad[(int64_t)v0 * 3 + c] : 0.f;
                const float a1 = v1 != INT_MAX ? edge_grad[(int64_t)v1 * 3 + c] : 0.f;
                float t = a0 + a1;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
                g[c] = t;
            }
        } else if (lane == 0) {
            for (int32_t t = b + 1; t < b + m; ++t) {
                const int32_t v = ent[t];
                int32_t u = t;
                while (u > b && ent[u - 1] > v) {
                    ent[u] = ent[u - 1];
                    --u;
                }
                ent[u] = v;
            }
            for (int32_t t = b; t < b + m; ++t)
#pragma unroll
                for (int c = 0; c < 3; ++c) g[c] += edge_grad[(int64_t)ent[t] * 3 + c];
        }
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < 3; ++c) grad[3 * p + c] = self_grad[3 * p + c] + g[c];
    }
}

// dL/dh: the blocks' partial sums, each thread a fixed stride of them, then a
// fixed tree.
__global__ void __launch_bounds__(1024) k_sum_h(const double *__restrict__ part, int m, float *__restrict__ out) {
    __shared__ double red[1024];
    double t = 0.0;
    for (int i = threadIdx.x; i < m; i += 1024) t += part[i];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int s = 512; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = (float)red[0];
}

template <int DEG>
void launch_point(const float4 *xyz4, int64_t n, const int32_t *idx, int k, float h, int precision,
                  const int32_t *order, const float *gp, const float *gn, float *edge, float *self, double *hp,
                  int blocks, cudaStream_t st) {
    const size_t smem = (size_t)k * 32 * sizeof(int32_t) * (kBwdThreads / 32);
    if (precision == MLS_PREC_FP32) {
        auto kern = k_backward_point<DEG, MLS_PREC_FP32>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<blocks, kBwdThreads, smem, st>>>(xyz4, n, idx, k, h, order, gp, gn, edge, self, hp);
    } else {
        auto kern = k_backward_point<DEG, MLS_PREC_MIXED>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<blocks, kBwdThreads, smem, st>>>(xyz4, n, idx, k, h, order, gp, gn, edge, self, hp);
    }
}

}  // namespace

int launch_backward(const float *xyz, int64_t n, const int32_t *idx, int k, float h, int degree, int precision,
                    const int32_t *order, const float *gp, const float *gn, float *grad_xyz, float *grad_h,
                    cudaStream_t st) {
    const int64_t ne = n * k;
    const int blocks = (int)((n + kBwdThreads - 1) / kBwdThreads);
    float4 *xyz4 = nullptr;
    float *edge = nullptr, *self = nullptr;
    double *hp = nullptr;
    int32_t *cnt = nullptr, *off = nullptr, *ent = nullptr;
    MLS_CUDA_TRY(cudaMallocAsync((void **)&xyz4, (size_t)n * sizeof(float4), st));
    MLS_CUDA_TRY(cudaMallocAsync((void **)&edge, (size_t)ne * 3 * sizeof(float), st));
    MLS_CUDA_TRY(cudaMallocAsync((void **)&self, (size_t)n * 3 * sizeof(float), st));
    MLS_CUDA_TRY(cudaMallocAsync((void **)&hp, (size_t)blocks * sizeof(double), st));
    MLS_CUDA_TRY(cudaMallocAsync((void **)&cnt, (size_t)(2 * n + 2) * sizeof(int32_t), st));
    MLS_CUDA_TRY(cudaMallocAsync((void **)&off, (size_t)(n + 1) * sizeof(int32_t), st));
    MLS_CUDA_TRY(cudaMallocAsync((void **)&ent, (size_t)ne * sizeof(int32_t), st));
    int32_t *fill = cnt + n + 1;
    const int gs = (int)std::min<int64_t>((ne + 255) / 256, 152 * 16);
    k_pack4<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, st>>>(xyz, n, xyz4);
    switch (degree) {
        case 0: launch_point<0>(xyz4, n, idx, k, h, precision, order, gp, gn, edge, self, hp, blocks, st); break;
        case 1: launch_point<1>(xyz4, n, idx, k, h, precision, order, gp, gn, edge, self, hp, blocks, st); break;
        default: launch_point<2>(xyz4, n, idx, k, h, precision, order, gp, gn, edge, self, hp, blocks, st); break;
    }
    MLS_CUDA_TRY(cudaMemsetAsync(cnt, 0, (size_t)(2 * n + 2) * sizeof(int32_t), st));
    k_edge_count<<<gs, 256, 0, st>>>(idx, ne, cnt);
    int rc = device_exclusive_scan(cnt, off, n + 1, st);
    if (rc != MLS_OK) return rc;
    k_edge_fill<<<gs, 256, 0, st>>>(idx, ne, off, fill, ent);
    k_gather<<<(int)std::min<int64_t>((n * 32 + 255) / 256, 152 * 32), 256, 0, st>>>(n, off, ent, edge, self, grad_xyz);
    k_sum_h<<<1, 1024, 0, st>>>(hp, blocks, grad_h);
    count_launches(6);
    MLS_CUDA_TRY(cudaGetLastError());
    cudaFreeAsync(xyz4, st);
    cudaFreeAsync(edge, st);
    cudaFreeAsync(self, st);
    cudaFreeAsync(hp, st);
    cudaFreeAsync(cnt, st);
    cudaFreeAsync(off, st);
    cudaFreeAsync(ent, st);
    return MLS_OK;
}

}  // namespace mls
