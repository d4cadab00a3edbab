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
// that neighbour's bucket of a reverse adjacency (bucket sizes are counted
// from the neighbour rows beforehand), and the gradient of its own position
// separately.  Each bucket, with its point's own term, is then summed exactly
// in 64-bit fixed point (a per-bucket, per-component power-of-two scale from
// the largest magnitude) and rounded once: the sum does not depend on the
// order in which the records reached the bucket, so results do not depend on
// scheduling or on the processing order.
//
// Everything is indexed by sorted (grid order) position when a processing order
// is given: point slot s of the order sends its records to the sorted
// positions of its neighbours.  Neighbours are close in that order, so the
// bucket writes of a block touch a narrow window of memory at a time.
#include <algorithm>
#include <climits>

#include "fixed_point.cuh"
#include "project_point.cuh"

namespace mls {

int device_exclusive_scan(const int32_t *in, int32_t *out, int64_t n, cudaStream_t st);

namespace {

constexpr int kBwdThreads = 128;
constexpr int kSumLanes = 4;        // lanes per bucket in the bucket sum (at least 3: one per component written)
constexpr int kSumCached = 9;       // values per lane held in registers there
constexpr float kBwdGapFlag = 1e-3f;
constexpr float kBwdCondFlag = 1e5f;

// The points as float4, in processing order when one is given (xyz4[s] is
// point order[s]): the neighbours of nearby points then lie close together in
// memory, which the neighbour gathers' caches reward.
__global__ void k_pack4(const float *__restrict__ xyz, int64_t n, const int32_t *__restrict__ order,
                        float4 *__restrict__ xyz4) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = order ? (int64_t)__ldg(order + s) : s;
        xyz4[s] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], 0.f);
    }
}

template <typename T, int M>
__device__ bool factor_and_solve(const T A[M][M], const T b[M], const T e0bar, T a[M], T z[M], T &cond) {
    T L[M][M], invd[M], pmin, pmax;
    if (!cholesky<T, M>(A, L, invd, T(1e-12), pmin, pmax)) return false;
    cond = (pmax / pmin) * (pmax / pmin);
    chol_solve<T, M>(L, invd, b, a);
    T rhs[M];
#pragma unroll
    for (int r = 0; r < M; ++r) rhs[r] = r == 0 ? e0bar : T(0);
    chol_solve<T, M>(L, invd, rhs, z);
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

// Six blocks per SM (80 registers): the kernel waits on its neighbour gathers,
// and more resident warps hide more of that latency than the spills cost.
// With SORTED, xyz4 is the grid's sorted copy of the points, slot s is sorted
// position s, idx holds rows of sorted positions by sorted position (no
// translation), and order[s] is the point's original index.
// With STATE (SORTED only), the frame, eigenvalues, centroid offset, weight
// sum, fit coefficients, A^-1 e_0 and status of sorted position s come from
// state[c * n + s] (FitState, saved by the forward): the recompute passes and
// solves are skipped, and z = a0-bar A^-1 e_0.
template <int DEG, int PREC, bool SORTED = false, bool STATE = false>
__global__ void __launch_bounds__(kBwdThreads, 6) k_backward_point(
    const float4 *__restrict__ xyz4, int64_t n, const int32_t *__restrict__ idx, int k, float h,
    const int32_t *__restrict__ order, const int32_t *__restrict__ pos, const float *__restrict__ gout_xyz,
    const float *__restrict__ gout_n, const int32_t *__restrict__ off, int32_t *__restrict__ fill,
    float4 *__restrict__ rec, float4 *__restrict__ self4, double *__restrict__ h_part,
    const float *__restrict__ state = nullptr) {
    static_assert(!STATE || SORTED, "the fit state is indexed by sorted position");
    constexpr int M = Basis<DEG>::M;
    extern __shared__ int32_t rows[];
    __shared__ double hred[kBwdThreads / 32];
    const int lane = threadIdx.x & 31;
    int32_t *my_rows = rows + (threadIdx.x >> 5) * k * kRowStride;
    const int64_t slot = blockIdx.x * (int64_t)kBwdThreads + threadIdx.x;
    const int64_t warp_base = slot - lane;
    const int64_t i = slot < n ? (order ? (int64_t)__ldg(order + slot) : slot) : -1;
    const int64_t row_of = SORTED ? slot : i;
    const int nrows = (int)min((int64_t)32, n - warp_base);
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
        const int64_t i_r = __shfl_sync(0xffffffffu, row_of, r);
        if (r < nrows)
            for (int c = lane; c < k; c += 32) {
                // the rows as sorted positions (xyz4 is in processing order)
                const int32_t p = __ldg(idx + i_r * k + c);
                my_rows[c * kRowStride + r] = (!SORTED && pos) ? __ldg(pos + p) : p;
            }
    }
    __syncwarp();
    float hbar = 0.f;
    if (slot < n) {
        const float4 r4 = __ldg(xyz4 + slot);
        const float rx = r4.x, ry = r4.y, rz = r4.z;
        const float h2 = h * h, ih = 1.f / h;
        const float neg_scale = -1.4426950408889634f / h2;
        float W = 0.f, m[3] = {0.f, 0.f, 0.f};
        float nv[3], e1[3], e2[3], lam[3];
        int flag = 0;
        if constexpr (STATE) {
            const float *sv = state + slot;
            W = __ldg(sv + kStW * n);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                m[a] = __ldg(sv + (kStM + a) * n);
                nv[a] = __ldg(sv + (kStN + a) * n);
                e1[a] = __ldg(sv + (kStE1 + a) * n);
                e2[a] = __ldg(sv + (kStE2 + a) * n);
                lam[a] = __ldg(sv + (kStLam + a) * n);
            }
            flag = __float_as_int(__ldg(sv + kStStatus * n));
        } else {
        // ---- forward recompute: weights, centroid offset, covariance ----
        float C[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        float D2 = 0.f;     // the largest squared distance to a row entry
        for (int j = 0; j < k; ++j) {
            const float4 p = __ldg(xyz4 + my_rows[j * kRowStride + lane]);
            const float d[3] = {p.x - rx, p.y - ry, p.z - rz};
            const float dd = fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2]));
            D2 = fmaxf(D2, dd);
            const float w = exp2f(dd * neg_scale);
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
        flag = frame_from<float>(C, nv, e1, e2, lam);
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
        if (!(lam[2] > kMinSpread * W * D2)) flag = MLS_PT_PLANE_DEGENERATE;
        }
        const float gp[3] = {gout_xyz[3 * i], gout_xyz[3 * i + 1], gout_xyz[3 * i + 2]};
        float rbar[3] = {gp[0], gp[1], gp[2]};
        // a free place in the bucket of neighbour j (its sorted position)
        auto bucket_slot = [&](int j) {
            const int32_t t = my_rows[j * kRowStride + lane];
            return __ldg(off + t) + atomicAdd(fill + t, 1);
        };
        if (flag & MLS_PT_PLANE_DEGENERATE) {
            // p' = r and the normal is taken as constant: nothing reaches the neighbours
            for (int j = 0; j < k; ++j) rec[bucket_slot(j)] = make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            const float gn[3] = {gout_n ? gout_n[3 * i] : 0.f, gout_n ? gout_n[3 * i + 1] : 0.f,
                                 gout_n ? gout_n[3 * i + 2] : 0.f};
            const float ofs = nv[0] * m[0] + nv[1] * m[1] + nv[2] * m[2];
            const float s0bar = gp[0] * nv[0] + gp[1] * nv[1] + gp[2] * nv[2];
            float a[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, z[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            bool ok;
            if constexpr (STATE) {
                ok = !(flag & MLS_PT_POLY_SINGULAR);
                const float *sv = state + slot;
#pragma unroll
                for (int c = 0; c < M; ++c) {
                    a[c] = __ldg(sv + (kStA + c) * n);
                    z[c] = s0bar * __ldg(sv + (kStC0 + c) * n);
                }
            } else {
            // ---- height-fit moments and the two solves ----
            float mom[15], rhs[6];
#pragma unroll
            for (int c = 0; c < 15; ++c) mom[c] = 0.f;
#pragma unroll
            for (int c = 0; c < 6; ++c) rhs[c] = 0.f;
            for (int j = 0; j < k; ++j) {
                const float4 p = __ldg(xyz4 + my_rows[j * kRowStride + lane]);
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
            }
            // ---- reverse: projection, polynomial (global part) ----
            const float s = ofs + a[0];
            float nbar[3], e1bar[3] = {0.f, 0.f, 0.f}, e2bar[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int c = 0; c < 3; ++c) nbar[c] = s * gp[c] + gn[c];
            float ofsbar = s0bar;
            if (ok) {
                for (int j = 0; j < k; ++j) {
                    const float4 p = __ldg(xyz4 + my_rows[j * kRowStride + lane]);
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
                const int32_t at = bucket_slot(j);      // taken early: its latency overlaps the arithmetic
                const float4 p = __ldg(xyz4 + my_rows[j * kRowStride + lane]);
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
                }
                rec[at] = make_float4(dbar[0], dbar[1], dbar[2], 0.f);
                hbar += 2.f * wb * dd / (h2 * h);
            }
        }
        self4[slot] = make_float4(rbar[0], rbar[1], rbar[2], 0.f);
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

// Inverse of the processing order: pos[order[s]] = s.
__global__ void k_inverse(const int32_t *__restrict__ order, int64_t n, int32_t *__restrict__ pos) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
        pos[order[s]] = (int32_t)s;
}

// Bucket sizes: the number of row entries naming each point (at its sorted
// position).
__global__ void k_count(const int32_t *__restrict__ idx, int64_t ne, const int32_t *__restrict__ pos,
                        int32_t *__restrict__ cnt) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = __ldg(idx + e);
        atomicAdd(cnt + (pos ? __ldg(pos + p) : p), 1);
    }
}

// The same counts with a processing order: a block takes the rows of
// kCountSlots consecutive sorted positions, whose neighbours mostly lie within
// a window of kCountWindow sorted positions around them; those are counted in
// shared memory and added to the global counts once per block, the rest
// directly.
constexpr int kCountSlots = 256;
constexpr int kCountWindow = 4096;

// With SORTED, idx holds rows of sorted positions by sorted position (order
// and pos unused).
template <bool SORTED = false>
__global__ void __launch_bounds__(256) k_count_window(const int32_t *__restrict__ idx, int64_t n, int k,
                                                      const int32_t *__restrict__ order,
                                                      const int32_t *__restrict__ pos, int32_t *__restrict__ cnt) {
    __shared__ int32_t win[kCountWindow];
    const int64_t s0 = (int64_t)blockIdx.x * kCountSlots;
    const int64_t lo = s0 + kCountSlots / 2 - kCountWindow / 2;
    for (int w = threadIdx.x; w < kCountWindow; w += blockDim.x) win[w] = 0;
    __syncthreads();
    const int edges = (int)(min(n, s0 + kCountSlots) - s0) * k;
    for (int e = threadIdx.x; e < edges; e += blockDim.x) {
        const int64_t slot = s0 + e / k;
        const int32_t t = SORTED ? __ldg(idx + slot * k + e % k)
                                 : __ldg(pos + __ldg(idx + (int64_t)__ldg(order + slot) * k + e % k));
        const int64_t w = (int64_t)t - lo;
        if (w >= 0 && w < kCountWindow)
            atomicAdd(win + w, 1);
        else
            atomicAdd(cnt + t, 1);
    }
    __syncthreads();
    for (int w = threadIdx.x; w < kCountWindow; w += blockDim.x) {
        const int32_t c = win[w];
        if (c) atomicAdd(cnt + (lo + w), c);      // c > 0 only for positions in [0, n)
    }
}

// 2^e as a float, e in [-126, 127].
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

// The integer q 2^-s, rounded once to float.
__device__ __forceinline__ float from_fixed(long long q, int s) {
    float x = __ll2float_rn(q);
    if (s > 120) {
        x *= pow2f(-120);
        s -= 120;
    }
    return x * pow2f(-s);
}

// Sum of the records in t's bucket plus t's own term, G lanes per point (a
// warp sums 32 / G consecutive buckets, which are adjacent in memory), the
// first V x G values held in registers.  Per component: the largest
// magnitude M = m 2^E (m in [1, 2)) over the bucket's c values fixes the scale
// 2^s, s = 61 - E - ceil(log2 c), so that every scaled value is below
// 2^(62 - ceil(log2 c)) and the integer sum below 2^62; each value is rounded
// to an integer once (an error below 2^-s, that is 2^-60 M or less), the
// integers are summed exactly, and the total is rounded once to float.
// Non-finite components are summed in float.  The largest magnitude is taken
// over the bit patterns with the sign cleared, which order non-negative
// floats and put infinities and NaNs above every finite value.
template <int G, int V>
__global__ void __launch_bounds__(256) k_bucket_sum(int64_t n, const int32_t *__restrict__ order,
                                                    const int32_t *__restrict__ off, const float4 *__restrict__ rec,
                                                    const float4 *__restrict__ self4, float *__restrict__ grad) {
    static_assert(G >= 3 && G <= 32 && 32 % G == 0, "G lanes per point, one per written component");
    constexpr int P = 32 / G;     // points per warp
    constexpr uint32_t kAbs = 0x7fffffffu, kInf = 0x7f800000u;
    const int lane = threadIdx.x & 31, sub = lane % G;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t t0 = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * P; t0 < n; t0 += warps * P) {
        const int64_t t = t0 + lane / G;
        const bool live = t < n;
        const int32_t b = live ? __ldg(off + t) : 0;
        const int32_t m = live ? __ldg(off + t + 1) - b : 0;
        const int c = live ? m + 1 : 0;    // the records and the point's own term (value number m)
        auto value = [&](int e) { return e < m ? __ldg(rec + b + e) : __ldg(self4 + t); };
        float4 v[V];
#pragma unroll
        for (int r = 0; r < V; ++r) {
            const int e = r * G + sub;
            v[r] = e < c ? value(e) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        uint32_t mb[3] = {0u, 0u, 0u};
        auto take = [&](float4 a) {
            mb[0] = max(mb[0], __float_as_uint(a.x) & kAbs);
            mb[1] = max(mb[1], __float_as_uint(a.y) & kAbs);
            mb[2] = max(mb[2], __float_as_uint(a.z) & kAbs);
        };
#pragma unroll
        for (int r = 0; r < V; ++r) take(v[r]);
        for (int e = V * G + sub; e < c; e += G) take(value(e));
        const int lc = c > 1 ? 32 - __clz(c - 1) : 0;     // ceil(log2 c)
        float out[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) mb[a] = max(mb[a], __shfl_xor_sync(0xffffffffu, mb[a], o));
        }
        const bool finite = mb[0] < kInf && mb[1] < kInf && mb[2] < kInf;
        if (finite) {
            int sh[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int E = max((int)(mb[a] >> 23) - 127, -126);
                sh[a] = 61 - E - lc;
            }
            long long q[3] = {0, 0, 0};
            auto add = [&](float4 a) {
                q[0] += to_fixed(a.x, sh[0]);
                q[1] += to_fixed(a.y, sh[1]);
                q[2] += to_fixed(a.z, sh[2]);
            };
#pragma unroll
            for (int r = 0; r < V; ++r) add(v[r]);
            for (int e = V * G + sub; e < c; e += G) add(value(e));
#pragma unroll
            for (int a = 0; a < 3; ++a) {
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) q[a] += __shfl_xor_sync(0xffffffffu, q[a], o);
                out[a] = from_fixed(q[a], sh[a]);
            }
        } else {
            float fs[3] = {0.f, 0.f, 0.f};
            for (int e = sub; e < c; e += G) {
                const float4 a = value(e);
                fs[0] += a.x;
                fs[1] += a.y;
                fs[2] += a.z;
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) {
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) fs[a] += __shfl_xor_sync(0xffffffffu, fs[a], o);
                out[a] = fs[a];
            }
        }
        if (live && sub < 3) {
            const int64_t o = order ? (int64_t)order[t] : t;
            grad[3 * o + sub] = sub == 0 ? out[0] : (sub == 1 ? out[1] : out[2]);
        }
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

template <int DEG, bool SORTED = false, bool STATE = false>
void launch_point(const float4 *xyz4, int64_t n, const int32_t *idx, int k, float h, int precision,
                  const int32_t *order, const int32_t *pos, const float *gp, const float *gn, const int32_t *off,
                  int32_t *fill, float4 *rec, float4 *self4, double *hp, int blocks, cudaStream_t st,
                  const float *state = nullptr) {
    const size_t smem = (size_t)k * kRowStride * sizeof(int32_t) * (kBwdThreads / 32);
    auto kern = precision == MLS_PREC_FP32 ? k_backward_point<DEG, MLS_PREC_FP32, SORTED, STATE>
                                           : k_backward_point<DEG, MLS_PREC_MIXED, SORTED, STATE>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<blocks, kBwdThreads, smem, st>>>(xyz4, n, idx, k, h, order, pos, gp, gn, off, fill, rec, self4, hp,
                                            state);
}

}  // namespace

int launch_backward(const float *xyz, int64_t n, const int32_t *idx, int k, float h, int degree, int precision,
                    const int32_t *order, const float *gp, const float *gn, float *grad_xyz, float *grad_h,
                    cudaStream_t st) {
    const int64_t ne = n * (int64_t)k;
    const int blocks = (int)((n + kBwdThreads - 1) / kBwdThreads);
    float4 *xyz4 = nullptr, *rec = nullptr, *self4 = nullptr;
    double *hp = nullptr;
    int32_t *cnt = nullptr, *off = nullptr, *pos = nullptr;
    ScratchSet scratch(st);     // every buffer freed on every return below
    MLS_CUDA_TRY(scratch.alloc(&xyz4, (size_t)n * sizeof(float4)));
    MLS_CUDA_TRY(scratch.alloc(&rec, (size_t)ne * sizeof(float4)));
    MLS_CUDA_TRY(scratch.alloc(&self4, (size_t)n * sizeof(float4)));
    MLS_CUDA_TRY(scratch.alloc(&hp, (size_t)blocks * sizeof(double)));
    MLS_CUDA_TRY(scratch.alloc(&cnt, (size_t)(2 * n + 2) * sizeof(int32_t)));
    MLS_CUDA_TRY(scratch.alloc(&off, (size_t)(n + 1) * sizeof(int32_t)));
    if (order) MLS_CUDA_TRY(scratch.alloc(&pos, (size_t)n * sizeof(int32_t)));
    int32_t *fill = cnt + n + 1;
    const int sms = sm_count();
    const int grid_n = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 16);
    MLS_CUDA_TRY(cudaMemsetAsync(cnt, 0, (size_t)(2 * n + 2) * sizeof(int32_t), st));
    k_pack4<<<grid_n, 256, 0, st>>>(xyz, n, order, xyz4);
    int launches = 1;
    if (order) {
        MLS_CUDA_TRY(cudaMemsetAsync(pos, 0, (size_t)n * sizeof(int32_t), st));   // in range for any order
        k_inverse<<<grid_n, 256, 0, st>>>(order, n, pos);
        ++launches;
    }
    if (order)
        k_count_window<false><<<(int)((n + kCountSlots - 1) / kCountSlots), 256, 0, st>>>(idx, n, k, order, pos, cnt);
    else
        k_count<<<(int)std::min<int64_t>((ne + 255) / 256, (int64_t)sms * 32), 256, 0, st>>>(idx, ne, pos, cnt);
    int rc = device_exclusive_scan(cnt, off, n + 1, st);
    if (rc != MLS_OK) return rc;
    switch (degree) {
        case 0: launch_point<0>(xyz4, n, idx, k, h, precision, order, pos, gp, gn, off, fill, rec, self4, hp, blocks, st); break;
        case 1: launch_point<1>(xyz4, n, idx, k, h, precision, order, pos, gp, gn, off, fill, rec, self4, hp, blocks, st); break;
        default: launch_point<2>(xyz4, n, idx, k, h, precision, order, pos, gp, gn, off, fill, rec, self4, hp, blocks, st); break;
    }
    k_bucket_sum<kSumLanes, kSumCached><<<(int)std::min<int64_t>((n * kSumLanes + 255) / 256, (int64_t)sms * 32), 256, 0, st>>>(
        n, order, off, rec, self4, grad_xyz);
    k_sum_h<<<1, 1024, 0, st>>>(hp, blocks, grad_h);
    count_launches(launches + 4);   // + count, point, bucket sum, sum_h (the scan counts its own)
    MLS_CUDA_TRY(cudaGetLastError());
    return MLS_OK;
}

// The offsets of the adjoint's reverse adjacency for rows of sorted
// positions: off[t] = how many row entries name sorted positions below t
// (n + 1 int32).
int launch_backward_offsets(const int32_t *rows, int64_t n, int k, int32_t *off, cudaStream_t st) {
    int32_t *cnt = nullptr;
    ScratchSet scratch(st);
    MLS_CUDA_TRY(scratch.alloc(&cnt, (size_t)(n + 1) * sizeof(int32_t)));
    MLS_CUDA_TRY(cudaMemsetAsync(cnt, 0, (size_t)(n + 1) * sizeof(int32_t), st));
    k_count_window<true><<<(int)((n + kCountSlots - 1) / kCountSlots), 256, 0, st>>>(rows, n, k, nullptr, nullptr,
                                                                                      cnt);
    count_launches(1);
    MLS_CUDA_TRY(cudaGetLastError());
    return device_exclusive_scan(cnt, off, n + 1, st);
}

int launch_backward_sorted(const float4 *pts, const int32_t *order, int64_t n, const int32_t *rows, int k, float h,
                           int degree, int precision, const float *gp, const float *gn, float *grad_xyz,
                           float *grad_h, const float *state, const int32_t *offsets, cudaStream_t st) {
    const int64_t ne = n * (int64_t)k;
    const int blocks = (int)((n + kBwdThreads - 1) / kBwdThreads);
    float4 *rec = nullptr, *self4 = nullptr;
    double *hp = nullptr;
    int32_t *fill = nullptr, *own_off = nullptr;
    ScratchSet scratch(st);     // every buffer freed on every return below
    MLS_CUDA_TRY(scratch.alloc(&rec, (size_t)ne * sizeof(float4)));
    MLS_CUDA_TRY(scratch.alloc(&self4, (size_t)n * sizeof(float4)));
    MLS_CUDA_TRY(scratch.alloc(&hp, (size_t)blocks * sizeof(double)));
    MLS_CUDA_TRY(scratch.alloc(&fill, (size_t)(n + 1) * sizeof(int32_t)));
    const int sms = sm_count();
    MLS_CUDA_TRY(cudaMemsetAsync(fill, 0, (size_t)(n + 1) * sizeof(int32_t), st));
    // the bucket offsets: the caller's (counted beside the forward), else here
    const int32_t *off = offsets;
    if (!off) {
        MLS_CUDA_TRY(scratch.alloc(&own_off, (size_t)(n + 1) * sizeof(int32_t)));
        const int rc = launch_backward_offsets(rows, n, k, own_off, st);
        if (rc != MLS_OK) return rc;
        off = own_off;
    }
    if (state) {
        switch (degree) {
            case 0: launch_point<0, true, true>(pts, n, rows, k, h, precision, order, nullptr, gp, gn, off, fill, rec, self4, hp, blocks, st, state); break;
            case 1: launch_point<1, true, true>(pts, n, rows, k, h, precision, order, nullptr, gp, gn, off, fill, rec, self4, hp, blocks, st, state); break;
            default: launch_point<2, true, true>(pts, n, rows, k, h, precision, order, nullptr, gp, gn, off, fill, rec, self4, hp, blocks, st, state); break;
        }
    } else {
        switch (degree) {
            case 0: launch_point<0, true>(pts, n, rows, k, h, precision, order, nullptr, gp, gn, off, fill, rec, self4, hp, blocks, st); break;
            case 1: launch_point<1, true>(pts, n, rows, k, h, precision, order, nullptr, gp, gn, off, fill, rec, self4, hp, blocks, st); break;
            default: launch_point<2, true>(pts, n, rows, k, h, precision, order, nullptr, gp, gn, off, fill, rec, self4, hp, blocks, st); break;
        }
    }
    k_bucket_sum<kSumLanes, kSumCached><<<(int)std::min<int64_t>((n * kSumLanes + 255) / 256, (int64_t)sms * 32), 256, 0, st>>>(
        n, order, off, rec, self4, grad_xyz);
    k_sum_h<<<1, 1024, 0, st>>>(hp, blocks, grad_h);
    count_launches(3);   // point, bucket sum, sum_h (the offsets count their own)
    MLS_CUDA_TRY(cudaGetLastError());
    return MLS_OK;
}

}  // namespace mls
