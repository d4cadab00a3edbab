// The per-point MLS projection (Sec. 1.4, Eq. 1; Algorithm 1) as one device
// routine, shared by the single-cloud kernel and the batched persistent one.
//
// A point is handled by a group of G consecutive lanes (G = 1, 2, 4, 8, 16 or
// 32).  Lane `sub` of the group takes the neighbours j = sub, sub + G, ... .
// Pass 1 gathers each of them once and accumulates the weight, the weighted
// centroid offset and the covariance about it with the weighted online update
// of West (1979): with W' = W + w, delta = d - m: m += delta w / W',
// C += (W w / W') delta delta^T -- as accurate as a second centred pass,
// without storing d.  The G partial states are then merged pairwise with the
// combination rule of Chan, Golub and LeVeque (1979): W = Wa + Wb,
// m = ma + (mb - ma) Wb / W, C = Ca + Cb + (Wa Wb / W) (mb - ma)(mb - ma)^T,
// always with the lower lane's state as `a`, so every lane of the group ends
// with bit-identical moments.  Pass 2 gathers again (now from L1) for the 15
// monomial moments and 6 right-hand sides of the height fit, summed over the
// group with xor shuffles (a + b == b + a exactly, so the sums agree too).
// Every lane of the group then solves the same small systems; the caller
// writes the result from one of them.
#pragma once

#include "solve.cuh"

namespace mls {

constexpr float kMixedGapFlag = 1e-3f;     // FP32 eigensolve trusted above this gap ratio
constexpr float kMixedCondFlag = 1e5f;     // FP32 Cholesky trusted below this condition estimate
// A covariance (unnormalised, weights summing to W) whose largest eigenvalue
// is at most 2^-40 W D^2, D the largest distance from the point to an entry
// of its row, is a degenerate plane: the neighbours' weights are then
// negligible beside the point's own, and FP32 does not resolve the plane
// they would define (eigenvalues near the subnormal range); the point stays.
constexpr float kMinSpread = 0x1p-40f;
// Returned instead of a status when DEFER is set and the point needs an FP64
// step: nothing is computed for it, a later pass runs it without DEFER.
constexpr uint8_t kDeferFP64 = 0x80;

// The fit state a forward pass can save for the adjoint (MLS_FIT_STATE_FLOATS
// floats per point, component c of a point at state[c * stride]): the weight
// sum W, the weighted centroid offset m = c - r, the frame n, e1, e2 and the
// covariance eigenvalues (ascending), the height-fit coefficients a and the
// first column of the inverse normal matrix A^-1 e_0 (zero past M and when
// singular), and the status bits (as the float's bits).
enum FitState : int {
    kStW = 0, kStM = 1, kStN = 4, kStE1 = 7, kStE2 = 10, kStLam = 13, kStA = 16, kStC0 = 22, kStStatus = 28,
    kStFloats = 29
};
static_assert(kStFloats == MLS_FIT_STATE_FLOATS, "fit state layout");

// Row: callable, Row(j) = index of the point's neighbour j.  All 32 lanes of
// the warp must call this together when G > 1 (the merges are warp shuffles,
// and no lane leaves before the last of them); with G = 1 no lane talks to
// another.  Returns the status bits; out = the
// projected point, nf = the normal.
//
// LEVIN selects the weights of Eq. 1 taken about q = r + t n instead of r:
// the plane pass is repeated from t = 0, each time with the weights about
// the q of the previous plane, until t moves by at most tol * h (at most
// max_iter passes, else status bit MLS_PT_NOT_CONVERGED); the height fit
// then uses the weights about the final q.  Points stop after different
// numbers of passes, so LEVIN takes one lane per point (G = 1).
//
// STATE (G = 1, not LEVIN) also writes the point's fit state (FitState) to
// state[c * stride], unless the point is deferred.
template <int DEG, int PREC, bool LEVIN = false, bool DEFER = false, bool STATE = false, class Row>
__device__ __forceinline__ uint8_t project_point(const float4 *__restrict__ xyz4, const Row &row, int k, int sub,
                                                 int G, float h, float rx, float ry, float rz, float out[3],
                                                 float nf[3], int max_iter = 1, float tol = 0.f,
                                                 float *__restrict__ state = nullptr, int64_t stride = 0) {
    static_assert(!(STATE && LEVIN), "the fit state is that of the weights about r");
    // exp(-|d|^2 / h^2) = exp2(-|d|^2 * log2(e) / h^2)
    const float neg_scale = -1.4426950408889634f / (h * h);
    uint8_t st = 0;
    float W, mx, my, mz;
    float D2 = 0.f;                       // the largest squared distance to a row entry
    float e1f[3], e2f[3];
    float lam_s[3] = {0.f, 0.f, 0.f};     // eigenvalues, kept for the state
    // q = r + tq * (qx, qy, qz): the centre of the weights (r unless LEVIN)
    float tq = 0.f, qx = 0.f, qy = 0.f, qz = 0.f;
    for (int it = 0;; ++it) {
        // pass 1: weight W, centroid offset m, covariance C (unnormalised)
        W = 0.f;
        mx = 0.f;
        my = 0.f;
        mz = 0.f;
        float C[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
        for (int j = sub; j < k; j += G) {
            const float4 p = __ldg(xyz4 + row(j));
            const float dx = p.x - rx, dy = p.y - ry, dz = p.z - rz;
            const float dd = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            D2 = fmaxf(D2, dd);
            float w;
            if (LEVIN) {
                const float ax = fmaf(-tq, qx, dx), ay = fmaf(-tq, qy, dy), az = fmaf(-tq, qz, dz);
                w = exp2f(fmaf(ax, ax, fmaf(ay, ay, az * az)) * neg_scale);
            } else {
                w = exp2f(dd * neg_scale);
            }
            const float Wn = W + w;
            const float c = Wn > 0.f ? __fdividef(w, Wn) : 0.f;
            const float ex = dx - mx, ey = dy - my, ez = dz - mz;
            mx = fmaf(ex, c, mx);
            my = fmaf(ey, c, my);
            mz = fmaf(ez, c, mz);
            const float f = W * c;
            const float fx = f * ex, fy = f * ey, fz = f * ez;
            C[0] = fmaf(fx, ex, C[0]);
            C[1] = fmaf(fx, ey, C[1]);
            C[2] = fmaf(fx, ez, C[2]);
            C[3] = fmaf(fy, ey, C[3]);
            C[4] = fmaf(fy, ez, C[4]);
            C[5] = fmaf(fz, ez, C[5]);
            W = Wn;
        }
        for (int s = 1; s < G; s <<= 1) {
            D2 = fmaxf(D2, __shfl_xor_sync(0xffffffffu, D2, s));
            const float Wo = __shfl_xor_sync(0xffffffffu, W, s);
            const float mox = __shfl_xor_sync(0xffffffffu, mx, s);
            const float moy = __shfl_xor_sync(0xffffffffu, my, s);
            const float moz = __shfl_xor_sync(0xffffffffu, mz, s);
            float Co[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) Co[c] = __shfl_xor_sync(0xffffffffu, C[c], s);
            const bool lower = (sub & s) == 0;
            const float Wa = lower ? W : Wo, Wb = lower ? Wo : W;
            const float max_ = lower ? mx : mox, may = lower ? my : moy, maz = lower ? mz : moz;
            const float dx = (lower ? mox : mx) - max_, dy = (lower ? moy : my) - may, dz = (lower ? moz : mz) - maz;
            const float Wn = Wa + Wb;
            const float fb = Wn > 0.f ? __fdividef(Wb, Wn) : 0.f;
            const float g = Wa * fb;
            const float gx = g * dx, gy = g * dy, gz = g * dz;
            float Cs[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) Cs[c] = lower ? C[c] + Co[c] : Co[c] + C[c];
            C[0] = fmaf(gx, dx, Cs[0]);
            C[1] = fmaf(gx, dy, Cs[1]);
            C[2] = fmaf(gx, dz, Cs[2]);
            C[3] = fmaf(gy, dy, Cs[3]);
            C[4] = fmaf(gy, dz, Cs[4]);
            C[5] = fmaf(gz, dz, Cs[5]);
            mx = fmaf(dx, fb, max_);
            my = fmaf(dy, fb, may);
            mz = fmaf(dz, fb, maz);
            W = Wn;
        }
        {
            float lam[3];
            int deg_flag = frame_from<float>(C, nf, e1f, e2f, lam);
            if (STATE) {
#pragma unroll
                for (int a = 0; a < 3; ++a) lam_s[a] = lam[a];
            }
            // the FP32 eigenvector error grows like eps * l2 / (l1 - l0): in the
            // mixed form, narrow gaps are solved again in FP64 from the same moments
            if (PREC == MLS_PREC_MIXED && (!(lam[2] > 0.f) || (lam[1] - lam[0]) < kMixedGapFlag * lam[2])) {
                if (DEFER) return kDeferFP64;
                double Cd[6], nd[3], e1d[3], e2d[3], ld[3];
#pragma unroll
                for (int c = 0; c < 6; ++c) Cd[c] = (double)C[c];
                deg_flag = frame_from<double>(Cd, nd, e1d, e2d, ld);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    nf[a] = (float)nd[a];
                    e1f[a] = (float)e1d[a];
                    e2f[a] = (float)e2d[a];
                    lam[a] = (float)ld[a];
                    if (STATE) lam_s[a] = (float)ld[a];
                }
                st |= MLS_PT_FP64_USED;
            }
            if (!(lam[2] > kMinSpread * W * D2)) deg_flag = MLS_PT_PLANE_DEGENERATE;
            st = (uint8_t)((st & ~MLS_PT_PLANE_DEGENERATE) | deg_flag);
        }
        if (!LEVIN || (st & MLS_PT_PLANE_DEGENERATE)) break;
        {
            // q of this plane: the projection of r onto it
            const float tn = nf[0] * mx + nf[1] * my + nf[2] * mz;
            const bool done = it > 0 && fabsf(tn - tq) <= tol * h;
            tq = tn;
            qx = nf[0];
            qy = nf[1];
            qz = nf[2];
            if (done) break;
            if (it + 1 >= max_iter) {
                st |= MLS_PT_NOT_CONVERGED;
                break;
            }
        }
    }
    out[0] = rx;
    out[1] = ry;
    out[2] = rz;
    // a degenerate plane leaves the point where it is; its lanes still take
    // part in the group's shuffles below, with nothing accumulated
    const bool degenerate = (st & MLS_PT_PLANE_DEGENERATE) != 0;
    const float ofs = nf[0] * mx + nf[1] * my + nf[2] * mz;
    const float ih = 1.f / h;
    const float a1x = e1f[0] * ih, a1y = e1f[1] * ih, a1z = e1f[2] * ih;
    const float a2x = e2f[0] * ih, a2y = e2f[1] * ih, a2z = e2f[2] * ih;
    // pass 2: moments of the height fit
    float mom[15], rhs[6];
#pragma unroll
    for (int c = 0; c < 15; ++c) mom[c] = 0.f;
#pragma unroll
    for (int c = 0; c < 6; ++c) rhs[c] = 0.f;
#pragma unroll 2
    for (int j = degenerate ? k : sub; j < k; j += G) {
        const float4 p = __ldg(xyz4 + row(j));
        const float dx = p.x - rx, dy = p.y - ry, dz = p.z - rz;
        float w;
        if (LEVIN) {   // about the final q = r + ofs n
            const float ax = fmaf(-ofs, nf[0], dx), ay = fmaf(-ofs, nf[1], dy), az = fmaf(-ofs, nf[2], dz);
            w = exp2f(fmaf(ax, ax, fmaf(ay, ay, az * az)) * neg_scale);
        } else {
            w = exp2f(fmaf(dx, dx, fmaf(dy, dy, dz * dz)) * neg_scale);
        }
        const float f = fmaf(nf[2], dz, fmaf(nf[1], dy, fmaf(nf[0], dx, -ofs)));
        const float wf = w * f;
        mom[0] += w;
        rhs[0] += wf;
        if (DEG >= 1) {
            const float u = fmaf(a1z, dz, fmaf(a1y, dy, a1x * dx));
            const float vv = fmaf(a2z, dz, fmaf(a2y, dy, a2x * dx));
            const float wu = w * u, wv = w * vv;
            mom[1] += wu;
            mom[2] += wv;
            rhs[1] = fmaf(wf, u, rhs[1]);
            rhs[2] = fmaf(wf, vv, rhs[2]);
            const float wuu = wu * u, wuv = wu * vv, wvv = wv * vv;
            mom[3] += wuu;
            mom[4] += wuv;
            mom[5] += wvv;
            if (DEG >= 2) {
                const float uu = u * u, uv = u * vv, v2 = vv * vv;
                mom[6] = fmaf(wuu, u, mom[6]);
                mom[7] = fmaf(wuu, vv, mom[7]);
                mom[8] = fmaf(wvv, u, mom[8]);
                mom[9] = fmaf(wvv, vv, mom[9]);
                mom[10] = fmaf(wuu, uu, mom[10]);
                mom[11] = fmaf(wuu, uv, mom[11]);
                mom[12] = fmaf(wuu, v2, mom[12]);
                mom[13] = fmaf(wvv, uv, mom[13]);
                mom[14] = fmaf(wvv, v2, mom[14]);
                rhs[3] = fmaf(wf, uu, rhs[3]);
                rhs[4] = fmaf(wf, uv, rhs[4]);
                rhs[5] = fmaf(wf, v2, rhs[5]);
            }
        }
    }
    for (int s = 1; s < G; s <<= 1) {
#pragma unroll
        for (int c = 0; c < 15; ++c) mom[c] += __shfl_xor_sync(0xffffffffu, mom[c], s);
#pragma unroll
        for (int c = 0; c < 6; ++c) rhs[c] += __shfl_xor_sync(0xffffffffu, rhs[c], s);
    }
    constexpr int M = Basis<DEG>::M;
    float a_s[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, c0_s[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    // the state of the point (status st, coefficients a_s, column c0_s)
    auto save = [&]() {
        if (!STATE) return;
        const float v[kStFloats] = {W, mx, my, mz, nf[0], nf[1], nf[2], e1f[0], e1f[1], e1f[2], e2f[0], e2f[1],
                                    e2f[2], lam_s[0], lam_s[1], lam_s[2], a_s[0], a_s[1], a_s[2], a_s[3], a_s[4],
                                    a_s[5], c0_s[0], c0_s[1], c0_s[2], c0_s[3], c0_s[4], c0_s[5],
                                    __int_as_float((int)st)};
#pragma unroll
        for (int c = 0; c < kStFloats; ++c) state[c * stride] = v[c];
    };
    if (degenerate) {
        save();
        return st;
    }
    bool singular;
    float cond;
    float a0 = solve_a0<float, DEG, STATE>(mom, rhs, true, singular, cond, a_s, c0_s);
    if (PREC == MLS_PREC_MIXED && (singular || !(cond < kMixedCondFlag))) {
        if (DEFER) return kDeferFP64;
        double condd, ad[6], cd[6];
        a0 = (float)solve_a0<double, DEG, STATE>(mom, rhs, false, singular, condd, ad, cd);
        if (STATE) {
#pragma unroll
            for (int r = 0; r < M; ++r) {
                a_s[r] = (float)ad[r];
                c0_s[r] = (float)cd[r];
            }
        }
        st |= MLS_PT_FP64_USED;
    }
    if (singular) {
        st |= MLS_PT_POLY_SINGULAR;
        a0 = 0.f;
    }
    save();
    const float s = ofs + a0;
    out[0] = fmaf(s, nf[0], rx);
    out[1] = fmaf(s, nf[1], ry);
    out[2] = fmaf(s, nf[2], rz);
    return st;
}

}  // namespace mls
