// Small dense solvers of the per-point fit, shared by the forward and the
// adjoint kernels: cyclic Jacobi for the 3x3 covariance, Cholesky for the
// height-fit normal equations, the frame construction.
#pragma once

#include "common.cuh"

namespace mls {

template <int DEG>
struct Basis {
    static constexpr int M = DEG == 0 ? 1 : (DEG == 1 ? 3 : 6);
};

// Rotation (c, s) of a Jacobi step with theta = (a_qq - a_pp) / (2 a_pq):
// t = sign(theta) / (|theta| + sqrt(theta^2 + 1)), c = 1 / sqrt(t^2 + 1),
// s = t c.  In FP32 with the hardware reciprocal square root and the fast
// quotient (c^2 + s^2 = 1 to a few ulps; the rotations' rounding is then of
// the order of the FP32 moments' own); past |theta| = 2^40 the first-order
// value t = 1 / (2 theta) is exact in float.
__device__ __forceinline__ void jacobi_rotation(float app, float aqq, float apq, float &c, float &s) {
    const float theta = __fdividef(aqq - app, 2.0f * apq);
    const float at = fabsf(theta);
    float t = at > 0x1p40f ? __fdividef(0.5f, at) : __fdividef(1.0f, at + fmaf(theta, theta, 1.0f) * rsqrtf(fmaf(theta, theta, 1.0f)));
    t = theta >= 0.f ? t : -t;
    c = rsqrtf(fmaf(t, t, 1.0f));
    s = t * c;
}
__device__ __forceinline__ void jacobi_rotation(double app, double aqq, double apq, double &c, double &s) {
    const double theta = (aqq - app) / (2.0 * apq);
    const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
    c = 1.0 / sqrt(t * t + 1.0);
    s = t * c;
}

// Cyclic Jacobi on the symmetric 3x3 matrix a (xx, xy, xz, yy, yz, zz).
// Eigenvalues ascending in lam, eigenvectors as columns of V.
template <typename T>
__device__ void jacobi3(const T a6[6], T lam[3], T V[3][3]) {
    T A[3][3] = {{a6[0], a6[1], a6[2]}, {a6[1], a6[3], a6[4]}, {a6[2], a6[4], a6[5]}};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? T(1) : T(0);
    const T tol = sizeof(T) == 4 ? T(1e-15) : T(1e-30);
    for (int sweep = 0; sweep < (sizeof(T) == 4 ? 8 : 20); ++sweep) {
        T off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        T all = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2] + T(2) * off;
        if (off <= tol * all) break;
#pragma unroll
        for (int pq = 0; pq < 3; ++pq) {
            const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
            T apq = A[p][q];
            if (apq == T(0)) continue;
            T c, s;
            jacobi_rotation(A[p][p], A[q][q], apq, c, s);
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                T arp = A[r][p], arq = A[r][q];
                A[r][p] = c * arp - s * arq;
                A[r][q] = s * arp + c * arq;
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                T apr = A[p][r], aqr = A[q][r];
                A[p][r] = c * apr - s * aqr;
                A[q][r] = s * apr + c * aqr;
            }
            A[p][q] = A[q][p] = T(0);
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                T vrp = V[r][p], vrq = V[r][q];
                V[r][p] = c * vrp - s * vrq;
                V[r][q] = s * vrp + c * vrq;
            }
        }
    }
    lam[0] = A[0][0];
    lam[1] = A[1][1];
    lam[2] = A[2][2];
    // sort ascending (three compare-swaps)
#pragma unroll
    for (int pass = 0; pass < 3; ++pass) {
        const int i = pass == 1 ? 1 : 0, j = i + 1;
        if (lam[j] < lam[i]) {
            T tl = lam[i];
            lam[i] = lam[j];
            lam[j] = tl;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                T tv = V[r][i];
                V[r][i] = V[r][j];
                V[r][j] = tv;
            }
        }
    }
}

// Square root and its reciprocal of a positive pivot: in FP32 from the
// hardware reciprocal square root, in FP64 correctly rounded.
__device__ __forceinline__ void root_and_inverse(float d, float &l, float &inv) {
    inv = rsqrtf(d);
    l = d * inv;
}
__device__ __forceinline__ void root_and_inverse(double d, double &l, double &inv) {
    l = sqrt(d);
    inv = 1.0 / l;
}

// Cholesky A = L L^T of an M x M symmetric matrix (lower triangle used),
// with the reciprocals of L's diagonal in invd.  Returns false when a pivot
// is <= rel_tol * trace.  min/max pivot (of L) are returned for the
// conditioning estimate.
template <typename T, int M>
__device__ bool cholesky(const T A[M][M], T L[M][M], T invd[M], T rel_tol, T &pmin, T &pmax) {
    T tr = T(0);
#pragma unroll
    for (int i = 0; i < M; ++i) tr += A[i][i];
    pmin = T(INFINITY);
    pmax = T(0);
    bool ok = true;
#pragma unroll
    for (int j = 0; j < M; ++j) {
        T d = A[j][j];
#pragma unroll
        for (int c = 0; c < j; ++c) d -= L[j][c] * L[j][c];
        if (!(d > rel_tol * tr)) {
            ok = false;
            d = T(1);
        }
        T l, inv;
        root_and_inverse(d, l, inv);
        L[j][j] = l;
        invd[j] = inv;
        pmin = fmin(pmin, l);
        pmax = fmax(pmax, l);
#pragma unroll
        for (int i = j + 1; i < M; ++i) {
            T s = A[i][j];
#pragma unroll
            for (int c = 0; c < j; ++c) s -= L[i][c] * L[j][c];
            L[i][j] = s * inv;
        }
    }
    return ok;
}

template <typename T, int M>
__device__ void chol_solve(const T L[M][M], const T invd[M], const T b[M], T x[M]) {
    T y[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        T s = b[i];
#pragma unroll
        for (int c = 0; c < i; ++c) s -= L[i][c] * y[c];
        y[i] = s * invd[i];
    }
#pragma unroll
    for (int i = M - 1; i >= 0; --i) {
        T s = y[i];
#pragma unroll
        for (int c = i + 1; c < M; ++c) s -= L[c][i] * x[c];
        x[i] = s * invd[i];
    }
}

// Normal matrix and right-hand side from the moments.
// mom: M00 M10 M01 M20 M11 M02 M30 M21 M12 M03 M40 M31 M22 M13 M04 (Mab = sum w u^a v^b)
template <typename T, int DEG>
__device__ void assemble(const float mom[15], T A[Basis<DEG>::M][Basis<DEG>::M]) {
    constexpr int M = Basis<DEG>::M;
    // exponent pairs of the basis monomials
    const int ea[6] = {0, 1, 0, 2, 1, 0}, eb[6] = {0, 0, 1, 0, 1, 2};
#pragma unroll
    for (int r = 0; r < M; ++r)
#pragma unroll
        for (int c = 0; c < M; ++c) {
            const int a = ea[r] + ea[c], b = eb[r] + eb[c], dg = a + b;
            // position of (a, b) in the moment list: degree blocks 1, 2, 3, 4, 5 long
            const int at = dg * (dg + 1) / 2 + b;
            A[r][c] = (T)mom[at];
        }
}

// Solve the height fit A a = b: returns a0 and whether the system was
// singular.  With FULL, also every coefficient a[0..M) and the first column
// of A^-1, c0 = A^-1 e_0 (what the adjoint needs: b-bar = a0-bar c0), both
// zero when singular; a[0] is the returned a0 bit for bit.
template <typename T, int DEG, bool FULL = false>
__device__ T solve_a0(const float mom[15], const float rhs[6], bool refine, bool &singular, T &cond_est,
                      T *a_out = nullptr, T *c0_out = nullptr) {
    constexpr int M = Basis<DEG>::M;
    T A[M][M], L[M][M], invd[M], b[M], x[M];
    assemble<T, DEG>(mom, A);
#pragma unroll
    for (int r = 0; r < M; ++r) b[r] = (T)rhs[r];
    T pmin, pmax;
    singular = !cholesky<T, M>(A, L, invd, T(1e-12), pmin, pmax);
    cond_est = (pmax / pmin) * (pmax / pmin);
    if (singular) {
        if (FULL) {
#pragma unroll
            for (int r = 0; r < M; ++r) a_out[r] = c0_out[r] = T(0);
        }
        return T(0);
    }
    chol_solve<T, M>(L, invd, b, x);
    if (refine) {
        T res[M], dx[M];
#pragma unroll
        for (int r = 0; r < M; ++r) {
            T s = b[r];
#pragma unroll
            for (int c = 0; c < M; ++c) s -= A[r][c] * x[c];
            res[r] = s;
        }
        chol_solve<T, M>(L, invd, res, dx);
#pragma unroll
        for (int r = 0; r < M; ++r) x[r] += dx[r];
    }
    if (FULL) {
        T e0[M];
#pragma unroll
        for (int r = 0; r < M; ++r) {
            e0[r] = r == 0 ? T(1) : T(0);
            a_out[r] = x[r];
        }
        chol_solve<T, M>(L, invd, e0, c0_out);
    }
    return x[0];
}

template <typename T>
__device__ void canonical(T n[3]) {
    int a = 0;
    if (fabs(n[1]) > fabs(n[a])) a = 1;
    if (fabs(n[2]) > fabs(n[a])) a = 2;
    if (n[a] < T(0)) {
        n[0] = -n[0];
        n[1] = -n[1];
        n[2] = -n[2];
    }
}

// Frame from the eigen-decomposition: n = v0 (canonical sign), e1 = v1,
// e2 = n x e1.  Returns the status bit for a degenerate plane.
template <typename T>
__device__ int frame_from(const T C[6], T nrm[3], T e1[3], T e2[3], T lam[3]) {
    T V[3][3];
    jacobi3<T>(C, lam, V);
    nrm[0] = V[0][0];
    nrm[1] = V[1][0];
    nrm[2] = V[2][0];
    e1[0] = V[0][1];
    e1[1] = V[1][1];
    e1[2] = V[2][1];
    canonical(nrm);
    e2[0] = nrm[1] * e1[2] - nrm[2] * e1[1];
    e2[1] = nrm[2] * e1[0] - nrm[0] * e1[2];
    e2[2] = nrm[0] * e1[1] - nrm[1] * e1[0];
    if (!(lam[2] > T(0)) || (lam[1] - lam[0]) <= T(1e-6) * lam[2]) return MLS_PT_PLANE_DEGENERATE;
    return 0;
}

}  // namespace mls
