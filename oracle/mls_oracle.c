/*
 * mls_oracle.c -- plain, single-threaded FP64 CPU oracle for the per-point
 * moving least squares (MLS) projection.
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg load this library.  It shares no
 * code, header, table or helper with the CUDA path; the two meet only in the
 * seeded input generators.
 *
 * What it computes, and where the paper defines it:
 *   - Sec. 1.4 (Moving least squares method), Eq. 1: the reference plane H is
 *     the weighted least-squares plane of the neighbours; the query is moved
 *     to its projection q on H, a local orthonormal frame is set on H with q as
 *     origin, and a local polynomial of the heights is fitted over H.
 *   - Sec. 2.1 (Proposed parallel method), Algorithm 1: per point, build the
 *     plane, fit the local height polynomial g, and return the projection of
 *     the point onto g.
 *   - Sec. 2.2 (Computational complexity) names the neighbour search that
 *     precedes each fit; the paper uses a radius R and a k-d tree.
 *
 * Readings where the paper is silent or incomplete:
 *   - neighbourhood = the k nearest points, self included, ranked by a fixed
 *     FP32 key (oracle_knn_key below) with ties broken by the lower point index;
 *   - weight theta(d) = exp(-d^2 / h^2), taken about the query r and used for
 *     both the plane and the polynomial;
 *   - plane normal = eigenvector of the smallest eigenvalue of the weighted
 *     covariance about the weighted centroid; canonical sign: the component of
 *     largest magnitude is positive (ties: lowest axis);
 *   - polynomial = full bivariate basis of the requested degree (0, 1, 2) in
 *     coordinates (u, v) scaled by 1/h; heights f are not scaled;
 *   - degenerate plane ((l1 - l0) <= 1e-6 l2, or l2 <= 2^-40 D^2 with the
 *     covariance normalised by W and D the largest distance from r to a row
 *     entry): output r and the computed normal, status bit 1; singular polynomial system (a Cholesky
 *     pivot <= 1e-12 trace): output q, status bit 2.
 *
 * Every computation after the neighbour ranking runs in double precision on
 * coordinates converted exactly from float.  Build with -ffp-contract=off so
 * that the FP32 key is rounded after every operation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ST_PLANE_DEGENERATE 1

/* Reading R9: a plane whose weighted covariance (normalised by W) has its
 * largest eigenvalue at most 2^-40 D^2, D the largest distance from the point
 * to an entry of its row, is degenerate as well: the neighbours' weights are
 * then negligible beside the point's own (all of them many h away), and the
 * plane they would define is not resolved by the weights' precision.  Such a
 * point stays where it is. */
#define PLANE_MIN_SPREAD 0x1p-40
#define ST_POLY_SINGULAR 2

/* ------------------------------------------------------------------------- */
/* Neighbour ranking                                                          */
/* ------------------------------------------------------------------------- */

/* The ranking key between query q and candidate p: each difference, square and
 * sum rounded to float, association ((dx^2 + dy^2) + dz^2).  No fused
 * multiply-add: the file is compiled with -ffp-contract=off. */
float oracle_knn_key(const float *p, const float *q)
{
    float dx = p[0] - q[0];
    float dy = p[1] - q[1];
    float dz = p[2] - q[2];
    float sx = dx * dx;
    float sy = dy * dy;
    float sz = dz * dz;
    float sxy = sx + sy;
    return sxy + sz;
}

/* (key, index) pairs compare lexicographically. */
typedef struct {
    float key;
    int32_t idx;
} kv_t;

static int kv_less(kv_t a, kv_t b)
{
    return a.key < b.key || (a.key == b.key && a.idx < b.idx);
}

static int kv_cmp(const void *pa, const void *pb)
{
    kv_t a = *(const kv_t *)pa, b = *(const kv_t *)pb;
    if (kv_less(a, b)) return -1;
    if (kv_less(b, a)) return 1;
    return 0;
}

/* Brute force: rank every point for every query and keep the first k.
 * O(n^2 log n); meant for n up to a few thousand. */
int oracle_knn_brute(const float *xyz, int64_t n, int k, int32_t *out_idx, float *out_key)
{
    if (k < 1 || k > n) return -1;
    kv_t *all = (kv_t *)malloc(sizeof(kv_t) * (size_t)n);
    if (!all) return -2;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            all[j].key = oracle_knn_key(xyz + 3 * j, xyz + 3 * i);
            all[j].idx = (int32_t)j;
        }
        qsort(all, (size_t)n, sizeof(kv_t), kv_cmp);
        for (int s = 0; s < k; ++s) {
            out_idx[i * k + s] = all[s].idx;
            if (out_key) out_key[i * k + s] = all[s].key;
        }
    }
    free(all);
    return 0;
}

/* ---- k-d tree ------------------------------------------------------------ */

typedef struct {
    double lo[3], hi[3];       /* bounding box of the node's points */
    int64_t begin, end;        /* range in the permutation array */
    int64_t left, right;       /* children, -1 for a leaf */
} kd_node;

typedef struct {
    const float *xyz;
    int32_t *perm;
    kd_node *nodes;
    int64_t n_nodes, cap;
} kd_tree;

#define KD_LEAF 8

static double coord(const kd_tree *t, int64_t slot, int axis)
{
    return (double)t->xyz[3 * (int64_t)t->perm[slot] + axis];
}

/* Partially order perm[begin, end) so that slot `mid` holds the point of
 * rank mid along `axis` (Hoare quickselect). */
static void select_median(kd_tree *t, int64_t begin, int64_t end, int64_t mid, int axis)
{
    int64_t lo = begin, hi = end - 1;
    while (lo < hi) {
        double pivot = coord(t, (lo + hi) / 2, axis);
        int64_t i = lo, j = hi;
        while (i <= j) {
            while (coord(t, i, axis) < pivot) ++i;
            while (coord(t, j, axis) > pivot) --j;
            if (i <= j) {
                int32_t tmp = t->perm[i];
                t->perm[i] = t->perm[j];
                t->perm[j] = tmp;
                ++i;
                --j;
            }
        }
        if (mid <= j) hi = j;
        else if (mid >= i) lo = i;
        else break;
    }
}

static int64_t kd_build(kd_tree *t, int64_t begin, int64_t end)
{
    int64_t id = t->n_nodes++;
    kd_node *nd = &t->nodes[id];
    nd->begin = begin;
    nd->end = end;
    nd->left = nd->right = -1;
    for (int a = 0; a < 3; ++a) {
        nd->lo[a] = INFINITY;
        nd->hi[a] = -INFINITY;
    }
    for (int64_t s = begin; s < end; ++s)
        for (int a = 0; a < 3; ++a) {
            double c = coord(t, s, a);
            if (c < nd->lo[a]) nd->lo[a] = c;
            if (c > nd->hi[a]) nd->hi[a] = c;
        }
    if (end - begin <= KD_LEAF) return id;
    int axis = 0;
    for (int a = 1; a < 3; ++a)
        if (nd->hi[a] - nd->lo[a] > nd->hi[axis] - nd->lo[axis]) axis = a;
    int64_t mid = begin + (end - begin) / 2;
    select_median(t, begin, end, mid, axis);
    int64_t l = kd_build(t, begin, mid);
    int64_t r = kd_build(t, mid, end);
    t->nodes[id].left = l;
    t->nodes[id].right = r;
    return id;
}

/* Bounded max-heap of the k best (key, index) pairs seen so far. */
typedef struct {
    kv_t *a;
    int size, k;
} kheap;

static void heap_push(kheap *h, kv_t v)
{
    if (h->size < h->k) {
        int i = h->size++;
        h->a[i] = v;
        while (i > 0) {
            int p = (i - 1) / 2;
            if (!kv_less(h->a[p], h->a[i])) break;
            kv_t tmp = h->a[p];
            h->a[p] = h->a[i];
            h->a[i] = tmp;
            i = p;
        }
        return;
    }
    if (!kv_less(v, h->a[0])) return;
    h->a[0] = v;
    int i = 0;
    for (;;) {
        int l = 2 * i + 1, r = l + 1, m = i;
        if (l < h->size && kv_less(h->a[m], h->a[l])) m = l;
        if (r < h->size && kv_less(h->a[m], h->a[r])) m = r;
        if (m == i) break;
        kv_t tmp = h->a[m];
        h->a[m] = h->a[i];
        h->a[i] = tmp;
        i = m;
    }
}

static void kd_search(const kd_tree *t, int64_t id, const float *q, kheap *h)
{
    const kd_node *nd = &t->nodes[id];
    /* lower bound on the float key of any point in this box: the exact squared
     * distance to the box, shrunk by a relative 1e-6, which covers the rounding
     * of the float key (at most ~5 units of 2^-24) */
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double x = (double)q[a], g = 0.0;
        if (x < nd->lo[a]) g = nd->lo[a] - x;
        else if (x > nd->hi[a]) g = x - nd->hi[a];
        d2 += g * g;
    }
    if (h->size == h->k && d2 * (1.0 - 1e-6) > (double)h->a[0].key) return;
    if (nd->left < 0) {
        for (int64_t s = nd->begin; s < nd->end; ++s) {
            int32_t j = t->perm[s];
            kv_t v = {oracle_knn_key(t->xyz + 3 * (int64_t)j, q), j};
            heap_push(h, v);
        }
        return;
    }
    /* visit the child whose box centre is nearer first */
    const kd_node *L = &t->nodes[nd->left], *R = &t->nodes[nd->right];
    double dl = 0.0, dr = 0.0;
    for (int a = 0; a < 3; ++a) {
        double cl = 0.5 * (L->lo[a] + L->hi[a]) - q[a];
        double cr = 0.5 * (R->lo[a] + R->hi[a]) - q[a];
        dl += cl * cl;
        dr += cr * cr;
    }
    if (dl <= dr) {
        kd_search(t, nd->left, q, h);
        kd_search(t, nd->right, q, h);
    } else {
        kd_search(t, nd->right, q, h);
        kd_search(t, nd->left, q, h);
    }
}

/* k nearest neighbours of the points listed in `queries` (all points when
 * queries == NULL), against the whole cloud, with the k-d tree of Sec. 2.2.
 * Row s of the output belongs to queries[s] (or point s). */
int oracle_knn_kdtree(const float *xyz, int64_t n, int k, const int64_t *queries, int64_t nq,
                      int32_t *out_idx, float *out_key)
{
    if (k < 1 || k > n) return -1;
    kd_tree t;
    t.xyz = xyz;
    t.perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    /* a node splits only above KD_LEAF points, so every leaf holds at least
     * KD_LEAF / 2 of them: fewer than n / 4 leaves and n / 2 nodes */
    t.cap = n / 2 + 16;
    t.nodes = (kd_node *)malloc(sizeof(kd_node) * (size_t)t.cap);
    t.n_nodes = 0;
    kv_t *buf = (kv_t *)malloc(sizeof(kv_t) * (size_t)k);
    if (!t.perm || !t.nodes || !buf) {
        free(t.perm);
        free(t.nodes);
        free(buf);
        return -2;
    }
    for (int64_t i = 0; i < n; ++i) t.perm[i] = (int32_t)i;
    kd_build(&t, 0, n);
    int64_t m = queries ? nq : n;
    for (int64_t s = 0; s < m; ++s) {
        int64_t i = queries ? queries[s] : s;
        kheap h = {buf, 0, k};
        kd_search(&t, 0, xyz + 3 * i, &h);
        qsort(buf, (size_t)h.size, sizeof(kv_t), kv_cmp);
        for (int c = 0; c < k; ++c) {
            out_idx[s * k + c] = buf[c].idx;
            if (out_key) out_key[s * k + c] = buf[c].key;
        }
    }
    free(t.perm);
    free(t.nodes);
    free(buf);
    return 0;
}

/* Bandwidth helper (not in the paper): the mean distance from each point to
 * the members of its neighbour list other than itself, in FP64 (the
 * workloads take h = 2 x this mean). */
double oracle_mean_knn_dist(const float *xyz, int64_t n, const int32_t *idx, int k)
{
    double sum = 0.0;
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int s = 0; s < k; ++s) {
            int64_t j = idx[i * k + s];
            if (j == i) continue;
            double d2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                double d = (double)xyz[3 * j + a] - (double)xyz[3 * i + a];
                d2 += d * d;
            }
            sum += sqrt(d2);
            ++cnt;
        }
    return cnt ? sum / (double)cnt : 0.0;
}

/* ------------------------------------------------------------------------- */
/* Dense linear algebra (textbook forms)                                      */
/* ------------------------------------------------------------------------- */

/* Cyclic Jacobi eigen-decomposition of a symmetric m x m matrix (m <= 6),
 * row-major in A (destroyed).  Sweeps until the off-diagonal Frobenius norm is
 * at most 1e-15 of the full norm.  Output: eigenvalues ascending in lam, the
 * matching unit eigenvectors as the COLUMNS of V (row-major m x m). */
void oracle_jacobi_eig(int m, double *A, double *lam, double *V)
{
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) V[i * m + j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, all = 0.0;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                double a2 = A[i * m + j] * A[i * m + j];
                all += a2;
                if (i != j) off += a2;
            }
        if (off <= 1e-30 * all) break;
        for (int p = 0; p < m - 1; ++p)
            for (int q = p + 1; q < m; ++q) {
                double apq = A[p * m + q];
                if (apq == 0.0) continue;
                /* rotation angle phi with tan(phi) = t, the root of smaller
                 * magnitude of t^2 + 2 theta t - 1 = 0, zeroes A[p][q] */
                double theta = (A[q * m + q] - A[p * m + p]) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int r = 0; r < m; ++r) {          /* A <- A J */
                    double arp = A[r * m + p], arq = A[r * m + q];
                    A[r * m + p] = c * arp - s * arq;
                    A[r * m + q] = s * arp + c * arq;
                }
                for (int r = 0; r < m; ++r) {          /* A <- J^T A */
                    double apr = A[p * m + r], aqr = A[q * m + r];
                    A[p * m + r] = c * apr - s * aqr;
                    A[q * m + r] = s * apr + c * aqr;
                }
                A[p * m + q] = A[q * m + p] = 0.0;
                for (int r = 0; r < m; ++r) {          /* V <- V J */
                    double vrp = V[r * m + p], vrq = V[r * m + q];
                    V[r * m + p] = c * vrp - s * vrq;
                    V[r * m + q] = s * vrp + c * vrq;
                }
            }
    }
    for (int i = 0; i < m; ++i) lam[i] = A[i * m + i];
    /* selection sort of the eigenpairs, ascending */
    for (int i = 0; i < m; ++i) {
        int b = i;
        for (int j = i + 1; j < m; ++j)
            if (lam[j] < lam[b]) b = j;
        if (b != i) {
            double tl = lam[i];
            lam[i] = lam[b];
            lam[b] = tl;
            for (int r = 0; r < m; ++r) {
                double tv = V[r * m + i];
                V[r * m + i] = V[r * m + b];
                V[r * m + b] = tv;
            }
        }
    }
}

/* Cholesky factorisation A = L L^T (m x m, row-major).  Returns 0 when a
 * pivot is <= rel_tol * trace(A) (the system is then treated as singular). */
int oracle_cholesky(int m, const double *A, double *L, double rel_tol)
{
    double tr = 0.0;
    for (int i = 0; i < m; ++i) tr += A[i * m + i];
    memset(L, 0, sizeof(double) * (size_t)(m * m));
    for (int j = 0; j < m; ++j) {
        double d = A[j * m + j];
        for (int c = 0; c < j; ++c) d -= L[j * m + c] * L[j * m + c];
        if (!(d > rel_tol * tr)) return 0;
        L[j * m + j] = sqrt(d);
        for (int i = j + 1; i < m; ++i) {
            double s = A[i * m + j];
            for (int c = 0; c < j; ++c) s -= L[i * m + c] * L[j * m + c];
            L[i * m + j] = s / L[j * m + j];
        }
    }
    return 1;
}

/* Solve L L^T x = b given the Cholesky factor. */
void oracle_cholesky_solve(int m, const double *L, const double *b, double *x)
{
    double y[6];
    for (int i = 0; i < m; ++i) {
        double s = b[i];
        for (int c = 0; c < i; ++c) s -= L[i * m + c] * y[c];
        y[i] = s / L[i * m + i];
    }
    for (int i = m - 1; i >= 0; --i) {
        double s = y[i];
        for (int c = i + 1; c < m; ++c) s -= L[c * m + i] * x[c];
        x[i] = s / L[i * m + i];
    }
}

/* ------------------------------------------------------------------------- */
/* The MLS projection of one point                                            */
/* ------------------------------------------------------------------------- */

static int n_basis(int degree)
{
    return degree == 0 ? 1 : (degree == 1 ? 3 : 6);
}

/* Monomials of the height polynomial g(u, v) = sum a_c phi_c(u, v):
 * (1), (1, u, v) or (1, u, v, u^2, u v, v^2). */
static void basis(int degree, double u, double v, double *phi)
{
    phi[0] = 1.0;
    if (degree >= 1) {
        phi[1] = u;
        phi[2] = v;
    }
    if (degree >= 2) {
        phi[3] = u * u;
        phi[4] = u * v;
        phi[5] = v * v;
    }
}

/* Fit the height polynomial over a given frame (Sec. 1.4 and Algorithm 1's
 * local polynomial approximation): local coordinates of neighbour p are
 * u = <e1, p - q> / h, v = <e2, p - q> / h, height f = <nrm, p - q>; minimise
 * sum_j w_j (g(u_j, v_j) - f_j)^2 through the normal equations A a = b with
 * A = sum w phi phi^T, b = sum w phi f, solved by Cholesky.
 * Returns 1 and the coefficients in a[], or 0 when the system is singular.
 * cond (optional) receives the 2-norm condition number of A. */
int oracle_fit_height(int m_nb, const double *P, const double *w, const double *nrm,
                      const double *e1, const double *e2, const double *q, double h,
                      int degree, double *a, double *cond)
{
    int nb = n_basis(degree);
    double A[36] = {0}, b[6] = {0}, L[36], phi[6];
    for (int j = 0; j < m_nb; ++j) {
        double d[3] = {P[3 * j] - q[0], P[3 * j + 1] - q[1], P[3 * j + 2] - q[2]};
        double u = (e1[0] * d[0] + e1[1] * d[1] + e1[2] * d[2]) / h;
        double v = (e2[0] * d[0] + e2[1] * d[1] + e2[2] * d[2]) / h;
        double f = nrm[0] * d[0] + nrm[1] * d[1] + nrm[2] * d[2];
        basis(degree, u, v, phi);
        for (int r = 0; r < nb; ++r) {
            b[r] += w[j] * phi[r] * f;
            for (int c = 0; c < nb; ++c) A[r * nb + c] += w[j] * phi[r] * phi[c];
        }
    }
    if (cond) {
        double Ac[36], lam[6], V[36];
        memcpy(Ac, A, sizeof(double) * (size_t)(nb * nb));
        oracle_jacobi_eig(nb, Ac, lam, V);
        *cond = lam[0] > 0.0 ? lam[nb - 1] / lam[0] : INFINITY;
    }
    if (!oracle_cholesky(nb, A, L, 1e-12)) return 0;
    oracle_cholesky_solve(nb, L, b, a);
    return 1;
}

/* Canonical orientation of the plane normal: flip so that the component of
 * largest magnitude is positive (ties go to the lowest axis). */
static void canonical_sign(double *v)
{
    int a = 0;
    for (int c = 1; c < 3; ++c)
        if (fabs(v[c]) > fabs(v[a])) a = c;
    if (v[a] < 0.0)
        for (int c = 0; c < 3; ++c) v[c] = -v[c];
}

/* Everything the projection of one point computes, kept for the adjoint. */
typedef struct {
    int k, degree, status;
    double h, r[3];
    double *P, *d, *w;          /* k x 3, k x 3, k */
    double W, m[3];             /* total weight, centroid offset c - r */
    double C[9], lam[3], V[9];  /* covariance about c; eigenpairs (columns) */
    double nrm[3], e1[3], e2[3];
    double ofs;                 /* <n, c - r>, so q = r + ofs n */
    double q[3];
    double a[6];                /* polynomial coefficients (zero if singular) */
    double cond;                /* condition number of the normal matrix */
    double out[3];
} point_state;

static void project_point(const float *xyz, const int32_t *row, int k, double h, int degree,
                          int64_t i, point_state *st)
{
    st->k = k;
    st->degree = degree;
    st->h = h;
    st->status = 0;
    for (int a = 0; a < 3; ++a) st->r[a] = (double)xyz[3 * i + a];
    /* weights about r (Eq. 1's theta, Gaussian) */
    st->W = 0.0;
    double sw[3] = {0, 0, 0}, D2 = 0.0;
    for (int j = 0; j < k; ++j) {
        int64_t p = row[j];
        double d2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            st->P[3 * j + a] = (double)xyz[3 * p + a];
            st->d[3 * j + a] = st->P[3 * j + a] - st->r[a];
            d2 += st->d[3 * j + a] * st->d[3 * j + a];
        }
        if (d2 > D2) D2 = d2;
        st->w[j] = exp(-d2 / (h * h));
        st->W += st->w[j];
        for (int a = 0; a < 3; ++a) sw[a] += st->w[j] * st->d[3 * j + a];
    }
    /* weighted centroid c = r + m */
    for (int a = 0; a < 3; ++a) st->m[a] = sw[a] / st->W;
    /* weighted covariance about c, second pass */
    memset(st->C, 0, sizeof st->C);
    for (int j = 0; j < k; ++j) {
        double e[3];
        for (int a = 0; a < 3; ++a) e[a] = st->d[3 * j + a] - st->m[a];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) st->C[3 * a + b] += st->w[j] * e[a] * e[b];
    }
    for (int c = 0; c < 9; ++c) st->C[c] /= st->W;
    /* plane of Eq. 1: the normal minimises the weighted sum of squared
     * distances, i.e. the eigenvector of the smallest eigenvalue */
    double Cw[9];
    memcpy(Cw, st->C, sizeof Cw);
    oracle_jacobi_eig(3, Cw, st->lam, st->V);
    for (int a = 0; a < 3; ++a) {
        st->nrm[a] = st->V[3 * a + 0];
        st->e1[a] = st->V[3 * a + 1];
    }
    canonical_sign(st->nrm);
    st->e2[0] = st->nrm[1] * st->e1[2] - st->nrm[2] * st->e1[1];
    st->e2[1] = st->nrm[2] * st->e1[0] - st->nrm[0] * st->e1[2];
    st->e2[2] = st->nrm[0] * st->e1[1] - st->nrm[1] * st->e1[0];
    memset(st->a, 0, sizeof st->a);
    st->cond = 0.0;
    if (!(st->lam[2] > PLANE_MIN_SPREAD * D2) || (st->lam[1] - st->lam[0]) <= 1e-6 * st->lam[2]) {
        st->status = ST_PLANE_DEGENERATE;
        for (int a = 0; a < 3; ++a) st->out[a] = st->r[a];
        st->ofs = 0.0;
        for (int a = 0; a < 3; ++a) st->q[a] = st->r[a];
        return;
    }
    /* q: projection of r onto H, which passes through c with normal n */
    st->ofs = st->nrm[0] * st->m[0] + st->nrm[1] * st->m[1] + st->nrm[2] * st->m[2];
    for (int a = 0; a < 3; ++a) st->q[a] = st->r[a] + st->ofs * st->nrm[a];
    /* local height polynomial and the projection onto it: p' = q + g(0,0) n */
    if (!oracle_fit_height(k, st->P, st->w, st->nrm, st->e1, st->e2, st->q, h, degree, st->a,
                           &st->cond)) {
        st->status |= ST_POLY_SINGULAR;
        memset(st->a, 0, sizeof st->a);
    }
    for (int a = 0; a < 3; ++a) st->out[a] = st->q[a] + st->a[0] * st->nrm[a];
}

static int alloc_state(point_state *st, int k)
{
    st->P = (double *)malloc(sizeof(double) * 3 * (size_t)k);
    st->d = (double *)malloc(sizeof(double) * 3 * (size_t)k);
    st->w = (double *)malloc(sizeof(double) * (size_t)k);
    return st->P && st->d && st->w;
}

static void free_state(point_state *st)
{
    free(st->P);
    free(st->d);
    free(st->w);
}

/* Project the points listed in `queries` (all when NULL).  Neighbour rows:
 * idx holds one row of k indices per projected point, in output order (row s
 * belongs to queries[s], or to point s when queries is NULL).
 * out_diag (optional, 5 per row): l0, l1, l2, cond(A), W. */
int oracle_project(const float *xyz, int64_t n, const int32_t *idx, int k, double h, int degree,
                   const int64_t *queries, int64_t nq, double *out_xyz, double *out_normal,
                   uint8_t *out_status, double *out_diag)
{
    if (k < 1 || k > n || !(h > 0.0) || degree < 0 || degree > 2) return -1;
    point_state st;
    if (!alloc_state(&st, k)) {
        free_state(&st);
        return -2;
    }
    int64_t m = queries ? nq : n;
    for (int64_t s = 0; s < m; ++s) {
        int64_t i = queries ? queries[s] : s;
        project_point(xyz, idx + s * k, k, h, degree, i, &st);
        for (int a = 0; a < 3; ++a) {
            out_xyz[3 * s + a] = st.out[a];
            if (out_normal) out_normal[3 * s + a] = st.nrm[a];
        }
        if (out_status) out_status[s] = (uint8_t)st.status;
        if (out_diag) {
            out_diag[5 * s + 0] = st.lam[0];
            out_diag[5 * s + 1] = st.lam[1];
            out_diag[5 * s + 2] = st.lam[2];
            out_diag[5 * s + 3] = st.cond;
            out_diag[5 * s + 4] = st.W;
        }
    }
    free_state(&st);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Adjoint (not in the paper): gradients of L = sum_i <gp_i, p'_i> +          */
/* <gn_i, n_i> with respect to every input coordinate and h, neighbour rows   */
/* and the normal's sign held fixed.                                          */
/* ------------------------------------------------------------------------- */

static double dot3(const double *a, const double *b)
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* Reverse pass through one point; adds into grad (n x 3) and *grad_h.
 * Points with a degenerate plane pass the position gradient to r only (the
 * output is r) and none through the normal.  With a singular polynomial
 * system the polynomial value is 0 and only the plane part is differentiated. */
static void adjoint_point(const point_state *st, const int32_t *row, int64_t i,
                          const double *gp, const double *gn, double *grad, double *grad_h,
                          double *grad_abs)
{
    int k = st->k, nb = n_basis(st->degree);
    double h = st->h;
    if (st->status & ST_PLANE_DEGENERATE) {
        for (int a = 0; a < 3; ++a) grad[3 * i + a] += gp[a];
        if (grad_abs) grad_abs[i] += sqrt(dot3(gp, gp));
        return;
    }
    double *dbar = (double *)calloc(3 * (size_t)k, sizeof(double));
    double *wbar = (double *)calloc((size_t)k, sizeof(double));
    double rbar[3], nbar[3], e1bar[3] = {0, 0, 0}, e2bar[3] = {0, 0, 0}, mbar[3];
    double hbar = 0.0;
    /* p' = r + s n with s = ofs + a0 */
    double s = st->ofs + st->a[0];
    double sbar = dot3(gp, st->nrm);
    for (int a = 0; a < 3; ++a) {
        rbar[a] = gp[a];
        nbar[a] = s * gp[a] + (gn ? gn[a] : 0.0);
    }
    double ofsbar = sbar;
    if (!(st->status & ST_POLY_SINGULAR)) {
        /* a = A^{-1} b, a0 = e_0^T a: z = A^{-1} (abar0 e_0), bbar = z,
         * Abar = -z a^T.  Rebuild A to factor it. */
        double A[36] = {0}, L[36], rhs[6] = {0}, z[6], phi[6];
        double *uu = (double *)malloc(sizeof(double) * (size_t)k);
        double *vv = (double *)malloc(sizeof(double) * (size_t)k);
        double *ff = (double *)malloc(sizeof(double) * (size_t)k);
        for (int j = 0; j < k; ++j) {
            const double *dj = st->d + 3 * j;
            uu[j] = dot3(st->e1, dj) / h;
            vv[j] = dot3(st->e2, dj) / h;
            ff[j] = dot3(st->nrm, dj) - st->ofs;
            basis(st->degree, uu[j], vv[j], phi);
            for (int r = 0; r < nb; ++r)
                for (int c = 0; c < nb; ++c) A[r * nb + c] += st->w[j] * phi[r] * phi[c];
        }
        oracle_cholesky(nb, A, L, 0.0);
        rhs[0] = sbar;
        oracle_cholesky_solve(nb, L, rhs, z);
        for (int j = 0; j < k; ++j) {
            const double *dj = st->d + 3 * j;
            basis(st->degree, uu[j], vv[j], phi);
            double g = 0.0, zeta = 0.0;
            for (int c = 0; c < nb; ++c) {
                g += phi[c] * st->a[c];
                zeta += phi[c] * z[c];
            }
            double res = ff[j] - g;
            wbar[j] += zeta * res;
            double fbar = st->w[j] * zeta;
            double phibar[6];
            for (int c = 0; c < nb; ++c) phibar[c] = st->w[j] * (res * z[c] - zeta * st->a[c]);
            double ubar = 0.0, vbar = 0.0;
            if (st->degree >= 1) {
                ubar = phibar[1];
                vbar = phibar[2];
            }
            if (st->degree >= 2) {
                ubar += 2.0 * uu[j] * phibar[3] + vv[j] * phibar[4];
                vbar += uu[j] * phibar[4] + 2.0 * vv[j] * phibar[5];
            }
            /* u = <e1, d>/h, v = <e2, d>/h, f = <n, d> - ofs */
            for (int a = 0; a < 3; ++a) {
                dbar[3 * j + a] += ubar / h * st->e1[a] + vbar / h * st->e2[a] + fbar * st->nrm[a];
                e1bar[a] += ubar / h * dj[a];
                e2bar[a] += vbar / h * dj[a];
                nbar[a] += fbar * dj[a];
            }
            hbar -= (ubar * uu[j] + vbar * vv[j]) / h;
            ofsbar -= fbar;
        }
        free(uu);
        free(vv);
        free(ff);
    }
    /* ofs = <n, m> */
    for (int a = 0; a < 3; ++a) {
        nbar[a] += ofsbar * st->m[a];
        mbar[a] = ofsbar * st->nrm[a];
    }
    /* frame: eigenvector derivative of n, and the tilt of (e1, e2) that keeps
     * the frame orthonormal; the spin within the plane does not change g(0,0)
     * (the basis is rotation invariant in (u, v)) and is left out. */
    double Cbar[9] = {0};
    const double *eb[2] = {st->e1, st->e2};
    const double *ebbar[2] = {e1bar, e2bar};
    for (int b = 0; b < 2; ++b) {
        double gap = st->lam[0] - st->lam[b + 1];
        double gamma = (dot3(nbar, eb[b]) - dot3(ebbar[b], st->nrm)) / gap;
        for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y)
                Cbar[3 * x + y] += 0.5 * gamma * (eb[b][x] * st->nrm[y] + st->nrm[x] * eb[b][y]);
    }
    /* C = sum w e e^T / W with e = d - m */
    double CC = 0.0;
    for (int c = 0; c < 9; ++c) CC += Cbar[c] * st->C[c];
    double sum_ebar[3] = {0, 0, 0};
    for (int j = 0; j < k; ++j) {
        double e[3], Ce[3];
        for (int a = 0; a < 3; ++a) e[a] = st->d[3 * j + a] - st->m[a];
        for (int x = 0; x < 3; ++x) Ce[x] = Cbar[3 * x] * e[0] + Cbar[3 * x + 1] * e[1] + Cbar[3 * x + 2] * e[2];
        wbar[j] += (dot3(e, Ce) - CC) / st->W;
        for (int a = 0; a < 3; ++a) {
            double ebar = 2.0 * st->w[j] * Ce[a] / st->W;
            dbar[3 * j + a] += ebar;
            sum_ebar[a] += ebar;
        }
    }
    for (int a = 0; a < 3; ++a) mbar[a] -= sum_ebar[a];
    /* m = sum w d / W */
    for (int j = 0; j < k; ++j) {
        double e[3];
        for (int a = 0; a < 3; ++a) e[a] = st->d[3 * j + a] - st->m[a];
        wbar[j] += dot3(mbar, e) / st->W;
        for (int a = 0; a < 3; ++a) dbar[3 * j + a] += st->w[j] * mbar[a] / st->W;
    }
    /* w = exp(-|d|^2 / h^2) */
    for (int j = 0; j < k; ++j) {
        const double *dj = st->d + 3 * j;
        double d2 = dot3(dj, dj);
        for (int a = 0; a < 3; ++a) dbar[3 * j + a] += wbar[j] * st->w[j] * (-2.0 * dj[a] / (h * h));
        hbar += wbar[j] * st->w[j] * (2.0 * d2 / (h * h * h));
    }
    /* d = p_j - r */
    for (int j = 0; j < k; ++j) {
        int64_t p = row[j];
        for (int a = 0; a < 3; ++a) {
            grad[3 * p + a] += dbar[3 * j + a];
            rbar[a] -= dbar[3 * j + a];
        }
        if (grad_abs) grad_abs[p] += sqrt(dot3(dbar + 3 * j, dbar + 3 * j));
    }
    for (int a = 0; a < 3; ++a) grad[3 * i + a] += rbar[a];
    if (grad_abs) grad_abs[i] += sqrt(dot3(rbar, rbar));
    *grad_h += hbar;
    free(dbar);
    free(wbar);
}

/* Vector-Jacobian product of the projection: grad_xyz (n x 3, overwritten)
 * and *grad_h (overwritten) for the cotangents gout_xyz (n x 3) and
 * gout_normal (n x 3, or NULL for zero).  With queries != NULL only the
 * listed points' terms are summed (their rows are idx rows s, in order):
 * the full product is the sum over all points.
 * grad_abs (optional, n, overwritten): per point, the sum of the Euclidean
 * norms of the terms added into its gradient (one per projected point whose
 * row holds it, plus its own); a scale for the rounding error of the sum,
 * which can be far above the norm of the sum when the terms cancel. */
int oracle_project_grad(const float *xyz, int64_t n, const int32_t *idx, int k, double h,
                        int degree, const double *gout_xyz, const double *gout_normal,
                        const int64_t *queries, int64_t nq, double *grad_xyz, double *grad_h,
                        double *grad_abs)
{
    if (k < 1 || k > n || !(h > 0.0) || degree < 0 || degree > 2) return -1;
    point_state st;
    if (!alloc_state(&st, k)) {
        free_state(&st);
        return -2;
    }
    memset(grad_xyz, 0, sizeof(double) * 3 * (size_t)n);
    if (grad_abs) memset(grad_abs, 0, sizeof(double) * (size_t)n);
    *grad_h = 0.0;
    int64_t m = queries ? nq : n;
    for (int64_t s = 0; s < m; ++s) {
        int64_t i = queries ? queries[s] : s;
        project_point(xyz, idx + s * k, k, h, degree, i, &st);
        adjoint_point(&st, idx + s * k, i, gout_xyz + 3 * i, gout_normal ? gout_normal + 3 * i : NULL,
                      grad_xyz, grad_h, grad_abs);
    }
    free_state(&st);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* The projection with weights about q (Sec. 1.4, Eq. 1)                      */
/* ------------------------------------------------------------------------- */

#define ST_NOT_CONVERGED 8

/* Eq. 1 weighs each neighbour by theta(|p_i - q|), q = r + t n being the
 * projection of r onto the plane H that the weighted fit returns.  Reading:
 * H is the self-consistent plane -- the weighted least-squares plane (normal
 * = eigenvector of the smallest eigenvalue of the weighted covariance about
 * the weighted centroid) for weights taken about the projection of r onto
 * that same plane.  It is reached by the fixed-point iteration that starts
 * at q = r (t = 0, the root nearest the point, Sec. 1.4's smallest t) and
 * alternates "weights about q" and "plane of those weights, q = projection of
 * r onto it", until t changes by at most tol * h (or max_iter iterations,
 * status bit 8).  The polynomial is then fitted in the frame at the final q
 * with the weights about that q, and the result is q + g(0, 0) n.
 * Status, degenerate and singular rules as in oracle_project.
 * out_iter (optional): iterations used per point.
 * out_diag (optional, 5 per row, as oracle_project's): eigenvalues of the
 * last plane's covariance, condition number of the final height fit's normal
 * matrix (0 when not fitted), and the last plane's total weight. */
int oracle_project_levin(const float *xyz, int64_t n, const int32_t *idx, int k, double h, int degree,
                         int max_iter, double tol, const int64_t *queries, int64_t nq, double *out_xyz,
                         double *out_normal, uint8_t *out_status, int32_t *out_iter, double *out_diag)
{
    if (k < 1 || k > n || !(h > 0.0) || degree < 0 || degree > 2 || max_iter < 1) return -1;
    double *P = (double *)malloc(sizeof(double) * 3 * (size_t)k);
    double *w = (double *)malloc(sizeof(double) * (size_t)k);
    if (!P || !w) {
        free(P);
        free(w);
        return -2;
    }
    int64_t m = queries ? nq : n;
    for (int64_t s = 0; s < m; ++s) {
        int64_t i = queries ? queries[s] : s;
        const int32_t *row = idx + s * k;
        double r[3], q[3], nrm[3] = {0, 0, 0}, e1[3] = {0, 0, 0}, e2[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a) r[a] = q[a] = (double)xyz[3 * i + a];
        double D2 = 0.0;     /* the largest squared distance from r to a row entry (R9) */
        for (int j = 0; j < k; ++j) {
            double d2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                P[3 * j + a] = (double)xyz[3 * (int64_t)row[j] + a];
                d2 += (P[3 * j + a] - r[a]) * (P[3 * j + a] - r[a]);
            }
            if (d2 > D2) D2 = d2;
        }
        int status = ST_NOT_CONVERGED, iters = 0;
        double t = 0.0, last_lam[3] = {0, 0, 0}, last_W = 0.0, cond = 0.0;
        for (int it = 0; it < max_iter; ++it) {
            iters = it + 1;
            /* weights about q */
            double W = 0.0, c[3] = {0, 0, 0};
            for (int j = 0; j < k; ++j) {
                double d2 = 0.0;
                for (int a = 0; a < 3; ++a) d2 += (P[3 * j + a] - q[a]) * (P[3 * j + a] - q[a]);
                w[j] = exp(-d2 / (h * h));
                W += w[j];
                for (int a = 0; a < 3; ++a) c[a] += w[j] * P[3 * j + a];
            }
            for (int a = 0; a < 3; ++a) c[a] /= W;
            /* the weighted plane through c */
            double C[9] = {0}, lam[3], V[9];
            for (int j = 0; j < k; ++j) {
                double e[3];
                for (int a = 0; a < 3; ++a) e[a] = P[3 * j + a] - c[a];
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) C[3 * a + b] += w[j] * e[a] * e[b];
            }
            for (int x = 0; x < 9; ++x) C[x] /= W;
            oracle_jacobi_eig(3, C, lam, V);
            for (int a = 0; a < 3; ++a) {
                nrm[a] = V[3 * a + 0];
                e1[a] = V[3 * a + 1];
            }
            canonical_sign(nrm);
            e2[0] = nrm[1] * e1[2] - nrm[2] * e1[1];
            e2[1] = nrm[2] * e1[0] - nrm[0] * e1[2];
            e2[2] = nrm[0] * e1[1] - nrm[1] * e1[0];
            for (int a = 0; a < 3; ++a) last_lam[a] = lam[a];
            last_W = W;
            if (!(lam[2] > PLANE_MIN_SPREAD * D2) || (lam[1] - lam[0]) <= 1e-6 * lam[2]) {
                status = ST_PLANE_DEGENERATE;
                break;
            }
            /* q: the projection of r onto the plane */
            double tn = nrm[0] * (c[0] - r[0]) + nrm[1] * (c[1] - r[1]) + nrm[2] * (c[2] - r[2]);
            for (int a = 0; a < 3; ++a) q[a] = r[a] + tn * nrm[a];
            int done = it > 0 && fabs(tn - t) <= tol * h;
            t = tn;
            if (done) {
                status = 0;
                break;
            }
        }
        double out[3] = {r[0], r[1], r[2]};
        if (!(status & ST_PLANE_DEGENERATE)) {
            /* weights about the final q, the height polynomial, the projection */
            for (int j = 0; j < k; ++j) {
                double d2 = 0.0;
                for (int a = 0; a < 3; ++a) d2 += (P[3 * j + a] - q[a]) * (P[3 * j + a] - q[a]);
                w[j] = exp(-d2 / (h * h));
            }
            double coef[6] = {0, 0, 0, 0, 0, 0};
            if (!oracle_fit_height(k, P, w, nrm, e1, e2, q, h, degree, coef, out_diag ? &cond : NULL)) {
                status |= ST_POLY_SINGULAR;
                coef[0] = 0.0;
            }
            for (int a = 0; a < 3; ++a) out[a] = q[a] + coef[0] * nrm[a];
        }
        for (int a = 0; a < 3; ++a) {
            out_xyz[3 * s + a] = out[a];
            if (out_normal) out_normal[3 * s + a] = nrm[a];
        }
        if (out_status) out_status[s] = (uint8_t)status;
        if (out_iter) out_iter[s] = iters;
        if (out_diag) {
            for (int a = 0; a < 3; ++a) out_diag[5 * s + a] = last_lam[a];
            out_diag[5 * s + 3] = cond;
            out_diag[5 * s + 4] = last_W;
        }
    }
    free(P);
    free(w);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Radius neighbourhoods (Sec. 1.4, Sec. 2.2, Sec. 3.3)                       */
/* ------------------------------------------------------------------------- */

#define ST_OUTLIER 16
#define ST_DEGREE_REDUCED 32

/* Reading R8b (radius mode): a neighbourhood of m points (the point included)
 * is fitted at the highest degree d <= the requested one whose basis has at
 * most m / 2 coefficients (degree 2: 6, so m >= 12; degree 1: 3, so m >= 6;
 * degree 0 otherwise).  With fewer points the fit would interpolate rather
 * than smooth, and over 4-6 points a quadratic can move the point far from
 * its neighbours; degrees 1 and 0 project the point onto its plane. */
static int radius_degree(int degree, int m)
{
    static const int coeffs[3] = {1, 3, 6};
    int d = degree;
    while (d > 0 && m < 2 * coeffs[d]) --d;
    return d;
}

typedef struct {
    kv_t *a;
    int64_t size, cap;
} kvlist;

static int kvlist_push(kvlist *l, kv_t v)
{
    if (l->size == l->cap) {
        int64_t c = l->cap ? 2 * l->cap : 64;
        kv_t *p = (kv_t *)realloc(l->a, sizeof(kv_t) * (size_t)c);
        if (!p) return 0;
        l->a = p;
        l->cap = c;
    }
    l->a[l->size++] = v;
    return 1;
}

/* Every point of the subtree with key <= R2 (the same FP32 key as the kNN). */
static int kd_range(const kd_tree *t, int64_t id, const float *q, float R2, kvlist *out)
{
    const kd_node *nd = &t->nodes[id];
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double x = (double)q[a], g = 0.0;
        if (x < nd->lo[a]) g = nd->lo[a] - x;
        else if (x > nd->hi[a]) g = x - nd->hi[a];
        d2 += g * g;
    }
    if (d2 * (1.0 - 1e-6) > (double)R2) return 1;
    if (nd->left < 0) {
        for (int64_t s = nd->begin; s < nd->end; ++s) {
            int32_t j = t->perm[s];
            kv_t v = {oracle_knn_key(t->xyz + 3 * (int64_t)j, q), j};
            if (v.key <= R2 && !kvlist_push(out, v)) return 0;
        }
        return 1;
    }
    return kd_range(t, nd->left, q, R2, out) && kd_range(t, nd->right, q, R2, out);
}

/* The radius-R neighbourhood of every point: all j with key(i, j) <= R2,
 * the point itself included, ordered by (key, index).  out_count[i] always;
 * when offsets and out_rows are given, row i is written at offsets[i]
 * (offsets[i + 1] - offsets[i] must equal the count). */
int oracle_radius_kdtree(const float *xyz, int64_t n, float R2, const int64_t *offsets, int32_t *out_rows,
                         int32_t *out_count)
{
    if (n < 1 || !(R2 >= 0.0f)) return -1;
    kd_tree t;
    t.xyz = xyz;
    t.perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    t.cap = n / 2 + 16;
    t.nodes = (kd_node *)malloc(sizeof(kd_node) * (size_t)t.cap);
    t.n_nodes = 0;
    kvlist l = {NULL, 0, 0};
    if (!t.perm || !t.nodes) {
        free(t.perm);
        free(t.nodes);
        return -2;
    }
    for (int64_t i = 0; i < n; ++i) t.perm[i] = (int32_t)i;
    kd_build(&t, 0, n);
    int rc = 0;
    for (int64_t i = 0; i < n && rc == 0; ++i) {
        l.size = 0;
        if (!kd_range(&t, 0, xyz + 3 * i, R2, &l)) {
            rc = -2;
            break;
        }
        qsort(l.a, (size_t)l.size, sizeof(kv_t), kv_cmp);
        out_count[i] = (int32_t)l.size;
        if (offsets && out_rows) {
            if (offsets[i + 1] - offsets[i] != l.size) {
                rc = -3;
                break;
            }
            for (int64_t c = 0; c < l.size; ++c) out_rows[offsets[i] + c] = l.a[c].idx;
        }
    }
    free(l.a);
    free(t.perm);
    free(t.nodes);
    return rc;
}

/* The projection over variable neighbourhoods (row i = rows[offsets[i] ..
 * offsets[i + 1])), with Sec. 3.3's outlier rule: a point with fewer than
 * min_neighbors other points in its neighbourhood is not projected (status
 * bit 16, output = the point, to be dropped from the result; diagnostics 0).
 * A small neighbourhood is fitted at a lower degree (radius_degree; status
 * bit 32).  Everything else as oracle_project. */
int oracle_project_rows(const float *xyz, int64_t n, const int64_t *offsets, const int32_t *rows, double h,
                        int degree, int min_neighbors, double *out_xyz, double *out_normal, uint8_t *out_status,
                        double *out_diag)
{
    if (n < 1 || !(h > 0.0) || degree < 0 || degree > 2) return -1;
    int64_t kmax = 1;
    for (int64_t i = 0; i < n; ++i)
        if (offsets[i + 1] - offsets[i] > kmax) kmax = offsets[i + 1] - offsets[i];
    point_state st;
    if (!alloc_state(&st, (int)kmax)) {
        free_state(&st);
        return -2;
    }
    for (int64_t i = 0; i < n; ++i) {
        int k = (int)(offsets[i + 1] - offsets[i]);
        if (k - 1 < min_neighbors) {
            for (int a = 0; a < 3; ++a) {
                out_xyz[3 * i + a] = (double)xyz[3 * i + a];
                if (out_normal) out_normal[3 * i + a] = 0.0;
            }
            if (out_status) out_status[i] = ST_OUTLIER;
            if (out_diag)
                for (int c = 0; c < 5; ++c) out_diag[5 * i + c] = 0.0;
            continue;
        }
        const int d = radius_degree(degree, k);
        project_point(xyz, rows + offsets[i], k, h, d, i, &st);
        for (int a = 0; a < 3; ++a) {
            out_xyz[3 * i + a] = st.out[a];
            if (out_normal) out_normal[3 * i + a] = st.nrm[a];
        }
        if (out_status) out_status[i] = (uint8_t)(st.status | (d < degree ? ST_DEGREE_REDUCED : 0));
        if (out_diag) {
            out_diag[5 * i + 0] = st.lam[0];
            out_diag[5 * i + 1] = st.lam[1];
            out_diag[5 * i + 2] = st.lam[2];
            out_diag[5 * i + 3] = st.cond;
            out_diag[5 * i + 4] = st.W;
        }
    }
    free_state(&st);
    return 0;
}
