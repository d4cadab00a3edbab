/*
 * mls.h -- C ABI of libmls, the GB300 (sm_103a) implementation of the per-point
 * moving least squares (MLS) projection.
 *
 * The method (Sec. 1.4, Eq. 1 and Algorithm 1 of "Investigation of the
 * efficiency of the moving least squares method in the reconstruction of a
 * three-dimensional surface on a supercomputer"): for every point r of the
 * cloud, take its neighbourhood, fit a weighted least-squares reference plane
 * H, move r to its projection q on H, fit a local polynomial g of the
 * neighbours' heights over H in an orthonormal frame with origin q, and return
 * the projection of r onto g, i.e. q + g(0, 0) n.
 *
 * Readings fixed by this library where the paper is silent:
 *   neighbourhood   the k nearest points, the point itself included, ranked by
 *                   key(i, j) = fl((fl(dx*dx) + fl(dy*dy)) + fl(dz*dz)) with
 *                   dx = fl(x_j - x_i) in IEEE float, round to nearest, no fused
 *                   multiply-add; ties go to the lower point index;
 *   weight          theta(d) = exp(-d^2 / h^2), about r, for plane and polynomial;
 *   plane           weighted centroid c, weighted covariance about c, normal =
 *                   eigenvector of the smallest eigenvalue, sign chosen so that
 *                   its largest-magnitude component is positive;
 *   polynomial      full bivariate basis of degree 0, 1 or 2 in local
 *                   coordinates (u, v) / h; heights unscaled;
 *   degenerate      (l1 - l0) <= 1e-6 l2 or l2 == 0: output r, status bit 1;
 *   singular        a Cholesky pivot <= 1e-12 trace of the normal matrix:
 *                   output q, status bit 2.
 *
 * Conventions for every entry point:
 *   - Point and output buffers are DEVICE memory owned by the caller; xyz is
 *     an array of n rows of 3 floats (x, y, z), row i = point i.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *     default stream) unless stated.  Argument errors are returned before any
 *     work is queued; no entry point aborts, throws or traps.
 *   - Return value: MLS_OK (0) or a negative mls_status_code;
 *     mls_last_error() gives a message for the calling thread's last failure.
 */
#ifndef MLS_H_
#define MLS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t, declared without the CUDA headers. */
typedef struct CUstream_st *mls_stream;

/* Opaque spatial index over one point cloud, owned by the library. */
typedef struct mls_grid mls_grid;

enum mls_status_code {
    MLS_OK = 0,
    MLS_ERR_INVALID_ARG = -1,        /* null pointer, n < 1, h <= 0 or not finite, ... */
    MLS_ERR_K_TOO_LARGE = -2,        /* k > MLS_MAX_K or k > n */
    MLS_ERR_UNSUPPORTED_DEGREE = -3, /* degree not in {0, 1, 2} */
    MLS_ERR_CUDA = -4,               /* a CUDA runtime call failed */
    MLS_ERR_OOM = -5,                /* device allocation failed */
    MLS_ERR_TIMEOUT = -6,            /* a bounded device-side wait gave up */
    MLS_ERR_NONFINITE = -7,          /* a coordinate is NaN or infinite */
    MLS_ERR_TOO_LARGE = -8           /* n beyond the 2^31 - 1 index range */
};

/* Precision of mls_project / mls_project_backward. */
enum mls_precision {
    MLS_PREC_FP32 = 0,   /* FP32 moments and solves */
    MLS_PREC_MIXED = 1,  /* FP32 moments; FP64 eigen/normal-equation solves only
                            where the FP32 solve is ill-conditioned */
    MLS_PREC_FP64 = 2    /* everything in FP64 */
};

/* Per-point status bits written by mls_project. */
enum mls_point_status {
    MLS_PT_OK = 0,
    MLS_PT_PLANE_DEGENERATE = 1,
    MLS_PT_POLY_SINGULAR = 2,
    MLS_PT_FP64_USED = 4
};

#define MLS_MAX_K 64

/*
 * mls_build_grid -- spatial index for the neighbour search that precedes each
 * fit (Sec. 2.2; the paper builds a k-d tree and mentions Morton reordering of
 * unordered clouds, Sec. 2 introduction).  Here: a uniform grid whose cells are
 * numbered by 63-bit Morton keys, points sorted by key with an LSD radix sort,
 * and one hash table per coarsening level (cell side doubling per level) from
 * a base level chosen from the cell occupancy.
 *
 *   d_xyz      device, n x 3 floats; must stay valid and unchanged until the
 *              grid is rebuilt or destroyed (mls_knn reads it through the grid)
 *   n          number of points, 1 <= n <= 2^31 - 1
 *   cell_size  > 0: base cell side (rounded to a power-of-two multiple of the
 *              finest cell); <= 0: chosen from the occupancy for k_hint
 *   k_hint     neighbour count the grid will be queried with (1..MLS_MAX_K)
 *   stream     stream for all work
 *   inout      *inout == NULL: a new grid is created and returned;
 *              otherwise the grid is rebuilt in place, reusing its memory.
 *
 * Synchronises `stream` once (level sizes are read back to size the tables),
 * so it cannot be captured in a CUDA graph.  Returns MLS_ERR_NONFINITE if any
 * coordinate is NaN or infinite.  On failure a new grid is not returned and an
 * existing one is left destroyed-safe (mls_grid_destroy may be called).
 */
int mls_build_grid(const float *d_xyz, int64_t n, float cell_size, int k_hint, mls_stream stream,
                   mls_grid **inout);

/* Frees the grid and its device memory (after synchronising its last stream).
 * NULL is ignored. */
void mls_grid_destroy(mls_grid *g);

/* Number of points the grid was built on, or -1 for NULL. */
int64_t mls_grid_size(const mls_grid *g);

/* Device pointer to the Morton order of the points: order[s] is the index of
 * the point at sorted position s (n int32, owned by the grid, valid until the
 * grid is rebuilt or destroyed).  Passing it to mls_project as d_order makes
 * neighbouring threads work on neighbouring points. */
const int32_t *mls_grid_order(const mls_grid *g);

/*
 * mls_knn -- exact k nearest neighbours of every point of the grid's cloud,
 * itself included (the neighbourhood of Sec. 1.4 / Algorithm 1, read as kNN).
 *
 *   d_idx   device, n x k int32: row i lists point i's neighbours by point
 *           index, ascending by (key, index); bit-exact and deterministic
 *   d_key   device, n x k floats or NULL: the matching keys
 *   k       1 <= k <= min(MLS_MAX_K, n)
 */
int mls_knn(const mls_grid *g, int k, int32_t *d_idx, float *d_key, mls_stream stream);

/*
 * mls_project -- the MLS projection of every point (Sec. 1.4, Eq. 1;
 * Algorithm 1: plane, local polynomial, projection onto the polynomial).
 *
 *   d_xyz        device, n x 3 floats
 *   d_idx        device, n x k int32 neighbour rows (as written by mls_knn;
 *                any row order works, every index must be in [0, n))
 *   h            Gaussian bandwidth, finite and > 0
 *   degree       0, 1 or 2
 *   precision    enum mls_precision
 *   d_order      device, n int32 permutation giving the processing order, or
 *                NULL for 0..n-1; affects speed only, never results
 *   d_out_xyz    device, n x 3 floats: projected points p'
 *   d_out_normal device, n x 3 floats or NULL: plane normals n
 *   d_status     device, n bytes or NULL: enum mls_point_status bits
 * Outputs must not alias inputs.
 */
int mls_project(const float *d_xyz, int64_t n, const int32_t *d_idx, int k, float h, int degree,
                int precision, const int32_t *d_order, float *d_out_xyz, float *d_out_normal,
                uint8_t *d_status, mls_stream stream);

/*
 * mls_project_noalloc -- mls_project for callers that must not allocate
 * device memory.  The paper has no counterpart: this is a deployment
 * variant.  Some callers cannot let a library allocate: hosts that hand out
 * all device memory from their own fixed pool or budget (inference servers,
 * embedded pipelines) and would not see a cudaMallocAsync, or loops that must
 * not risk an allocation failing half way.  This entry point takes its
 * scratch (a float4 copy of the points) from a fixed device array of
 * MLS_NOALLOC_MAX_POINTS entries (4 MiB), which every GPU that loads the
 * library holds until the process exits; it calls no allocation routine.
 *
 * Arguments, outputs and results are those of mls_project.
 * Returns MLS_ERR_TOO_LARGE when n > MLS_NOALLOC_MAX_POINTS.
 * The first call on a device looks the array's device address up (with that
 * device current); make that first call before any stream capture.
 * All calls share the one array: calls that overlap on the GPU (other
 * streams, other threads) race and corrupt each other's scratch; serialise
 * them.  Every call overwrites the part it uses, so no state carries over.
 */
#define MLS_NOALLOC_MAX_POINTS 262144
int mls_project_noalloc(const float *d_xyz, int64_t n, const int32_t *d_idx, int k, float h, int degree,
                        int precision, const int32_t *d_order, float *d_out_xyz, float *d_out_normal,
                        uint8_t *d_status, mls_stream stream);

/*
 * mls_project_backward -- vector-Jacobian product of mls_project (not in the
 * paper): with cotangents gp (of the projected points) and gn (of the
 * normals), the gradients of L = sum_i <gp_i, p'_i> + <gn_i, n_i> with
 * respect to every coordinate and to h, neighbour rows and normal signs held
 * fixed.  Points whose plane is degenerate pass gp to their own position only
 * (their normal counts as constant); with a singular height fit the fitted
 * height counts as zero, as in the forward.
 *
 *   d_xyz, n, d_idx, k, h, degree, precision, d_order   as for mls_project
 *                    (MLS_PREC_FP64 runs the mixed form)
 *   d_grad_out_xyz     device, n x 3 floats: gp
 *   d_grad_out_normal  device, n x 3 floats or NULL (zero)
 *   d_grad_xyz         device, n x 3 floats, overwritten: dL/dx
 *   d_grad_h           device, 1 float, overwritten: dL/dh
 * Deterministic: edge contributions are summed in a fixed order.  Uses
 * stream-ordered scratch (cudaMallocAsync) of about n * (28 + 16 k) bytes.
 */
int mls_project_backward(const float *d_xyz, int64_t n, const int32_t *d_idx, int k, float h, int degree,
                         int precision, const int32_t *d_order, const float *d_grad_out_xyz,
                         const float *d_grad_out_normal, float *d_grad_xyz, float *d_grad_h, mls_stream stream);

/*
 * mls_mean_knn_dist -- bandwidth helper (not in the paper): the mean distance,
 * in FP64, from each point to the entries of its neighbour row other than
 * itself.  Writes one double to d_out (device).  Typical use: h = 2 * value.
 */
int mls_mean_knn_dist(const float *d_xyz, int64_t n, const int32_t *d_idx, int k, double *d_out,
                      mls_stream stream);

/* Number of CUDA kernels this library has launched in the process so far
 * (all threads).  Host-side count, for accounting in benchmarks. */
int64_t mls_kernel_launches(void);

/* Message for the calling thread's most recent failed call ("" if none). */
const char *mls_last_error(void);

/* Static description of a status code. */
const char *mls_status_str(int code);

#ifdef __cplusplus
}
#endif

#endif /* MLS_H_ */
