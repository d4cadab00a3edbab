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
 *   degenerate      (l1 - l0) <= 1e-6 l2, or l2 <= 2^-40 D^2 (covariance
 *                   normalised by the weight sum, D the largest distance from
 *                   the point to a row entry: the neighbours' weights are
 *                   negligible beside its own): output r, status bit 1;
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
 *   - A grid handle holds per-call work space (the kNN's queue and lists, the
 *     pipelined call's side stream): calls on one handle must be ordered on
 *     one stream (or otherwise serialised), never issued from two threads or
 *     two unordered streams at once; different handles are independent.
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
    MLS_ERR_TOO_LARGE = -8           /* n beyond the entry point's limit: the 2^31 - 1 index
                                        range, MLS_NOALLOC_MAX_POINTS for
                                        mls_project_noalloc, (2^31 - 1) / MLS_MAX_K for
                                        mls_project_backward */
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
    MLS_PT_FP64_USED = 4,
    MLS_PT_NOT_CONVERGED = 8,  /* mls_project_levin: t still moving after max_iter passes */
    MLS_PT_OUTLIER = 16,       /* mls_project_rows: too few neighbours, not projected */
    MLS_PT_DEGREE_REDUCED = 32 /* mls_project_rows: fewer points than twice the basis size: a lower degree */
};

#define MLS_MAX_K 64
#define MLS_MAX_K_FUSED 32   /* largest k of mls_knn_project */
/* Floats per point of the fit state mls_project_sorted can save for
 * mls_project_backward_sorted (component c of sorted position s at
 * d_state[c * n + s]): W, m (3), n (3), e1 (3), e2 (3), eigenvalues (3),
 * a (6), A^-1 e_0 (6), status bits (1). */
#define MLS_FIT_STATE_FLOATS 29

/*
 * mls_build_grid -- spatial index for the neighbour search that precedes each
 * fit (Sec. 2.2; the paper builds a k-d tree and mentions Morton reordering of
 * unordered clouds, Sec. 2 introduction).  Here: a uniform grid whose cells are
 * numbered by 63-bit Morton keys, points sorted along the Hilbert curve of the
 * cells with an LSD radix sort (see mls_grid_order), and one hash table per
 * coarsening level (cell side doubling per level) from a base level chosen
 * from the cell occupancy.
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
 *              A rebuilt grid sorts only the key bits from about one level
 *              below its previous base level (fewer radix passes); if the new
 *              cloud needs a finer base than that resolves, it sorts the whole
 *              key again.  Results never depend on it.
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

/* Device pointer to the grid's order of the points: order[s] is the index of
 * the point at sorted position s (n int32, owned by the grid, valid until the
 * grid is rebuilt or destroyed).  The order is the Hilbert-curve order of the
 * level-0 cells (Skilling's index), resolved down to about one level below
 * the base level of the handle's previous build (the whole 63-bit index on a
 * handle's first build); points within one unresolved cell keep their input
 * order.  Every cell of every level searched is a run of consecutive
 * positions.  Passing it to mls_project as d_order makes neighbouring threads
 * work on neighbouring points. */
const int32_t *mls_grid_order(const mls_grid *g);

/*
 * mls_knn -- exact k nearest neighbours of every point of the grid's cloud,
 * itself included (the neighbourhood of Sec. 1.4 / Algorithm 1, read as kNN).
 *
 *   d_idx   device, n x k int32: row i lists point i's neighbours by point
 *           index, ascending by (key, index); bit-exact and deterministic
 *   d_key   device, n x k floats or NULL: the matching keys
 *   k       1 <= k <= min(MLS_MAX_K, n)
 * Scratch: from 2^18 points, 5 n + 32 bytes (the queries alone in a cell two
 * base cells wide, searched first, and their flags).
 */
int mls_knn(const mls_grid *g, int k, int32_t *d_idx, float *d_key, mls_stream stream);

/*
 * mls_knn_sorted -- the same neighbourhoods in the grid's own order, for
 * mls_project_sorted: row s (s = a sorted position, see mls_grid_order)
 * lists the sorted positions of the neighbours of the point at sorted
 * position s, ascending by (key, index) as in mls_knn.
 *   d_pos   device, n x k int32, written
 *   d_idx   device, n x k int32 or NULL: also the rows of mls_knn (original
 *           indexing, row = original index)
 *   d_key   device, n x k floats or NULL: the keys, in d_idx's layout
 * Scratch: as mls_knn.
 */
int mls_knn_sorted(const mls_grid *g, int k, int32_t *d_pos, int32_t *d_idx, float *d_key, mls_stream stream);

/*
 * mls_project_sorted -- mls_project over the grid's sorted copy of the points
 * and rows of sorted positions (from mls_knn_sorted on the same grid, which
 * must not have been rebuilt since): neighbouring threads read neighbouring
 * rows and neighbouring points.  Results are those of mls_project on the
 * matching original-index rows, bit for bit, written in the original order
 * (point i's result at i).  precision MLS_PREC_FP32 or MLS_PREC_MIXED
 * (MLS_ERR_INVALID_ARG for MLS_PREC_FP64: use mls_project).  The grid's
 * points must still be the cloud it was built on.  Scratch: in the mixed form
 * the list of the points that need an FP64 step (4 n bytes).
 *   d_state  device, MLS_FIT_STATE_FLOATS x n floats, or NULL: the fit state
 *            of every point by sorted position (the frame, the fit and the
 *            status the adjoint would otherwise recompute), for
 *            mls_project_backward_sorted; the other outputs are unchanged.
 */
int mls_project_sorted(const mls_grid *g, const int32_t *d_pos, int k, float h, int degree, int precision,
                       float *d_out_xyz, float *d_out_normal, uint8_t *d_status, float *d_state,
                       mls_stream stream);

/*
 * mls_knn_project -- the neighbour search and the projection in one pass
 * (Algorithm 1: each point's k nearest neighbours, then steps of Sec. 1.4,
 * Eq. 1 on them), without writing the rows unless asked: every warp of the
 * kNN keeps the rows of its last 32 queries in an on-chip-sized buffer and
 * projects those points when 32 are done.  Results equal those of
 * mls_knn_sorted followed by mls_project_sorted with the same k, h, degree
 * and precision (same rows, same per-point arithmetic; the mixed form
 * finishes its FP64 points in place instead of in a second pass).
 *   g         grid built on the cloud (mls_build_grid), not rebuilt since
 *   k         1 <= k <= min(MLS_MAX_K_FUSED, n), else MLS_ERR_K_TOO_LARGE
 *   h         Gaussian bandwidth of Eq. 1, finite and > 0 (it is not derived
 *             from the rows here: pass the value the cloud is filtered with)
 *   degree    0, 1 or 2; precision MLS_PREC_FP32 or MLS_PREC_MIXED
 *   d_out_xyz device, n x 3 floats, written in the original order (must not
 *             be the grid's points)
 *   d_out_normal, d_status  device, n x 3 floats / n bytes, or NULL
 *   d_pos     device, n x k int32 or NULL: also the rows of sorted positions
 *             of mls_knn_sorted
 * Scratch: 128 k bytes per resident warp of the kNN (about 20 MB at k = 32).
 */
int mls_knn_project(const mls_grid *g, int k, float h, int degree, int precision, float *d_out_xyz,
                    float *d_out_normal, uint8_t *d_status, int32_t *d_pos, mls_stream stream);

/*
 * mls_knn_project_sorted -- mls_knn_sorted followed by mls_project_sorted (the
 * neighbourhoods of Algorithm 1 and the projection of Sec. 1.4, Eq. 1 over
 * them), pipelined: once the kNN's first pass has written the rows of all but
 * the queries in sparse neighbourhoods, the kNN's second pass runs on a
 * high-priority stream of the grid's own while the projection of the other
 * points runs on `stream` beside it; the points of the second pass, and the
 * isolated queries the first pass took before its runs, are projected after
 * it.  Outputs (d_pos and the projection's, d_state included) equal those of
 * the two calls bit for bit.  Arguments as mls_knn_sorted (d_pos required)
 * and mls_project_sorted.
 * Scratch: 9 n + 32 bytes.  The grid's side stream and two events are created on
 * the first call and destroyed with the grid; `stream` waits for the side
 * stream before the call's last kernel, so the call is ordered on `stream`
 * like any other.
 *   d_offsets  device, n + 1 int32, or NULL: also the offsets of the
 *              adjoint's reverse adjacency of these rows (d_offsets[t] = how
 *              many row entries name sorted positions below t), counted on
 *              the side stream once the rows are complete, for
 *              mls_project_backward_sorted; MLS_ERR_TOO_LARGE when n k does
 *              not fit an int32.
 */
int mls_knn_project_sorted(const mls_grid *g, int k, float h, int degree, int precision, int32_t *d_pos,
                           float *d_out_xyz, float *d_out_normal, uint8_t *d_status, float *d_state,
                           int32_t *d_offsets, mls_stream stream);

/* Number of queries the last kNN call on this grid searched outside the runs
 * of consecutive queries: the isolated ones (alone in a cell two base cells
 * wide), taken first, and those handed to its second pass (whose first key
 * bound needs a cube above the base level: outliers, sparse regions); a
 * measure of the work, never of the result.  Synchronises `stream` (the
 * kNN's stream).  Negative: an error code. */
int64_t mls_knn_deferred(const mls_grid *g, mls_stream stream);

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
 * Outputs must not alias inputs.  Uses stream-ordered scratch (the library's
 * pool): the points as float4 (16 n bytes) and, in MLS_PREC_MIXED, a list of
 * the points that need an FP64 step (4 n bytes), finished by a second, compact
 * pass with the same arithmetic as in line.
 */
int mls_project(const float *d_xyz, int64_t n, const int32_t *d_idx, int k, float h, int degree,
                int precision, const int32_t *d_order, float *d_out_xyz, float *d_out_normal,
                uint8_t *d_status, mls_stream stream);

/*
 * mls_project_levin -- the projection with the weights of Eq. 1 (Sec. 1.4)
 * taken about q = r + t n, the projection of the point onto the reference
 * plane, rather than about the point itself.  Reading of the paper: the
 * plane is self-consistent -- the weighted least-squares plane for weights
 * about the projection of r onto that plane -- and is reached by fixed-point
 * iteration from q = r (t = 0, the smallest t): weights about q, plane, new q,
 * until t changes by at most tol * h.  The height polynomial is then fitted
 * in the frame at the final q with the weights about that q, and the result
 * is q + g(0, 0) n.
 *
 *   arguments as for mls_project, plus
 *   max_iter   1..64 plane passes; points still moving get MLS_PT_NOT_CONVERGED
 *   tol        > 0, convergence threshold on t relative to h (1e-6 typical)
 *   precision  MLS_PREC_FP32 or MLS_PREC_MIXED
 */
int mls_project_levin(const float *d_xyz, int64_t n, const int32_t *d_idx, int k, float h, int degree,
                      int precision, int max_iter, float tol, const int32_t *d_order, float *d_out_xyz,
                      float *d_out_normal, uint8_t *d_status, mls_stream stream);

/*
 * Radius-R neighbourhoods (Sec. 1.4: the points within radius R of the
 * query; Sec. 2.2) and the projection over them with Sec. 3.3's outlier rule.
 * The neighbourhood of point i is every j with key(i, j) <= fl(R * R), the
 * same FP32 key as mls_knn, the point itself included, ordered by (key,
 * index): bit-exact like the kNN rows.
 *
 * mls_radius_count: d_count (n int32, original order) = size of each
 *   neighbourhood; with d_offsets (n + 1 int64) non-NULL also the CSR
 *   offsets (exclusive prefix sum; d_offsets[n] = total).  Asynchronous.
 * mls_radius_rows: writes row i at d_rows[d_offsets[i] ..] (and the keys to
 *   d_keys when non-NULL).  At most MLS_MAX_RADIUS_NB neighbours per point:
 *   synchronises `stream` and returns MLS_ERR_K_TOO_LARGE (rows of such
 *   points unwritten) when any neighbourhood is larger.
 * mls_project_rows: the projection (weights about the point, as mls_project)
 *   over CSR neighbourhoods (d_offsets n + 1 int64, d_rows int32, rows of any
 *   length); a point with fewer than min_neighbors (>= 0) OTHER points in its
 *   row is an outlier: not projected, output = the point, normal = 0, status
 *   MLS_PT_OUTLIER.  A row of m points (the point included) is fitted at the
 *   highest degree <= `degree` whose basis has at most m / 2 coefficients
 *   (degree 2 needs m >= 12, degree 1 m >= 6), status MLS_PT_DEGREE_REDUCED
 *   when lowered: fewer points would be interpolated rather than smoothed.
 *   precision MLS_PREC_FP32 or MLS_PREC_MIXED.
 * mls_compact: d_kept (capacity n int32) = the indices i with
 *   (d_status[i] & mask) == 0 in increasing order; *d_num_kept (device int64)
 *   = their number (the paper's result drops the outliers: mask =
 *   MLS_PT_OUTLIER).
 */
#define MLS_MAX_RADIUS_NB 128
int mls_radius_count(const mls_grid *g, float R, int32_t *d_count, int64_t *d_offsets, mls_stream stream);
int mls_radius_rows(const mls_grid *g, float R, const int64_t *d_offsets, int32_t *d_rows, float *d_keys,
                    mls_stream stream);
int mls_project_rows(const float *d_xyz, int64_t n, const int64_t *d_offsets, const int32_t *d_rows, float h,
                     int degree, int precision, int min_neighbors, const int32_t *d_order, float *d_out_xyz,
                     float *d_out_normal, uint8_t *d_status, mls_stream stream);
int mls_compact(const uint8_t *d_status, int64_t n, int mask, int32_t *d_kept, int64_t *d_num_kept,
                mls_stream stream);

/*
 * mls_project_noalloc -- mls_project for callers that must not allocate
 * device memory.  The paper has no counterpart: this is a deployment
 * variant.  Some callers cannot let a library allocate: hosts that hand out
 * all device memory from their own fixed pool or budget (inference servers,
 * embedded pipelines) and would not see the library's own pool, or loops that must
 * not risk an allocation failing half way.  This entry point takes its
 * scratch (a float4 copy of the points) from a fixed device array of
 * MLS_NOALLOC_MAX_POINTS entries (4 MiB), which every GPU that loads the
 * library holds until the process exits; it calls no allocation routine.
 *
 * Arguments, outputs and results are those of mls_project.
 * Returns MLS_ERR_TOO_LARGE when n > MLS_NOALLOC_MAX_POINTS.
 * Every call made outside a stream capture looks the array's device address
 * up (with the device current), so a cudaDeviceReset between calls leaves
 * no stale address behind; a call made during a capture uses the address
 * found by the last call on that device, so make a first call on each device
 * before any stream capture.
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
 * Deterministic: each coordinate's gradient is the exact sum (64-bit fixed
 * point at a power-of-two scale chosen per point and component from the
 * largest term) of its terms, rounded once to float, so it depends neither on
 * scheduling nor on d_order.  Uses stream-ordered scratch (the library's pool,
 * see mls_release_scratch) of about n * (48 + 16 k) bytes.
 */
int mls_project_backward(const float *d_xyz, int64_t n, const int32_t *d_idx, int k, float h, int degree,
                         int precision, const int32_t *d_order, const float *d_grad_out_xyz,
                         const float *d_grad_out_normal, float *d_grad_xyz, float *d_grad_h, mls_stream stream);

/*
 * mls_project_backward_sorted -- mls_project_backward over the grid's sorted
 * copy of the points and the rows of sorted positions of mls_knn_sorted (the
 * grid not rebuilt since, its points still the cloud it was built on): the
 * same gradients bit for bit as mls_project_backward on the matching
 * original-index rows with the grid's order, without that form's repacking
 * of the points and translation of the rows.  d_grad_out_xyz,
 * d_grad_out_normal and d_grad_xyz in the original order, as there.
 * precision MLS_PREC_FP32 or MLS_PREC_MIXED.  Scratch: about n (32 + 16 k)
 * bytes.
 *   d_state  device, MLS_FIT_STATE_FLOATS x n floats, or NULL: the fit state
 *            mls_project_sorted saved with the same rows, h, degree and
 *            precision.  Given, the adjoint reads each point's frame, fit and
 *            status from it instead of recomputing them (two of its four
 *            passes over the neighbours and the solves): the gradients then
 *            differ from the recomputing form only by rounding (the saved
 *            coefficients carry the forward's refinement step).
 *   d_offsets  device, n + 1 int32, or NULL: the bucket offsets
 *            mls_knn_project_sorted counted for these rows (else counted
 *            here); the gradients do not depend on it.
 */
int mls_project_backward_sorted(const mls_grid *g, const int32_t *d_pos, int k, float h, int degree, int precision,
                                const float *d_grad_out_xyz, const float *d_grad_out_normal, float *d_grad_xyz,
                                float *d_grad_h, const float *d_state, const int32_t *d_offsets,
                                mls_stream stream);

/*
 * mls_mean_knn_dist -- bandwidth helper (not in the paper): the mean distance,
 * in FP64, from each point to the entries of its neighbour row other than
 * itself.  Writes one double to d_out (device).  Typical use: h = 2 * value.
 */
int mls_mean_knn_dist(const float *d_xyz, int64_t n, const int32_t *d_idx, int k, double *d_out,
                      mls_stream stream);

/*
 * Batched projection -- many independent clouds in one persistent launch.
 * Algorithm 1 projects every point of one cloud independently; here that
 * per-point loop runs over the union of B clouds of uneven size, each with
 * its own k and h, in a single kernel whose blocks take tiles of points from
 * a shared counter (the paper has no batched form; its per-point arithmetic is
 * that of mls_project).  A batch handle fixes the cloud sizes and k; the
 * point data can change between launches.
 *
 * Layouts (all DEVICE memory owned by the caller):
 *   d_xyz    total x 3 floats: the clouds one after another, cloud c at rows
 *            offsets[c] .. offsets[c+1]-1
 *   d_idx    the clouds' neighbour rows one after another: cloud c's n_c x k_c
 *            rows start at element mls_batch_idx_offset(b, c) =
 *            sum_{c' < c} n_c' k_c', with indices LOCAL to the cloud (0..n_c-1),
 *            as mls_knn writes them for that cloud alone
 *   d_order  total int32 or NULL: cloud c's slice is a permutation of 0..n_c-1
 *            (e.g. its mls_grid_order); speed only, never results
 *   d_h      B floats: each cloud's bandwidth, finite and > 0
 *   outputs  d_out_xyz total x 3, d_out_normal total x 3 or NULL, d_status
 *            total bytes or NULL, at the input's rows
 * degree 0, 1 or 2; precision MLS_PREC_FP32 or MLS_PREC_MIXED.
 */
typedef struct mls_batch mls_batch;

/* Creates a batch of `batch` clouds: h_offsets (HOST, batch + 1 entries,
 * offsets[0] = 0, every cloud at least one point, total < 2^31) and h_k (HOST,
 * batch entries, 1 <= k_c <= min(MLS_MAX_K, n_c)).  Allocates about
 * 16 x total bytes of device scratch on the current device and synchronises.
 * Launch shape starts at 1 lane per point, 128 threads, 1 round per tile. */
int mls_batch_create(int batch, const int64_t *h_offsets, const int32_t *h_k, mls_batch **out);

/* Synchronises the device and frees the batch (NULL is ignored). */
void mls_batch_destroy(mls_batch *b);

/* Total points of the batch (-1 for NULL). */
int64_t mls_batch_total(const mls_batch *b);

/* Element offset of cloud `cloud`'s rows in d_idx (cloud = batch gives the
 * total length); -1 for a bad argument. */
int64_t mls_batch_idx_offset(const mls_batch *b, int cloud);

/* Launch shape: lanes_per_point in {1, 2, 4, 8, 16, 32} (G lanes share a
 * point's neighbours and merge their moments), threads per block (multiple of
 * 32, <= 256), rounds of blockDim / G points per tile (1..64).  Changing the
 * shape drops a captured graph.  Synchronous. */
int mls_batch_set_shape(mls_batch *b, int lanes_per_point, int threads, int rounds);
int mls_batch_get_shape(const mls_batch *b, int *lanes_per_point, int *threads, int *rounds);

/* One batched projection on `stream`: a 4-byte memset of the tile counter, a
 * float4 copy of the points, and the persistent projection kernel. */
int mls_project_batched(mls_batch *b, const float *d_xyz, const int32_t *d_idx, const int32_t *d_order,
                        const float *d_h, int degree, int precision, float *d_out_xyz, float *d_out_normal,
                        uint8_t *d_status, mls_stream stream);

/* Captures mls_project_batched with these buffers (on a private stream) into a
 * CUDA graph held by the batch, replacing any earlier one.  Nothing runs.  The
 * buffers must stay valid while the graph is replayed; their contents (points,
 * rows, h) may change between replays. */
int mls_batch_capture(mls_batch *b, const float *d_xyz, const int32_t *d_idx, const int32_t *d_order,
                      const float *d_h, int degree, int precision, float *d_out_xyz, float *d_out_normal,
                      uint8_t *d_status);

/* Launches the captured graph on `stream`. */
int mls_batch_replay(mls_batch *b, mls_stream stream);

/* Autotuner: runs every candidate shape (lanes 1, 2, 4, 8 x threads 64, 128,
 * 256 x rounds 1, 4) once untimed and `reps` times timed with CUDA events on
 * `stream`, keeps the fastest, and leaves that shape's results in the outputs.
 * Synchronises `stream`.  Results of different shapes agree to rounding (the
 * lanes of a point sum in a different order). */
int mls_batch_autotune(mls_batch *b, const float *d_xyz, const int32_t *d_idx, const int32_t *d_order,
                       const float *d_h, int degree, int precision, float *d_out_xyz, float *d_out_normal,
                       uint8_t *d_status, int reps, mls_stream stream);

/* The last autotune's timings: up to `capacity` entries of (lanes, threads,
 * rounds) into shapes (3 int32 each, HOST) and the best time in ms into ms
 * (HOST); either may be NULL.  Returns the number of entries. */
int mls_batch_tune_results(const mls_batch *b, int capacity, int32_t *shapes, float *ms);

/*
 * mls_points_in_boxes -- the halo test of one cloud split over ranks (the
 * paper's contiguous segments, Sec. 2.1, exchanged exactly): sets
 * d_mask[i] = 1 for every point i of the grid's cloud that lies inside at
 * least one of the m axis-aligned boxes (closed: lo <= x <= hi on each axis),
 * and leaves every other entry as it was (zero it first).
 *   d_boxes  device, m x 6 floats: lo x, y, z, hi x, y, z (an empty or NaN
 *            box selects nothing); m >= 0
 *   d_mask   device, n bytes, original order
 * One warp per box over the grid's cells; cost grows with the number of
 * cells a box covers at the base level (a box far larger than the cloud's
 * cells is visited at a coarse level).  Asynchronous on `stream`.
 */
int mls_points_in_boxes(const mls_grid *g, const float *d_boxes, int64_t m, uint8_t *d_mask, mls_stream stream);

/* Scratch memory.  mls_project, mls_project_backward and the helpers take
 * their per-call buffers, stream-ordered, from a memory pool of the library's
 * own (one per device) that keeps freed memory mapped for the next call
 * instead of returning it to the system at every synchronisation.  This call
 * synchronises every device that has such a pool and returns its unused
 * memory to the system.  A cudaDeviceReset destroys a device's pool with the
 * rest of its context: do not reset a device that this library has used while
 * the process still calls it. */
int mls_release_scratch(void);

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
