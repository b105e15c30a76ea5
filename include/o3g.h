/*
 * o3g.h - C ABI of the GB300-native point-to-plane ICP library (libo3g.so).
 *
 * The library implements the local-refinement step of Open3D's pairwise
 * registration workflow (arXiv 1801.09847, Sec. 3.3, registration_icp with
 * TransformationEstimationPointToPlane) and the normal estimation that feeds it
 * (Fig. 1 and Sec. 3.3, estimate_normals with KDTreeSearchParamHybrid), on one
 * CUDA GPU.  The iteration is the Gauss-Newton step of Sec. 4, Eq. (1)-(2).
 *
 * Conventions shared by every entry point
 *  - Return value: an o3g_status code.  Negative = error: outputs are left
 *    untouched and o3g_last_error() describes the failure.  Positive = warning:
 *    outputs are valid.  No C++ exception and no abort crosses this boundary.
 *  - Point clouds are float32.  Point i of a cloud is (xyz[i*stride],
 *    xyz[i*stride+1], xyz[i*stride+2]); stride >= 3 floats.  Device pointers
 *    (prefix d_) are caller-owned, read-only unless documented as outputs, and
 *    never freed by the library.  They must stay valid until the call returns
 *    or, for asynchronous calls, until the stream has passed the work.
 *  - Poses are 4x4 row-major float64 matrices in HOST memory that map source
 *    coordinates into the target frame: q = T[0:3,0:3] p + T[0:3,3].
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls that return host-side results synchronise that stream
 *    before returning; the others only enqueue work.
 *  - The library allocates device memory from a private stream-ordered pool.
 *    Handles (o3g_grid) are library-owned and released with o3g_free_grid.
 *  - Non-finite input coordinates are rejected with O3G_ERR_NONFINITE.
 *  - The ICP sums over all correspondences are accumulated exactly as 64-bit
 *    fixed-point integers scaled by a-priori bounds (the number of source
 *    points, the radius, the target's coordinate box and the largest length of
 *    its normals), so they do not depend on the order of accumulation.  A term
 *    outside its bound (a NaN normal, say) makes the sums unusable and the call
 *    returns O3G_ERR_NONFINITE.
 *  - Thread safety: calls on different handles may run concurrently from
 *    different host threads; a handle must not be used by two calls at once.
 */
#ifndef O3G_H
#define O3G_H

#include <stdint.h>

#if defined(__GNUC__)
#define O3G_API __attribute__((visibility("default")))
#else
#define O3G_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  O3G_OK = 0,
  O3G_WARN_DEGENERATE = 1, /* some 6x6 pivot was frozen (unobservable DOF); pose still valid */
  O3G_WARN_FEW_CORR = 2,   /* ICP stopped early: fewer than 6 correspondences */
  O3G_ERR_ARG = -1,        /* invalid argument (null pointer, negative size, bad stride, ...) */
  O3G_ERR_OOM = -2,        /* device allocation failed */
  O3G_ERR_CUDA = -3,       /* a CUDA runtime call failed; see o3g_last_error() */
  O3G_ERR_NONFINITE = -4,  /* a coordinate, a normal or the pose is NaN or infinite */
  O3G_ERR_TIMEOUT = -5     /* reserved for a bounded device-side wait that gives up; no entry point of this
                              library returns it, since no kernel here waits on a flag */
} o3g_status;

/* Largest max_nn accepted by the hybrid search and normal estimation. */
#define O3G_MAX_NN 64

/* Opaque uniform grid over one point cloud, resident in device memory. */
typedef struct o3g_grid o3g_grid;

/* Human-readable description of the last error on the calling host thread. */
O3G_API const char* o3g_last_error(void);

/* ABI version of this header (bumped on any signature change). */
O3G_API int32_t o3g_abi_version(void);

/*
 * Builds the device uniform grid that replaces Open3D's kd-tree (Sec. 2: FLANN
 * for nearest-neighbour search) for fixed-radius and hybrid queries.
 *   d_xyz, n, stride : the cloud (device); n may be 0.
 *   cell_size        : edge of a grid cell (> 0).  Any query radius works with
 *                      any cell size; a cell near the typical query radius is
 *                      fastest.  If the cloud's bounding box would need more
 *                      than 32*n + 2^20 cells the library enlarges the cell.
 *   out              : receives the handle.
 * The grid copies the points (sorted by cell) and does not keep d_xyz.
 * Synchronises `stream` once (to size the grid from the bounding box).
 */
O3G_API int32_t o3g_build_grid(const float* d_xyz, int64_t n, int32_t stride, float cell_size, void* stream,
                       o3g_grid** out);

/* Releases a grid (NULL is accepted).  Enqueued on the stream given at build. */
O3G_API int32_t o3g_free_grid(o3g_grid* grid);

/* Number of points and the cell size actually used. */
O3G_API int32_t o3g_grid_info(const o3g_grid* grid, int64_t* n, float* cell_size);

/*
 * Attaches normals to a grid's points (Sec. 3.1: normals are valid only when
 * they have as many records as the points -> n != grid's n gives O3G_ERR_ARG).
 * d_nrm is read in the caller's point order and copied into the grid, and the
 * largest normal length is recorded (it bounds the ICP sums; normals need not
 * be unit length).  Asynchronous.
 */
O3G_API int32_t o3g_grid_set_normals(o3g_grid* grid, const float* d_nrm, int64_t n, int32_t stride, void* stream);

/*
 * Hybrid radius/kNN search (KDTreeSearchParamHybrid(radius, max_nn), Fig. 1):
 * for each query, the at most max_nn grid points with
 *   d2 = (dx*dx + dy*dy) + dz*dz <= fl(radius)*fl(radius)   (float32, each op rounded),
 * ordered by (d2, point index); indices are the grid cloud's original indices.
 *   d_idx [nq*max_nn] int32, -1 padded;  d_d2 [nq*max_nn] float32, 0 padded;
 *   d_cnt [nq] int32.  1 <= max_nn <= O3G_MAX_NN.  Asynchronous.
 */
O3G_API int32_t o3g_knn_hybrid(const o3g_grid* grid, const float* d_qry, int64_t nq, int32_t stride, float radius,
                       int32_t max_nn, int32_t* d_idx, float* d_d2, int32_t* d_cnt, void* stream);

/*
 * estimate_normals(pc, KDTreeSearchParamHybrid(radius, max_nn)) (Fig. 1,
 * Sec. 3.3) for the grid's own points: the hybrid neighbourhood of each point
 * (itself included), covariance of the neighbourhood about its mean divided by
 * m, unit eigenvector of the smallest eigenvalue, turned so that
 * n . (viewpoint - q) >= 0.  Fewer than 3 neighbours give (0, 0, 1).
 *   viewpoint  : 3 floats in host memory (NULL = origin).
 *   d_nrm_out  : n x nrm_stride floats (device) in the caller's point order, or
 *                NULL to only keep them in the grid.
 * The normals are also attached to the grid (as o3g_grid_set_normals would).
 * Asynchronous.
 */
O3G_API int32_t o3g_estimate_normals(o3g_grid* grid, float radius, int32_t max_nn, const float* viewpoint,
                             float* d_nrm_out, int32_t nrm_stride, void* stream);

/*
 * Normal estimation for many clouds in one launch (the step before every
 * registration, Sec. 3.3: both clouds of a pair, or every target of a batch).
 * Cloud c gets exactly what o3g_estimate_normals(grids[c], radius[c], max_nn,
 * viewpoints + 3 c, d_out[c], out_strides[c]) would give it.  grids: host
 * array of n_grids handles; radius: host array; viewpoints: host n_grids x 3
 * or NULL (origins); d_out: host array of device pointers (entries may be
 * NULL) or NULL; out_strides: host array or NULL (3).  max_nn > 32 runs one
 * launch per cloud.  Synchronous.
 */
O3G_API int32_t o3g_estimate_normals_batch(int32_t n_grids, o3g_grid* const* grids, const float* radius, int32_t max_nn,
                                           const float* viewpoints, float* const* d_out, const int32_t* out_strides,
                                           void* stream);

/*
 * Hybrid kNN queries against many grids in one launch: query set c (d_qry[c],
 * nq[c] rows of strides[c] floats) against grids[c] with radius[c], outputs as
 * o3g_knn_hybrid gives them in d_idx[c], d_d2[c], d_cnt[c].  All arrays are
 * host arrays of n_grids entries.  Synchronous.
 */
O3G_API int32_t o3g_knn_hybrid_batch(int32_t n_grids, const o3g_grid* const* grids, const float* const* d_qry,
                                     const int64_t* nq, const int32_t* strides, const float* radius, int32_t max_nn,
                                     int32_t* const* d_idx, float* const* d_d2, int32_t* const* d_cnt, void* stream);

/*
 * Correspondence step of registration_icp at a given pose (Sec. 3.3):
 * p_i = R s_i + t in float32 with R, t rounded to nearest from T and each row
 * evaluated as ((R0 sx + R1 sy) + R2 sz) + t, no fused multiply-add; then the
 * target j minimising (d2(p_i, q_j), j) with d2 <= fl(max_corr_dist)^2.
 *   d_corr [ns] int32 : original target index, or -1.   d_d2 [ns] float32 (0 if none).
 * Asynchronous.
 */
O3G_API int32_t o3g_correspondences(const o3g_grid* tgt, const float* d_src, int64_t ns, int32_t stride,
                            const double* T, float max_corr_dist, int32_t* d_corr, float* d_d2, void* stream);

/*
 * Gauss-Newton normal equations at a given pose (Sec. 4, Eq. 1-2):
 * over the correspondences of o3g_correspondences, r_i = (p_i - q_i) . n_i,
 * J_i = [p_i x n_i ; n_i] (target normals), and
 *   out_A [36] = sum J J^T (row-major, symmetric),  out_b [6] = sum J r,
 *   out_stats [3] = (sum r^2, sum d2, |C|).
 * Per-correspondence arithmetic is float32 with compensated block sums, which
 * are added across blocks as exact 64-bit fixed point and converted to float64
 * once.  Requires normals on the target grid.  A non-finite source coordinate
 * or a sum left unusable by a non-finite normal: O3G_ERR_NONFINITE.  Synchronous.
 */
O3G_API int32_t o3g_normal_equations(const o3g_grid* tgt, const float* d_src, int64_t ns, int32_t stride, const double* T,
                             float max_corr_dist, double* out_A, double* out_b, double* out_stats, void* stream);

/*
 * Arithmetic of the per-correspondence terms and of the block sums.
 *   O3G_PREC_F32_COMPENSATED  J, r and the 27 products in float32, block sums
 *                             compensated (TwoSum pairs), cross-block sums exact
 *                             in 64-bit fixed point, the solve in float64 (the
 *                             default everywhere).
 *   O3G_PREC_F64              J, r and the products in float64 from the float32
 *                             points and normals, each operation rounded once in
 *                             the order r = ((dx nx + dy ny) + dz nz), block sums
 *                             in plain float64, then the same fixed-point
 *                             cross-block sums (the precision study's all-FP64
 *                             variant).
 * Correspondences and the float32 transform are the same under both.
 */
typedef enum { O3G_PREC_F32_COMPENSATED = 0, O3G_PREC_F64 = 1 } o3g_precision;

/*
 * o3g_normal_equations with a chosen o3g_precision; an unknown value is
 * O3G_ERR_ARG.  Synchronous.
 */
O3G_API int32_t o3g_normal_equations_ex(const o3g_grid* tgt, const float* d_src, int64_t ns, int32_t stride,
                                        const double* T, float max_corr_dist, int32_t precision, double* out_A,
                                        double* out_b, double* out_stats, void* stream);

/*
 * Point-to-plane ICP against a resident target grid that carries normals
 * (registration_icp(source, target, max_correspondence_distance, init,
 * TransformationEstimationPointToPlane()), Sec. 3.3).  Each iteration: the
 * correspondence step, the normal equations, the solve of
 * (J^T J) xi = -J^T r (Eq. 2; pivots those of LDL^T) with
 * xi = (alpha, beta, gamma, tx, ty, tz), and
 * T <- [Rz(gamma) Ry(beta) Rx(alpha), t; 0 1] T.  A pivot D_kk <= 1e-12 max_j A_jj
 * freezes its unknown (status O3G_WARN_DEGENERATE).  Iteration stops after
 * max_iter updates, when fewer than 6 correspondences remain
 * (O3G_WARN_FEW_CORR, pose of the last update kept), or when
 * max(|(alpha,beta,gamma)|, |t|) < eps after an update (eps <= 0: never).
 * Results at the final pose: fitness = |C| / ns, rmse = sqrt(sum d2 / |C|)
 * (0 when C is empty).  out_iters may be NULL.  All iteration state stays on
 * the device; synchronous.
 */
O3G_API int32_t o3g_icp_point_to_plane_grid(const o3g_grid* tgt, const float* d_src, int64_t ns, int32_t stride,
                                    const double* init_T, double max_corr_dist, int32_t max_iter, double eps,
                                    double* out_T, double* out_fitness, double* out_rmse, int32_t* out_iters,
                                    void* stream);

/*
 * o3g_icp_point_to_plane_grid with a chosen o3g_precision for every iteration
 * and for the final evaluation; an unknown value is O3G_ERR_ARG.
 */
O3G_API int32_t o3g_icp_point_to_plane_grid_ex(const o3g_grid* tgt, const float* d_src, int64_t ns, int32_t stride,
                                               const double* init_T, double max_corr_dist, int32_t max_iter,
                                               double eps, int32_t precision, double* out_T, double* out_fitness,
                                               double* out_rmse, int32_t* out_iters, void* stream);

/*
 * o3g_icp_point_to_plane_grid_ex that also returns the correspondence set at
 * the final pose (the correspondence_set of Open3D's RegistrationResult,
 * Sec. 3.3): d_corr [ns] int32 = the original target index matched to source
 * point i (in the caller's order), or -1; d_d2 [ns] float32 = its squared
 * distance (0 if none).  Both device, caller-owned; null with ns > 0 is
 * O3G_ERR_ARG.  The set is the one fitness and rmse are computed from, found by
 * the same warm-started search as the iterations.  Synchronous.
 */
O3G_API int32_t o3g_icp_point_to_plane_grid_corr(const o3g_grid* tgt, const float* d_src, int64_t ns, int32_t stride,
                                                 const double* init_T, double max_corr_dist, int32_t max_iter,
                                                 double eps, int32_t precision, double* out_T, double* out_fitness,
                                                 double* out_rmse, int32_t* out_iters, int32_t* d_corr, float* d_d2,
                                                 void* stream);

/*
 * Point-to-point ICP against a resident target grid (registration_icp with
 * TransformationEstimationPointToPoint, Sec. 3.3; target normals not needed).
 * Each iteration: the correspondence step of o3g_correspondences at the current
 * pose, then the rigid motion (R, t) minimising sum_i |R p_i + t - q_i|^2 over
 * the correspondences in closed form (Horn's unit-quaternion solution: centroids,
 * centred cross-covariance, the eigenvector of the largest eigenvalue of Horn's
 * symmetric 4x4), and T <- [R t; 0 1] T.  Stops after max_iter updates, with
 * O3G_WARN_FEW_CORR when fewer than 3 correspondences remain (pose of the last
 * update kept), or when max(angle(R), |t|) < eps (eps <= 0: never).  When the
 * two largest eigenvalues of that 4x4 are within 1e-6 E0, E0 = (sum|p - mean p|^2
 * + sum|q - mean q|^2) / 2, the rotation is not determined (for example
 * collinear matches): R = I, t = mean q - mean p and the status is
 * O3G_WARN_DEGENERATE.  Results as in o3g_icp_point_to_plane_grid.
 * Synchronous.
 */
O3G_API int32_t o3g_icp_point_to_point_grid(const o3g_grid* tgt, const float* d_src, int64_t ns, int32_t stride,
                                            const double* init_T, double max_corr_dist, int32_t max_iter, double eps,
                                            double* out_T, double* out_fitness, double* out_rmse, int32_t* out_iters,
                                            void* stream);

/*
 * One-shot form of the above on raw device clouds: builds a grid over the
 * target (cell = 1.002 x max_corr_dist), attaches d_tgt_nrm (n_nrm must equal nt,
 * Sec. 3.1), runs ICP with eps = 0 on the legacy default stream and frees the
 * grid.
 */
O3G_API int32_t o3g_icp_point_to_plane(const float* d_src, int64_t ns, int32_t src_stride, const float* d_tgt, int64_t nt,
                               int32_t tgt_stride, const float* d_tgt_nrm, int64_t n_nrm, int32_t nrm_stride,
                               const double* init_T, double max_corr_dist, int32_t max_iter, double* out_T,
                               double* out_fitness, double* out_rmse);

/*
 * The whole pairwise refinement from DEVICE buffers (Sec. 3.3: estimate_normals
 * on the target, then registration_icp with TransformationEstimationPointToPlane()):
 * builds the target grid (cell = 1.002 x max_corr_dist), attaches d_tgt_nrm
 * (nt normals, nrm_stride floats per row) or, if it is NULL, estimates target
 * normals (normal_radius, normal_max_nn, viewpoint = origin), runs ICP (as
 * o3g_icp_point_to_plane_grid with eps) and frees the grid.  d_src / d_tgt are
 * device xyz rows of src_stride / tgt_stride floats (>= 3), read only.  The
 * source's spatial sort runs on a library-owned stream beside `stream` while the
 * grid is built and the normals are computed (events order it after the work
 * already on `stream` and the iterations after it), so the result equals the
 * separate calls bit for bit.  Results in host memory; synchronous; status codes
 * as o3g_icp_point_to_plane_grid, plus those of o3g_build_grid and the normals.
 */
O3G_API int32_t o3g_register_point_to_plane(const float* d_src, int64_t ns, int32_t src_stride, const float* d_tgt,
                                            int64_t nt, int32_t tgt_stride, const float* d_tgt_nrm,
                                            int32_t nrm_stride, float normal_radius, int32_t normal_max_nn,
                                            const double* init_T, double max_corr_dist, int32_t max_iter, double eps,
                                            double* out_T, double* out_fitness, double* out_rmse, int32_t* out_iters,
                                            void* stream);

/*
 * The whole pairwise refinement from HOST buffers (the call a user with data in
 * host memory makes): copies source and target to the device, builds the
 * target grid (cell = 1.002 x max_corr_dist), attaches h_tgt_nrm or, if it is NULL,
 * estimates target normals (normal_radius, normal_max_nn, viewpoint = origin),
 * runs ICP and returns the results in host memory (o3g_register_point_to_plane
 * on the copies).  h_src, h_tgt and h_tgt_nrm are packed xyz (stride 3);
 * page-locked buffers make the copies asynchronous.
 */
O3G_API int32_t o3g_register_point_to_plane_host(const float* h_src, int64_t ns, const float* h_tgt, int64_t nt,
                                         const float* h_tgt_nrm, float normal_radius, int32_t normal_max_nn,
                                         const double* init_T, double max_corr_dist, int32_t max_iter, double eps,
                                         double* out_T, double* out_fitness, double* out_rmse, int32_t* out_iters,
                                         void* stream);

/*
 * Batched point-to-plane ICP: n_pairs independent registrations, each exactly
 * as o3g_icp_point_to_plane_grid would run it alone (same arithmetic in the same
 * order, so the same result), advanced together: every iteration is one
 * persistent kernel launch whose blocks walk the (pair, tile) work items of all
 * pairs, and each pair stops on its own criterion.  The iteration sequence is
 * captured once as a CUDA graph and launched.
 *   tgts[p]                         target grid of pair p, with normals
 *   d_src[p], ns[p], strides[p]     source cloud of pair p (device pointers)
 *   init_T                          n_pairs x 16 row-major float64 poses
 *   max_corr_dist                   n_pairs radii
 *   out_T (n_pairs x 16), out_fitness, out_rmse, out_iters, out_status (n_pairs each)
 * All arrays are host memory.  The return value reports the call (an error
 * leaves every output untouched); out_status[p] holds pair p's status
 * (O3G_OK, a warning, or O3G_ERR_NONFINITE).  Synchronous.
 */
O3G_API int32_t o3g_icp_point_to_plane_batch(int32_t n_pairs, const o3g_grid* const* tgts, const float* const* d_src,
                                             const int64_t* ns, const int32_t* strides, const double* init_T,
                                             const double* max_corr_dist, int32_t max_iter, double eps,
                                             double* out_T, double* out_fitness, double* out_rmse,
                                             int32_t* out_iters, int32_t* out_status, void* stream);

/*
 * Launch configuration of the iteration kernels per size class (the knob the
 * autotuner sets; no counterpart in the paper).  size_class = floor(log2(work
 * tiles of a launch)), 0..31, a tile being 128 source points (of one pair, or of
 * one pose in o3g_evaluate_poses).  cfg: 0 automatic (the latency form -- large
 * shared-memory stage, 5 blocks per SM -- while every tile of the launch is
 * resident at once in it, else the throughput form -- per-thread searches from
 * global memory, candidate lists on large pairs, 9 blocks per SM; for pose
 * evaluation a smaller stage, 7 blocks per SM), 1 latency form, 2 throughput
 * form.  Process-wide; results do not
 * depend on it (both forms compute the same thing in the same order), only the
 * time does.  o3g_get_tile_config returns the setting or O3G_ERR_ARG.
 */
O3G_API int32_t o3g_set_tile_config(int32_t size_class, int32_t cfg);
O3G_API int32_t o3g_get_tile_config(int32_t size_class);

/*
 * Points per thread of the ICP iteration kernels (the autotuner's second knob;
 * no counterpart in the paper): a tile of the iteration kernel is ppt
 * consecutive groups of 128 spatially sorted source points, reduced group by
 * group into one partial of the pair's sums.  Set per size class of the PAIR,
 * size_class = floor(log2(source points)), 0..31, so that a registration tiles
 * the same way alone, in a batch and in the server (and gives the same result
 * in all three).  ppt: 0 automatic (1 below 2^18 points, 2 below 2^20, 4 from there), 1, 2 or
 * 4; anything else, or a class outside 0..31, is O3G_ERR_ARG.  A different ppt
 * changes the order in which the block partials are formed, so results change
 * in the last bits (within the parity tolerances).  Process-wide.
 * o3g_get_points_per_thread returns the setting or O3G_ERR_ARG.
 */
O3G_API int32_t o3g_set_points_per_thread(int32_t size_class, int32_t ppt);
O3G_API int32_t o3g_get_points_per_thread(int32_t size_class);

/*
 * Hypothesis validation (the step RANSAC-based global registration spends its
 * time in, Sec. 3.3): for each candidate pose T_h, the correspondence step of
 * o3g_correspondences at T_h over the whole source, then
 *   out_fitness[h] = |C_h| / ns,  out_rmse[h] = sqrt(sum_{C_h} d2 / |C_h|)
 *   (0 when C_h is empty),  out_inliers[h] = |C_h| (may be NULL).
 * poses: n_poses x 16 row-major float64, host.  Outputs: host arrays of
 * n_poses.  The target grid needs no normals.  A non-finite pose or source
 * coordinate: O3G_ERR_NONFINITE.  Synchronous.
 */
O3G_API int32_t o3g_evaluate_poses(const o3g_grid* tgt, const float* d_src, int64_t ns, int32_t stride, int32_t n_poses,
                                   const double* poses, double max_corr_dist, double* out_fitness, double* out_rmse,
                                   int64_t* out_inliers, void* stream);

/*
 * Voxel downsampling (voxel_down_sample, Sec. 3.1 and Fig. 1): one output point
 * per occupied voxel, the centroid of the input points in it.
 *   voxel index  (floor(x / voxel), floor(y / voxel), floor(z / voxel)), each
 *                quotient one correctly rounded float32 division
 *   order        voxels in increasing (ix, iy, iz), x most significant
 *   centroid     float64 sum of the voxel's points in increasing input index,
 *                divided by their count, rounded to float32
 * Points with a non-finite coordinate are dropped.  d_xyz: n rows of `stride`
 * floats (x, y, z first), device, caller-owned.  d_out: device, caller-owned,
 * room for 3 n floats (packed xyz; *out_n rows are written).  d_counts: device,
 * room for n int32 (points per voxel), or NULL.  A voxel index outside
 * [-2^30, 2^30], voxel <= 0 or not finite: O3G_ERR_ARG (outputs untouched).
 * Synchronous.
 */
O3G_API int32_t o3g_voxel_down_sample(const float* d_xyz, int64_t n, int32_t stride, float voxel, float* d_out,
                                      int32_t* d_counts, int64_t* out_n, void* stream);

/*
 * Serving: registration requests of any size handled as a continuously batched
 * loop on one stream.  Requests wait in a first-come-first-served queue until a
 * slot (max_active) and the device-memory budget (hbm_budget_bytes, estimated
 * per request from its sizes) allow their admission; admission copies the
 * request's clouds to the device, builds its target grid (cell = 1.002 x
 * max_corr_dist), attaches or estimates target normals and lays out its source,
 * on a stream of the library's own, so that it overlaps the iterations already
 * enqueued.  Each o3g_server_step then makes 8 persistent launches; in each,
 * every admitted request advances by one stage of its own, decided on the
 * device: an ICP iteration, or, once it has converged, stopped or used max_iter
 * iterations, its final evaluation.  The step reads the requests' state back
 * once, after the 8 launches, and retires the evaluated ones (their results
 * wait for o3g_server_poll).  Target grids and per-request pose state stay
 * resident on the device between steps.  Each request's result is the one the single-pair
 * entry points give for it (same arithmetic, order and tiling), whatever else is
 * being served.  A server and its requests belong to one host thread at a time.
 *   o3g_server_submit copies the host clouds (packed xyz; h_tgt_nrm may be NULL
 *   to estimate normals with normal_radius / normal_max_nn) and returns an id;
 *   a request larger than the whole budget gives O3G_ERR_OOM.
 *   o3g_server_step reports active, waiting and completed-this-step counts.
 *   o3g_server_poll sets *out_done; when done it fills the results (as
 *   o3g_icp_point_to_plane_grid; out_status holds the request's status) and
 *   forgets the request.
 *   o3g_server_completed lists (up to cap, ascending) the ids of finished
 *   requests that have not been polled yet.
 */
typedef struct o3g_server o3g_server;
O3G_API int32_t o3g_server_create(int32_t max_active, int64_t hbm_budget_bytes, void* stream, o3g_server** out);
/* The device-memory estimate a request of ns source and nt target points is
 * admitted against (bytes; ns, nt >= 0, else -1).  No device work. */
O3G_API int64_t o3g_server_request_bytes(int64_t ns, int64_t nt);
O3G_API int32_t o3g_server_destroy(o3g_server* server);
O3G_API int32_t o3g_server_submit(o3g_server* server, const float* h_src, int64_t ns, const float* h_tgt, int64_t nt,
                                  const float* h_tgt_nrm, float normal_radius, int32_t normal_max_nn,
                                  const double* init_T, double max_corr_dist, int32_t max_iter, double eps,
                                  int64_t* out_id);
O3G_API int32_t o3g_server_step(o3g_server* server, int32_t* out_active, int32_t* out_waiting,
                                int32_t* out_completed);
O3G_API int32_t o3g_server_poll(o3g_server* server, int64_t id, int32_t* out_done, double* out_T,
                                double* out_fitness, double* out_rmse, int32_t* out_iters, int32_t* out_status);
O3G_API int32_t o3g_server_completed(o3g_server* server, int64_t* ids, int32_t cap, int32_t* out_n);

/*
 * Allocation-free form of o3g_icp_point_to_plane_grid.  The paper has no
 * counterpart: this entry point exists for callers that must not allocate device
 * memory once they are running - for example a tracking loop that registers
 * every incoming frame under a fixed memory budget and cannot afford allocator
 * latency or failure mid-run, or a host program that hands all device memory to
 * its own allocator.  Such a caller builds the target grid (o3g_build_grid,
 * which allocates) during set-up and then calls this in its loop.
 *
 * Same arguments, results and status codes as o3g_icp_point_to_plane_grid, with
 * two differences: the source is processed in the caller's order (the sums of
 * J^T J and J^T r therefore round differently, within the usual tolerances),
 * and all working memory is one library-owned static device array of
 * 4,203,520 bytes (4.0 MiB) that every GPU loading the library holds until the
 * process exits.
 *   - ns > O3G_NOALLOC_MAX_POINTS gives O3G_ERR_ARG; nothing is allocated.
 *   - The first call on a device looks up that array's device address for the
 *     current device (cudaGetSymbolAddress); make that first call before any
 *     stream capture.
 *   - Every call uses the same array.  Calls whose work overlaps on the GPU
 *     (other streams, other host threads) race and corrupt each other's state:
 *     serialise them.  Each call clears what must start at zero.
 *   - Like the other ICP entry points it returns host values, so it
 *     synchronises `stream` before returning and cannot be captured in a
 *     CUDA graph.
 *   - It is slower per iteration: in the caller's order a block's queries are
 *     not spatially coherent and no previous matches are kept, so most
 *     searches run from global memory without a first bound (on a
 *     94,829-point RGB-D frame pair, GB300: 69.9 us per iteration against
 *     31.2 us for o3g_icp_point_to_plane_grid).
 */
#define O3G_NOALLOC_MAX_POINTS 262144
O3G_API int32_t o3g_icp_point_to_plane_grid_noalloc(const o3g_grid* tgt, const float* d_src, int64_t ns,
                                                    int32_t stride, const double* init_T, double max_corr_dist,
                                                    int32_t max_iter, double eps, double* out_T, double* out_fitness,
                                                    double* out_rmse, int32_t* out_iters, void* stream);

/*
 * Instrumentation (no counterpart in the paper; used by benchmarks and tests).
 * o3g_launch_count: kernels this library has launched since it was loaded.
 * o3g_timing_enable(1): from then on, each launch of the kernels listed below
 * is bracketed by CUDA events recorded on its launching stream.
 * o3g_timing_read(kind, ...): waits for the recorded events, returns the summed
 * device time in milliseconds and the number of launches timed, and (reset != 0)
 * forgets them.  kind: O3G_KERNEL_ICP_CORR (per-iteration correspondence +
 * reduction), O3G_KERNEL_ICP_SOLVE (per-iteration reduce + solve + update),
 * O3G_KERNEL_NORMALS (normal estimation), O3G_KERNEL_GRID (one whole grid build),
 * O3G_KERNEL_ICP_BATCH (all iteration launches of one batched call, one record),
 * O3G_KERNEL_VOXEL (one whole voxel downsampling call), O3G_KERNEL_EVAL (the
 * launches of one o3g_evaluate_poses call, one record).
 */
#define O3G_KERNEL_ICP_CORR 0
#define O3G_KERNEL_ICP_SOLVE 1
#define O3G_KERNEL_NORMALS 2
#define O3G_KERNEL_GRID 3
#define O3G_KERNEL_ICP_BATCH 4
#define O3G_KERNEL_VOXEL 5
#define O3G_KERNEL_EVAL 6
O3G_API int64_t o3g_launch_count(void);
O3G_API int32_t o3g_timing_enable(int32_t on);
O3G_API int32_t o3g_timing_read(int32_t kind, double* total_ms, int64_t* launches, int32_t reset);

#ifdef __cplusplus
}
#endif

#endif /* O3G_H */
