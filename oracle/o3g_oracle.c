/*
 * o3g oracle: plain, slow, obviously-correct CPU statement of the point-to-plane
 * ICP iteration and of the hybrid-kNN PCA normal estimation of Open3D
 * (arXiv 1801.09847).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or constant with the CUDA
 * library.
 *
 * Build:  gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fPIC -shared -pthread
 * (-ffp-contract=off matters: every FP32 expression below is meant as a chain of
 * separately rounded IEEE operations, and gcc on aarch64 would otherwise fuse
 * a*b+c into one FMA.)
 *
 * Passages followed (Open3D paper):
 *   Sec. 3.1           point clouds carry points and normals; normals are valid only
 *                      when they have as many records as the points.
 *   Sec. 3.3, Fig. 1   estimate_normals with KDTreeSearchParamHybrid(radius, max_nn)
 *                      and registration_icp(source, target,
 *                      max_correspondence_distance, init,
 *                      TransformationEstimationPointToPlane()).
 *   Sec. 4, Eq. (1)    objective L(x) = sum_i r_i(x)^2.
 *   Sec. 4, Eq. (2)    Gauss-Newton step x+ = x - (J^T J)^-1 J^T r, J and r at x^k;
 *                      the expensive part is the sum of J^T J and J^T r over records.
 *
 * Readings where the paper is silent (the residual and Jacobian of
 * point-to-plane ICP are not printed; it cites them):
 *   residual   r_i = (p_i - q_c(i)) . n_c(i),  p_i = R s_i + t  (target normal)
 *   Jacobian   left perturbation p -> p + w x p + v, so dr/d(w,v) = [p x n ; n]
 *   step       xi = (w, v) = -(A)^-1 b,  A = sum J J^T,  b = sum J r     (Eq. 2)
 *   update     dR = Rz(gamma) Ry(beta) Rx(alpha), (alpha,beta,gamma) = w;
 *              T <- [dR v; 0 1] * T
 *   NN         argmin over target j of (d2, j), d2 <= fl(r_max)*fl(r_max), where
 *              d2 = (dx*dx + dy*dy) + dz*dz in FP32, dx = p_x - q_x; the lowest
 *              target index wins a tie.
 *   transform  p = ((R00 sx + R01 sy) + R02 sz) + tx per row, FP32, R and t
 *              rounded to nearest from the FP64 pose.
 *   solve      LDL^T, no pivoting, pivot order 0..5; a pivot D_kk <= 1e-12 *
 *              max_j A_jj freezes that unknown (xi_k = 0, column k of L zeroed).
 *   stop       fewer than 6 correspondences, or max(|w|,|v|) < eps after an
 *              update, or max_iter updates done.
 *   result     fitness = |C| / N_s, rmse = sqrt(sum_C d2 / |C|) at the final pose.
 *   normals    the <= max_nn nearest points within radius (the point itself
 *              included; (d2, index) order), FP64 centred covariance divided by m,
 *              unit eigenvector of its smallest eigenvalue (cyclic Jacobi), turned
 *              so that n . (viewpoint - q) >= 0; fewer than 3 neighbours -> (0,0,1).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_OK 0
#define ORA_WARN_DEGENERATE 1
#define ORA_WARN_FEW_CORR 2
#define ORA_ERR_ARG (-1)
#define ORA_ERR_OOM (-2)

typedef struct ora_grid ora_grid;

/* ------------------------------------------------------------------ threads */

typedef void (*range_fn)(void* ctx, int64_t lo, int64_t hi);

typedef struct {
  range_fn fn;
  void* ctx;
  int64_t lo, hi;
} range_job;

static void* range_thread(void* arg) {
  range_job* j = (range_job*)arg;
  j->fn(j->ctx, j->lo, j->hi);
  return NULL;
}

/* Runs fn over [0, n) split into nthreads contiguous chunks.  The work items
 * are independent, so the result does not depend on the thread count. */
static void parallel_for(int64_t n, int nthreads, range_fn fn, void* ctx) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (n < 2 * nthreads) nthreads = 1;
  if (nthreads == 1) {
    fn(ctx, 0, n);
    return;
  }
  pthread_t th[256];
  range_job jobs[256];
  int started[256];
  for (int k = 0; k < nthreads; ++k) {
    jobs[k].fn = fn;
    jobs[k].ctx = ctx;
    jobs[k].lo = n * k / nthreads;
    jobs[k].hi = n * (k + 1) / nthreads;
    started[k] = pthread_create(&th[k], NULL, range_thread, &jobs[k]) == 0;
    if (!started[k]) fn(ctx, jobs[k].lo, jobs[k].hi);
  }
  for (int k = 0; k < nthreads; ++k)
    if (started[k]) pthread_join(th[k], NULL);
}

/* -------------------------------------------------------- a3: the transform */

void ora_pose_to_f32(const double T[16], float R[9], float t[3]) {
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) R[3 * r + c] = (float)T[4 * r + c];
    t[r] = (float)T[4 * r + 3];
  }
}

static void transform_one(const float R[9], const float t[3], const float s[3], float p[3]) {
  for (int r = 0; r < 3; ++r) {
    float acc = R[3 * r + 0] * s[0];
    acc = acc + R[3 * r + 1] * s[1];
    acc = acc + R[3 * r + 2] * s[2];
    p[r] = acc + t[r];
  }
}

/* p_i = R s_i + t in FP32 for every source point (xyz packed, 3 floats each). */
void ora_transform(const float* src, int64_t n, const double T[16], float* out) {
  float R[9], t[3];
  ora_pose_to_f32(T, R, t);
  for (int64_t i = 0; i < n; ++i) transform_one(R, t, src + 3 * i, out + 3 * i);
}

/* ----------------------------------------------- a4: brute-force fixed-radius NN */

static float dist2_f32(const float* a, const float* b) {
  float dx = a[0] - b[0];
  float dy = a[1] - b[1];
  float dz = a[2] - b[2];
  return (dx * dx + dy * dy) + dz * dz;
}

typedef struct {
  const float* p;
  const float* tgt;
  int64_t nt;
  float r2;
  int32_t* corr;
  float* d2;
} nn_ctx;

static void nn_range(void* vctx, int64_t lo, int64_t hi) {
  nn_ctx* c = (nn_ctx*)vctx;
  for (int64_t i = lo; i < hi; ++i) {
    int64_t best = -1;
    float best_d2 = 0.0f;
    for (int64_t j = 0; j < c->nt; ++j) {
      float d2 = dist2_f32(c->p + 3 * i, c->tgt + 3 * j);
      if (!(d2 <= c->r2)) continue;
      if (best < 0 || d2 < best_d2) { /* ascending j: ties keep the lowest index */
        best = j;
        best_d2 = d2;
      }
    }
    c->corr[i] = (int32_t)best;
    c->d2[i] = best < 0 ? 0.0f : best_d2;
  }
}

/* For every (already transformed) point p_i: the target index j minimising
 * (d2(p_i, q_j), j) among d2 <= fl(r_max)^2, or -1.  d2 of the match (0 if none). */
int ora_nn(const float* p, int64_t ns, const float* tgt, int64_t nt, float r_max, int32_t nthreads,
           int32_t* corr, float* d2) {
  if (ns < 0 || nt < 0 || nt > INT32_MAX || !(r_max >= 0.0f)) return ORA_ERR_ARG;
  nn_ctx c = {p, tgt, nt, r_max * r_max, corr, d2};
  parallel_for(ns, nthreads, nn_range, &c);
  return ORA_OK;
}

/* ------------------------------------- a4 at scale: exact grid-accelerated NN */

/* The same map as ora_nn, bit for bit, for clouds too large to scan in full.
 * Targets are bucketed in a uniform grid of cell h = 1.01 r_max, cell index
 * floor(x / h) per axis.  Why no match can be missed: a target with FP32
 * d2 <= fl(r_max)^2 differs from p by at most (1 + 1e-6) r_max in each
 * coordinate (the FP32 distance formula loses a few ulps at most), which is
 * below h, so its cell index differs from p's by at most 1 on every axis and it
 * lies in one of the 27 cells around p's cell.  The candidates of those cells
 * are compared by (d2, j) explicitly, so the order of the scan does not matter.
 * Targets with a non-finite coordinate never match in ora_nn (their d2 is not
 * <= r2) and are left out.  This is an acceleration of ora_nn, not a separate
 * definition: the pins compare the two on every input class. */

typedef struct {
  int64_t c[3];
  int32_t j;
} gcell;

struct ora_grid {
  const float* tgt;
  double inv_h;
  float r2;
  int64_t n;   /* bucketed (finite) targets */
  gcell* cells; /* sorted by (c[0], c[1], c[2], j) */
};

static int gcell_cmp(const void* a, const void* b) {
  const gcell* x = (const gcell*)a;
  const gcell* y = (const gcell*)b;
  for (int k = 0; k < 3; ++k) {
    if (x->c[k] < y->c[k]) return -1;
    if (x->c[k] > y->c[k]) return 1;
  }
  return (x->j > y->j) - (x->j < y->j);
}

/* floor(x / h) as an integer; clamping to +-2^62 is monotone and never moves two
 * indices further apart, so the 27-cell argument still holds. */
static int64_t cell_index(float x, double inv_h) {
  double v = floor((double)x * inv_h);
  if (v > 4611686018427387904.0) v = 4611686018427387904.0;
  if (v < -4611686018427387904.0) v = -4611686018427387904.0;
  return (int64_t)v;
}

static int finite3(const float* x) { return isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2]); }

ora_grid* ora_grid_build(const float* tgt, int64_t nt, float r_max) {
  if (nt < 0 || nt > INT32_MAX || !(r_max > 0.0f) || !isfinite(r_max)) return NULL;
  ora_grid* g = (ora_grid*)calloc(1, sizeof(ora_grid));
  if (!g) return NULL;
  g->tgt = tgt;
  g->inv_h = 1.0 / (1.01 * (double)r_max);
  g->r2 = r_max * r_max;
  g->cells = (gcell*)malloc(sizeof(gcell) * (size_t)(nt > 0 ? nt : 1));
  if (!g->cells) {
    free(g);
    return NULL;
  }
  int64_t m = 0;
  for (int64_t j = 0; j < nt; ++j) {
    const float* q = tgt + 3 * j;
    if (!finite3(q)) continue;
    for (int k = 0; k < 3; ++k) g->cells[m].c[k] = cell_index(q[k], g->inv_h);
    g->cells[m].j = (int32_t)j;
    ++m;
  }
  g->n = m;
  qsort(g->cells, (size_t)m, sizeof(gcell), gcell_cmp);
  return g;
}

void ora_grid_free(ora_grid* g) {
  if (!g) return;
  free(g->cells);
  free(g);
}

/* First bucketed target whose cell is >= c (binary search). */
static int64_t cell_lower_bound(const ora_grid* g, const int64_t c[3]) {
  int64_t lo = 0, hi = g->n;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    const int64_t* m = g->cells[mid].c;
    int less = m[0] < c[0] || (m[0] == c[0] && (m[1] < c[1] || (m[1] == c[1] && m[2] < c[2])));
    if (less) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

typedef struct {
  const ora_grid* g;
  const float* p;
  int32_t* corr;
  float* d2;
} gnn_ctx;

static void gnn_range(void* vctx, int64_t lo, int64_t hi) {
  gnn_ctx* c = (gnn_ctx*)vctx;
  const ora_grid* g = c->g;
  for (int64_t i = lo; i < hi; ++i) {
    const float* p = c->p + 3 * i;
    int64_t best = -1;
    float best_d2 = 0.0f;
    if (finite3(p)) {
      int64_t pc[3];
      for (int k = 0; k < 3; ++k) pc[k] = cell_index(p[k], g->inv_h);
      for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dz = -1; dz <= 1; ++dz) {
            int64_t nc[3] = {pc[0] + dx, pc[1] + dy, pc[2] + dz};
            for (int64_t e = cell_lower_bound(g, nc); e < g->n; ++e) {
              const gcell* q = &g->cells[e];
              if (q->c[0] != nc[0] || q->c[1] != nc[1] || q->c[2] != nc[2]) break;
              float d2 = dist2_f32(p, g->tgt + 3 * (int64_t)q->j);
              if (!(d2 <= g->r2)) continue;
              if (best < 0 || d2 < best_d2 || (d2 == best_d2 && q->j < best)) {
                best = q->j;
                best_d2 = d2;
              }
            }
          }
    }
    c->corr[i] = (int32_t)best;
    c->d2[i] = best < 0 ? 0.0f : best_d2;
  }
}

/* ora_nn against a grid built over the target with the same r_max. */
int ora_grid_nn(const ora_grid* g, const float* p, int64_t ns, int32_t nthreads, int32_t* corr, float* d2) {
  if (!g || ns < 0) return ORA_ERR_ARG;
  gnn_ctx c = {g, p, corr, d2};
  parallel_for(ns, nthreads, gnn_range, &c);
  return ORA_OK;
}

/* --------------------------------------- a5: residual, Jacobian, normal equations */

/* J = [p x n ; n] and r = (p - q) . n, both in FP64 from the FP32 inputs. */
void ora_residual_jacobian(const float p[3], const float q[3], const float n[3], double J[6], double* r) {
  double px = p[0], py = p[1], pz = p[2];
  double nx = n[0], ny = n[1], nz = n[2];
  double dx = px - (double)q[0], dy = py - (double)q[1], dz = pz - (double)q[2];
  *r = dx * nx + dy * ny + dz * nz;
  J[0] = py * nz - pz * ny;
  J[1] = pz * nx - px * nz;
  J[2] = px * ny - py * nx;
  J[3] = nx;
  J[4] = ny;
  J[5] = nz;
}

/* A = sum_i J_i J_i^T (6x6, row-major, full), b = sum_i J_i r_i, plus sum r^2,
 * sum d2 and |C|, summed over i in increasing order. */
void ora_normal_equations(const float* p, int64_t ns, const float* tgt, const float* nrm, const int32_t* corr,
                          const float* d2, double A[36], double b[6], double* sum_r2, double* sum_d2,
                          int64_t* count) {
  memset(A, 0, 36 * sizeof(double));
  memset(b, 0, 6 * sizeof(double));
  *sum_r2 = 0.0;
  *sum_d2 = 0.0;
  *count = 0;
  for (int64_t i = 0; i < ns; ++i) {
    int32_t j = corr[i];
    if (j < 0) continue;
    double J[6], r;
    ora_residual_jacobian(p + 3 * i, tgt + 3 * (int64_t)j, nrm + 3 * (int64_t)j, J, &r);
    for (int a = 0; a < 6; ++a) {
      for (int c = 0; c < 6; ++c) A[6 * a + c] += J[a] * J[c];
      b[a] += J[a] * r;
    }
    *sum_r2 += r * r;
    *sum_d2 += (double)d2[i];
    *count += 1;
  }
}

/* ----------------------------------------------------- a6: solve and update */

/* Solves A xi = -b by LDL^T without pivoting (Eq. 2: xi = -(J^T J)^-1 J^T r).
 * Pivots with D_kk <= 1e-12 * max_j A_jj are frozen: xi_k = 0.  Returns the
 * number of frozen pivots. */
int ora_ldlt_solve(const double A[36], const double b[6], double xi[6]) {
  double L[6][6], D[6], y[6];
  int frozen[6];
  int n_frozen = 0;
  double max_diag = A[0];
  for (int j = 1; j < 6; ++j)
    if (A[7 * j] > max_diag) max_diag = A[7 * j];
  double thr = 1e-12 * max_diag;
  memset(L, 0, sizeof(L));
  for (int k = 0; k < 6; ++k) {
    double s = A[6 * k + k];
    for (int m = 0; m < k; ++m) s -= L[k][m] * L[k][m] * D[m];
    D[k] = s;
    frozen[k] = !(s > thr);
    n_frozen += frozen[k];
    L[k][k] = 1.0;
    for (int i = k + 1; i < 6; ++i) {
      if (frozen[k]) {
        L[i][k] = 0.0;
        continue;
      }
      double v = A[6 * i + k];
      for (int m = 0; m < k; ++m) v -= L[i][m] * L[k][m] * D[m];
      L[i][k] = v / D[k];
    }
  }
  for (int i = 0; i < 6; ++i) { /* L y = -b */
    double v = -b[i];
    for (int m = 0; m < i; ++m) v -= L[i][m] * y[m];
    y[i] = v;
  }
  for (int i = 5; i >= 0; --i) { /* L^T xi = D^-1 y */
    double v = frozen[i] ? 0.0 : y[i] / D[i];
    for (int m = i + 1; m < 6; ++m) v -= L[m][i] * xi[m];
    xi[i] = v;
  }
  return n_frozen;
}

static void mat3_mul(const double a[9], const double b[9], double out[9]) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += a[3 * r + k] * b[3 * k + c];
      out[3 * r + c] = s;
    }
}

void ora_mat4_mul(const double a[16], const double b[16], double out[16]) {
  double tmp[16];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += a[4 * r + k] * b[4 * k + c];
      tmp[4 * r + c] = s;
    }
  memcpy(out, tmp, sizeof(tmp));
}

/* dT(xi) = [Rz(gamma) Ry(beta) Rx(alpha), (tx, ty, tz); 0 0 0 1]. */
void ora_delta_T(const double xi[6], double dT[16]) {
  double ca = cos(xi[0]), sa = sin(xi[0]);
  double cb = cos(xi[1]), sb = sin(xi[1]);
  double cg = cos(xi[2]), sg = sin(xi[2]);
  double Rx[9] = {1, 0, 0, 0, ca, -sa, 0, sa, ca};
  double Ry[9] = {cb, 0, sb, 0, 1, 0, -sb, 0, cb};
  double Rz[9] = {cg, -sg, 0, sg, cg, 0, 0, 0, 1};
  double RyRx[9], R[9];
  mat3_mul(Ry, Rx, RyRx);
  mat3_mul(Rz, RyRx, R);
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) dT[4 * r + c] = R[3 * r + c];
    dT[4 * r + 3] = xi[3 + r];
  }
  dT[12] = dT[13] = dT[14] = 0.0;
  dT[15] = 1.0;
}

/* --------------------------------------------------- the ICP loop, a3..a7 */

/* The ICP loop, steps a3..a7; grid == NULL scans every target (ora_nn). */
static int icp_impl(const float* src, int64_t ns, const float* tgt, int64_t nt, const float* tgt_nrm,
                    const double init_T[16], double max_corr_dist, int32_t max_iter, double eps, int32_t nthreads,
                    const ora_grid* grid, double out_T[16], double* out_fitness, double* out_rmse,
                    int32_t* out_iters) {
  float r_max = (float)max_corr_dist;
  int64_t nalloc = ns > 0 ? ns : 1;
  float* p = (float*)malloc(sizeof(float) * 3 * nalloc);
  int32_t* corr = (int32_t*)malloc(sizeof(int32_t) * nalloc);
  float* d2 = (float*)malloc(sizeof(float) * nalloc);
  if (!p || !corr || !d2) {
    free(p);
    free(corr);
    free(d2);
    return ORA_ERR_OOM;
  }
  double T[16];
  memcpy(T, init_T, sizeof(T));
  int status = ORA_OK, degenerate = 0, iters = 0;
  double A[36], b[6], sum_r2, sum_d2;
  int64_t count;
  for (int k = 0; k < max_iter; ++k) {
    ora_transform(src, ns, T, p);
    if (grid) ora_grid_nn(grid, p, ns, nthreads, corr, d2);
    else ora_nn(p, ns, tgt, nt, r_max, nthreads, corr, d2);
    ora_normal_equations(p, ns, tgt, tgt_nrm, corr, d2, A, b, &sum_r2, &sum_d2, &count);
    if (count < 6) {
      status = ORA_WARN_FEW_CORR;
      break;
    }
    double xi[6], dT[16];
    if (ora_ldlt_solve(A, b, xi) > 0) degenerate = 1;
    ora_delta_T(xi, dT);
    ora_mat4_mul(dT, T, T);
    ++iters;
    double w = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
    double v = sqrt(xi[3] * xi[3] + xi[4] * xi[4] + xi[5] * xi[5]);
    if ((w > v ? w : v) < eps) break;
  }
  /* a7: evaluation at the final pose */
  ora_transform(src, ns, T, p);
  if (grid) ora_grid_nn(grid, p, ns, nthreads, corr, d2);
  else ora_nn(p, ns, tgt, nt, r_max, nthreads, corr, d2);
  ora_normal_equations(p, ns, tgt, tgt_nrm, corr, d2, A, b, &sum_r2, &sum_d2, &count);
  memcpy(out_T, T, sizeof(T));
  *out_fitness = ns > 0 ? (double)count / (double)ns : 0.0;
  *out_rmse = count > 0 ? sqrt(sum_d2 / (double)count) : 0.0;
  *out_iters = iters;
  free(p);
  free(corr);
  free(d2);
  if (status == ORA_OK && degenerate) status = ORA_WARN_DEGENERATE;
  return status;
}

/* Point-to-plane ICP (Sec. 3.3, Eq. 1-2).  Clouds are packed xyz FP32.
 * Returns ORA_OK, ORA_WARN_DEGENERATE (some pivot was frozen),
 * ORA_WARN_FEW_CORR (stopped with < 6 correspondences), or an error. */
int ora_icp_point_to_plane(const float* src, int64_t ns, const float* tgt, int64_t nt, const float* tgt_nrm,
                           const double init_T[16], double max_corr_dist, int32_t max_iter, double eps,
                           int32_t nthreads, double out_T[16], double* out_fitness, double* out_rmse,
                           int32_t* out_iters) {
  if (ns < 0 || nt < 0 || nt > INT32_MAX || max_iter < 0 || !(max_corr_dist >= 0.0)) return ORA_ERR_ARG;
  return icp_impl(src, ns, tgt, nt, tgt_nrm, init_T, max_corr_dist, max_iter, eps, nthreads, NULL, out_T,
                  out_fitness, out_rmse, out_iters);
}

/* The same ICP with the correspondence step answered by the exact grid search
 * (identical correspondences, hence an identical result); for large clouds. */
int ora_icp_point_to_plane_gridnn(const float* src, int64_t ns, const float* tgt, int64_t nt, const float* tgt_nrm,
                                  const double init_T[16], double max_corr_dist, int32_t max_iter, double eps,
                                  int32_t nthreads, double out_T[16], double* out_fitness, double* out_rmse,
                                  int32_t* out_iters) {
  if (ns < 0 || nt < 0 || nt > INT32_MAX || max_iter < 0 || !((float)max_corr_dist > 0.0f) ||
      !isfinite((float)max_corr_dist))
    return ORA_ERR_ARG;
  ora_grid* g = ora_grid_build(tgt, nt, (float)max_corr_dist);
  if (!g) return ORA_ERR_OOM;
  int st = icp_impl(src, ns, tgt, nt, tgt_nrm, init_T, max_corr_dist, max_iter, eps, nthreads, g, out_T,
                    out_fitness, out_rmse, out_iters);
  ora_grid_free(g);
  return st;
}

/* ------------------------------------------------ a2: hybrid kNN and normals */

typedef struct {
  float d2;
  int32_t j;
} cand;

static int cand_cmp(const void* a, const void* b) {
  const cand* x = (const cand*)a;
  const cand* y = (const cand*)b;
  if (x->d2 < y->d2) return -1;
  if (x->d2 > y->d2) return 1;
  return (x->j > y->j) - (x->j < y->j);
}

typedef struct {
  const float* pts;
  int64_t n;
  const float* qry;
  float r2;
  int32_t max_nn;
  int32_t* idx;
  float* dd;
  int32_t* cnt;
  int failed;
} knn_ctx;

static void knn_range(void* vctx, int64_t lo, int64_t hi) {
  knn_ctx* c = (knn_ctx*)vctx;
  cand* buf = (cand*)malloc(sizeof(cand) * (c->n > 0 ? c->n : 1));
  if (!buf) {
    c->failed = 1;
    return;
  }
  for (int64_t i = lo; i < hi; ++i) {
    int64_t m = 0;
    for (int64_t j = 0; j < c->n; ++j) {
      float d2 = dist2_f32(c->qry + 3 * i, c->pts + 3 * j);
      if (d2 <= c->r2) {
        buf[m].d2 = d2;
        buf[m].j = (int32_t)j;
        ++m;
      }
    }
    qsort(buf, (size_t)m, sizeof(cand), cand_cmp);
    int64_t keep = m < c->max_nn ? m : c->max_nn;
    for (int64_t k = 0; k < c->max_nn; ++k) {
      c->idx[i * c->max_nn + k] = k < keep ? buf[k].j : -1;
      c->dd[i * c->max_nn + k] = k < keep ? buf[k].d2 : 0.0f;
    }
    c->cnt[i] = (int32_t)keep;
  }
  free(buf);
}

/* Hybrid search (KDTreeSearchParamHybrid, Fig. 1): for each query, the at most
 * max_nn points with d2 <= fl(radius)^2, in (d2, index) order.  out_idx and out_d2
 * are nq x max_nn, padded with -1 / 0. */
int ora_knn_hybrid(const float* pts, int64_t n, const float* qry, int64_t nq, float radius, int32_t max_nn,
                   int32_t nthreads, int32_t* out_idx, float* out_d2, int32_t* out_cnt) {
  if (n < 0 || nq < 0 || n > INT32_MAX || max_nn < 1 || !(radius >= 0.0f)) return ORA_ERR_ARG;
  knn_ctx c = {pts, n, qry, radius * radius, max_nn, out_idx, out_d2, out_cnt, 0};
  parallel_for(nq, nthreads, knn_range, &c);
  return c.failed ? ORA_ERR_OOM : ORA_OK;
}

/* Eigen-decomposition of a symmetric 3x3 matrix by cyclic Jacobi rotations, in
 * FP64.  Each rotation G in the (p, q) plane is chosen so that (G^T C G)_pq = 0;
 * sweeps repeat until the off-diagonal norm is below 1e-15 of the Frobenius norm.
 * evals[k] pairs with column k of V (row-major). */
void ora_jacobi_eig3(const double C[9], double evals[3], double V[9]) {
  double a[9];
  memcpy(a, C, sizeof(a));
  for (int k = 0; k < 9; ++k) V[k] = (k % 4 == 0) ? 1.0 : 0.0;
  double fro2 = 0.0;
  for (int k = 0; k < 9; ++k) fro2 += a[k] * a[k];
  static const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off2 = 2.0 * (a[1] * a[1] + a[2] * a[2] + a[5] * a[5]);
    if (off2 <= 1e-30 * fro2) break;
    for (int w = 0; w < 3; ++w) {
      int p = pairs[w][0], q = pairs[w][1];
      double apq = a[3 * p + q];
      if (apq == 0.0) continue;
      double theta = (a[3 * q + q] - a[3 * p + p]) / (2.0 * apq);
      double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
      double c = 1.0 / sqrt(t * t + 1.0);
      double s = t * c;
      double G[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
      G[3 * p + p] = c;
      G[3 * q + q] = c;
      G[3 * p + q] = s;
      G[3 * q + p] = -s;
      double Gt[9], tmp[9];
      for (int r = 0; r < 3; ++r)
        for (int cc = 0; cc < 3; ++cc) Gt[3 * r + cc] = G[3 * cc + r];
      mat3_mul(Gt, a, tmp);
      mat3_mul(tmp, G, a);
      a[3 * p + q] = 0.0; /* zero by construction of G */
      a[3 * q + p] = 0.0;
      mat3_mul(V, G, tmp);
      memcpy(V, tmp, sizeof(tmp));
    }
  }
  for (int k = 0; k < 3; ++k) evals[k] = a[4 * k];
}

/* Normal of one neighbourhood: FP64 centred covariance / m, smallest-eigenvalue
 * eigenvector, oriented toward the viewpoint.  Also returns the three
 * eigenvalues in ascending order (used by tests to assess conditioning). */
void ora_normal_from_neighbours(const float* pts, const int32_t* idx, int32_t m, const float q[3],
                                const double viewpoint[3], float out_n[3], double out_evals[3]) {
  if (m < 3) {
    out_n[0] = 0.0f;
    out_n[1] = 0.0f;
    out_n[2] = 1.0f;
    out_evals[0] = out_evals[1] = out_evals[2] = 0.0;
    return;
  }
  double mu[3] = {0, 0, 0};
  for (int32_t k = 0; k < m; ++k)
    for (int a = 0; a < 3; ++a) mu[a] += (double)pts[3 * (int64_t)idx[k] + a];
  for (int a = 0; a < 3; ++a) mu[a] /= (double)m;
  double C[9] = {0};
  for (int32_t k = 0; k < m; ++k) {
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = (double)pts[3 * (int64_t)idx[k] + a] - mu[a];
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) C[3 * a + c] += d[a] * d[c];
  }
  for (int k = 0; k < 9; ++k) C[k] /= (double)m;
  double ev[3], V[9];
  ora_jacobi_eig3(C, ev, V);
  int kmin = 0;
  for (int k = 1; k < 3; ++k)
    if (ev[k] < ev[kmin]) kmin = k;
  double n[3] = {V[kmin], V[3 + kmin], V[6 + kmin]};
  double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  for (int a = 0; a < 3; ++a) n[a] /= len;
  double facing = n[0] * (viewpoint[0] - q[0]) + n[1] * (viewpoint[1] - q[1]) + n[2] * (viewpoint[2] - q[2]);
  if (facing < 0.0)
    for (int a = 0; a < 3; ++a) n[a] = -n[a];
  for (int a = 0; a < 3; ++a) out_n[a] = (float)n[a];
  /* ascending eigenvalues */
  double e0 = ev[0], e1 = ev[1], e2 = ev[2], tmp;
  if (e0 > e1) { tmp = e0; e0 = e1; e1 = tmp; }
  if (e1 > e2) { tmp = e1; e1 = e2; e2 = tmp; }
  if (e0 > e1) { tmp = e0; e0 = e1; e1 = tmp; }
  out_evals[0] = e0;
  out_evals[1] = e1;
  out_evals[2] = e2;
}

/* estimate_normals (Fig. 1, Sec. 3.3) for every point of the cloud.  out_evals
 * (n x 3, ascending) may be NULL. */
int ora_estimate_normals(const float* pts, int64_t n, float radius, int32_t max_nn, const double viewpoint[3],
                         int32_t nthreads, float* out_nrm, double* out_evals) {
  if (n < 0 || n > INT32_MAX || max_nn < 1 || !(radius >= 0.0f)) return ORA_ERR_ARG;
  int64_t nalloc = n > 0 ? n : 1;
  int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * nalloc * max_nn);
  float* dd = (float*)malloc(sizeof(float) * nalloc * max_nn);
  int32_t* cnt = (int32_t*)malloc(sizeof(int32_t) * nalloc);
  if (!idx || !dd || !cnt) {
    free(idx);
    free(dd);
    free(cnt);
    return ORA_ERR_OOM;
  }
  int st = ora_knn_hybrid(pts, n, pts, n, radius, max_nn, nthreads, idx, dd, cnt);
  if (st == ORA_OK) {
    for (int64_t i = 0; i < n; ++i) {
      double ev[3];
      ora_normal_from_neighbours(pts, idx + i * max_nn, cnt[i], pts + 3 * i, viewpoint, out_nrm + 3 * i, ev);
      if (out_evals)
        for (int a = 0; a < 3; ++a) out_evals[3 * i + a] = ev[a];
    }
  }
  free(idx);
  free(dd);
  free(cnt);
  return st;
}

/* ------------------------------------------ point-to-point ICP (Sec. 3.3) */

static void mat4_mul(const double a[16], const double b[16], double out[16]) {
  double tmp[16];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += a[4 * r + k] * b[4 * k + c];
      tmp[4 * r + c] = s;
    }
  memcpy(out, tmp, sizeof(tmp));
}

/* Cyclic Jacobi eigen-decomposition of a symmetric 4x4 in FP64, the scheme of
 * ora_jacobi_eig3: each plane rotation G zeroes (G^T A G)_pq; sweeps repeat
 * until the off-diagonal norm is below 1e-15 of the Frobenius norm.
 * evals[k] pairs with column k of V (row-major). */
void ora_jacobi_eig4(const double C[16], double evals[4], double V[16]) {
  double a[16];
  memcpy(a, C, sizeof(a));
  for (int k = 0; k < 16; ++k) V[k] = (k % 5 == 0) ? 1.0 : 0.0;
  double fro2 = 0.0;
  for (int k = 0; k < 16; ++k) fro2 += a[k] * a[k];
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off2 = 0.0;
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c)
        if (r != c) off2 += a[4 * r + c] * a[4 * r + c];
    if (off2 <= 1e-30 * fro2) break;
    for (int p = 0; p < 3; ++p)
      for (int q = p + 1; q < 4; ++q) {
        double apq = a[4 * p + q];
        if (apq == 0.0) continue;
        double theta = (a[4 * q + q] - a[4 * p + p]) / (2.0 * apq);
        double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0);
        double s = t * c;
        double G[16], Gt[16], tmp[16];
        for (int k = 0; k < 16; ++k) G[k] = (k % 5 == 0) ? 1.0 : 0.0;
        G[4 * p + p] = c;
        G[4 * q + q] = c;
        G[4 * p + q] = s;
        G[4 * q + p] = -s;
        for (int r = 0; r < 4; ++r)
          for (int cc = 0; cc < 4; ++cc) Gt[4 * r + cc] = G[4 * cc + r];
        mat4_mul(Gt, a, tmp);
        mat4_mul(tmp, G, a);
        a[4 * p + q] = 0.0; /* zero by construction of G */
        a[4 * q + p] = 0.0;
        mat4_mul(V, G, tmp);
        memcpy(V, tmp, sizeof(tmp));
      }
  }
  for (int k = 0; k < 4; ++k) evals[k] = a[5 * k];
}

/* The rigid motion (R, t) minimising sum_i |R p_i + t - q_c(i)|^2 over the
 * correspondences (corr[i] >= 0), by Horn's closed form with unit quaternions
 * (J. Opt. Soc. Am. A 4(4), 1987), all in FP64 from the FP32 inputs:
 *   mu_p, mu_q  centroids of the matched source and target points (increasing i);
 *   S_ab        sum_i (p_i - mu_p)_a (q_i - mu_q)_b;
 *   N           the symmetric 4x4 of Horn's paper built from S (trace 0);
 *   (w, x, y, z) the unit eigenvector of N's largest eigenvalue, w >= 0;
 *   R           the rotation of that quaternion;  t = mu_q - R mu_p.
 * When the largest eigenvalue is not separated from the next one by more than
 * 1e-6 E0, E0 = (sum |p - mu_p|^2 + sum |q - mu_q|^2) / 2 (a bound on every
 * eigenvalue's magnitude), the rotation is not determined (for instance all
 * points on one line; float32 coordinates, good to 6e-8 relative, cannot fix a
 * rotation whose eigenvalue gap is smaller); then R = I, t = mu_q - mu_p and
 * the return value is 1.
 * dT = [R t; 0 1].  *angle = 2 atan2(|(x, y, z)|, w), the rotation angle of R.
 * *count = |C|.  Fewer than one correspondence: dT = I, return 0. */
int ora_rigid_align(const float* p, int64_t ns, const float* tgt, const int32_t* corr, double dT[16],
                    double* angle, int64_t* count) {
  double mp[3] = {0, 0, 0}, mq[3] = {0, 0, 0};
  int64_t n = 0;
  for (int64_t i = 0; i < ns; ++i) {
    if (corr[i] < 0) continue;
    const float* q = tgt + 3 * (int64_t)corr[i];
    for (int a = 0; a < 3; ++a) {
      mp[a] += (double)p[3 * i + a];
      mq[a] += (double)q[a];
    }
    ++n;
  }
  *count = n;
  for (int k = 0; k < 16; ++k) dT[k] = (k % 5 == 0) ? 1.0 : 0.0;
  *angle = 0.0;
  if (n < 1) return 0;
  for (int a = 0; a < 3; ++a) {
    mp[a] /= (double)n;
    mq[a] /= (double)n;
  }
  double S[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, gp = 0.0, gq = 0.0;
  for (int64_t i = 0; i < ns; ++i) {
    if (corr[i] < 0) continue;
    const float* q = tgt + 3 * (int64_t)corr[i];
    double dp[3], dq[3];
    for (int a = 0; a < 3; ++a) {
      dp[a] = (double)p[3 * i + a] - mp[a];
      dq[a] = (double)q[a] - mq[a];
    }
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) S[3 * a + b] += dp[a] * dq[b];
    gp += dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2];
    gq += dq[0] * dq[0] + dq[1] * dq[1] + dq[2] * dq[2];
  }
  const double Sxx = S[0], Sxy = S[1], Sxz = S[2], Syx = S[3], Syy = S[4], Syz = S[5], Szx = S[6], Szy = S[7],
               Szz = S[8];
  const double N[16] = {Sxx + Syy + Szz, Syz - Szy,        Szx - Sxz,        Sxy - Syx,
                        Syz - Szy,       Sxx - Syy - Szz,  Sxy + Syx,        Szx + Sxz,
                        Szx - Sxz,       Sxy + Syx,        -Sxx + Syy - Szz, Syz + Szy,
                        Sxy - Syx,       Szx + Sxz,        Syz + Szy,        -Sxx - Syy + Szz};
  double ev[4], V[16];
  ora_jacobi_eig4(N, ev, V);
  int k1 = 0;
  for (int k = 1; k < 4; ++k)
    if (ev[k] > ev[k1]) k1 = k;
  double second = -INFINITY;
  for (int k = 0; k < 4; ++k)
    if (k != k1 && ev[k] > second) second = ev[k];
  const double E0 = 0.5 * (gp + gq);
  int degenerate = !(ev[k1] - second > 1e-6 * E0);
  double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  if (!degenerate) {
    double w = V[k1], x = V[4 + k1], y = V[8 + k1], z = V[12 + k1];
    double len = sqrt(w * w + x * x + y * y + z * z);
    if (w < 0.0) len = -len;
    w /= len;
    x /= len;
    y /= len;
    z /= len;
    R[0] = w * w + x * x - y * y - z * z;
    R[1] = 2.0 * (x * y - w * z);
    R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);
    R[4] = w * w - x * x + y * y - z * z;
    R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);
    R[7] = 2.0 * (y * z + w * x);
    R[8] = w * w - x * x - y * y + z * z;
    *angle = 2.0 * atan2(sqrt(x * x + y * y + z * z), w);
  }
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) dT[4 * r + c] = R[3 * r + c];
    dT[4 * r + 3] = mq[r] - (R[3 * r] * mp[0] + R[3 * r + 1] * mp[1] + R[3 * r + 2] * mp[2]);
  }
  return degenerate;
}

/* Point-to-point ICP (registration_icp with TransformationEstimationPointToPoint,
 * Sec. 3.3): per iteration the FP32 transform and correspondence step of the
 * point-to-plane loop, then dT = ora_rigid_align and T <- dT T.  Stops with
 * ORA_WARN_FEW_CORR when fewer than 3 correspondences remain, after max_iter
 * updates, or when max(angle(dT), |t(dT)|) < eps.  ORA_WARN_DEGENERATE when some
 * update had an undetermined rotation.  use_grid selects the exact grid search. */
int ora_icp_point_to_point(const float* src, int64_t ns, const float* tgt, int64_t nt, const double init_T[16],
                           double max_corr_dist, int32_t max_iter, double eps, int32_t nthreads, int32_t use_grid,
                           double out_T[16], double* out_fitness, double* out_rmse, int32_t* out_iters) {
  if (ns < 0 || nt < 0 || nt > INT32_MAX || max_iter < 0 || !(max_corr_dist >= 0.0)) return ORA_ERR_ARG;
  float r_max = (float)max_corr_dist;
  if (use_grid && !(r_max > 0.0f && isfinite(r_max))) return ORA_ERR_ARG;
  int64_t nalloc = ns > 0 ? ns : 1;
  float* p = (float*)malloc(sizeof(float) * 3 * nalloc);
  int32_t* corr = (int32_t*)malloc(sizeof(int32_t) * nalloc);
  float* d2 = (float*)malloc(sizeof(float) * nalloc);
  ora_grid* g = use_grid ? ora_grid_build(tgt, nt, r_max) : NULL;
  if (!p || !corr || !d2 || (use_grid && !g)) {
    free(p);
    free(corr);
    free(d2);
    ora_grid_free(g);
    return ORA_ERR_OOM;
  }
  double T[16];
  memcpy(T, init_T, sizeof(T));
  int status = ORA_OK, degenerate = 0, iters = 0;
  int64_t count = 0;
  for (int k = 0; k < max_iter; ++k) {
    ora_transform(src, ns, T, p);
    if (g) ora_grid_nn(g, p, ns, nthreads, corr, d2);
    else ora_nn(p, ns, tgt, nt, r_max, nthreads, corr, d2);
    count = 0;
    for (int64_t i = 0; i < ns; ++i) count += corr[i] >= 0;
    if (count < 3) {
      status = ORA_WARN_FEW_CORR;
      break;
    }
    double dT[16], angle;
    if (ora_rigid_align(p, ns, tgt, corr, dT, &angle, &count)) degenerate = 1;
    mat4_mul(dT, T, T);
    ++iters;
    double tn = sqrt(dT[3] * dT[3] + dT[7] * dT[7] + dT[11] * dT[11]);
    if ((angle > tn ? angle : tn) < eps) break;
  }
  /* evaluation at the final pose */
  ora_transform(src, ns, T, p);
  if (g) ora_grid_nn(g, p, ns, nthreads, corr, d2);
  else ora_nn(p, ns, tgt, nt, r_max, nthreads, corr, d2);
  double sum_d2 = 0.0;
  count = 0;
  for (int64_t i = 0; i < ns; ++i)
    if (corr[i] >= 0) {
      sum_d2 += (double)d2[i];
      ++count;
    }
  memcpy(out_T, T, sizeof(T));
  *out_fitness = ns > 0 ? (double)count / (double)ns : 0.0;
  *out_rmse = count > 0 ? sqrt(sum_d2 / (double)count) : 0.0;
  *out_iters = iters;
  free(p);
  free(corr);
  free(d2);
  ora_grid_free(g);
  if (status == ORA_OK && degenerate) status = ORA_WARN_DEGENERATE;
  return status;
}

/* ------------------------------------------------ voxel downsampling (Sec. 3.1) */

typedef struct {
  int64_t k[3];
  int64_t i;
} vkey;

static int vkey_cmp(const void* a, const void* b) {
  const vkey* x = (const vkey*)a;
  const vkey* y = (const vkey*)b;
  for (int d = 0; d < 3; ++d) {
    if (x->k[d] < y->k[d]) return -1;
    if (x->k[d] > y->k[d]) return 1;
  }
  return (x->i > y->i) - (x->i < y->i);
}

/* voxel_down_sample: one output point per occupied voxel, the centroid of the
 * input points in it.
 *   voxel index   (floor(x / v), floor(y / v), floor(z / v)), each quotient a
 *                 single FP32 division; points with a non-finite coordinate are
 *                 dropped; an index outside [-2^30, 2^30] is an error (ORA_ERR_ARG)
 *   order         voxels in increasing (ix, iy, iz), x most significant
 *   centroid      FP64 sum of the voxel's points in increasing input index,
 *                 divided by their count, rounded to FP32
 * out (capacity 3 n floats) receives the centroids, counts (capacity n, may be
 * NULL) the number of points per voxel; *n_out the number of voxels. */
int ora_voxel_downsample(const float* pts, int64_t n, float voxel, float* out, int32_t* counts, int64_t* n_out) {
  *n_out = 0;
  if (n < 0 || !(voxel > 0.0f) || !isfinite(voxel)) return ORA_ERR_ARG;
  vkey* keys = (vkey*)malloc(sizeof(vkey) * (size_t)(n > 0 ? n : 1));
  if (!keys) return ORA_ERR_OOM;
  int64_t m = 0;
  for (int64_t i = 0; i < n; ++i) {
    const float* p = pts + 3 * i;
    if (!finite3(p)) continue;
    for (int d = 0; d < 3; ++d) {
      float q = floorf(p[d] / voxel);
      if (!(q >= -1073741824.0f && q <= 1073741824.0f)) {
        free(keys);
        return ORA_ERR_ARG;
      }
      keys[m].k[d] = (int64_t)q;
    }
    keys[m].i = i;
    ++m;
  }
  qsort(keys, (size_t)m, sizeof(vkey), vkey_cmp);
  int64_t nv = 0;
  for (int64_t a = 0; a < m;) {
    int64_t b = a + 1;
    while (b < m && keys[b].k[0] == keys[a].k[0] && keys[b].k[1] == keys[a].k[1] && keys[b].k[2] == keys[a].k[2]) ++b;
    double s[3] = {0.0, 0.0, 0.0};
    for (int64_t e = a; e < b; ++e)
      for (int d = 0; d < 3; ++d) s[d] += (double)pts[3 * keys[e].i + d];
    for (int d = 0; d < 3; ++d) out[3 * nv + d] = (float)(s[d] / (double)(b - a));
    if (counts) counts[nv] = (int32_t)(b - a);
    ++nv;
    a = b;
  }
  *n_out = nv;
  free(keys);
  return ORA_OK;
}

/* ------------------------------ hypothesis validation (Sec. 3.3, RANSAC) */

/* The validation RANSAC spends its time in (Sec. 3.3 global registration):
 * for each candidate pose T_h (n_poses x 16, row-major FP64), the transform and
 * correspondence step of ICP at T_h over the whole source, then
 *   count_h   = |C_h|
 *   fitness_h = |C_h| / ns
 *   rmse_h    = sqrt(sum_{C_h} d2 / |C_h|)   (0 when C_h is empty)
 * with the FP32 d2 of the matches summed in FP64 in increasing source index.
 * use_grid selects the exact grid search (same correspondences). */
int ora_evaluate_poses(const float* src, int64_t ns, const float* tgt, int64_t nt, const double* poses,
                       int32_t n_poses, double max_corr_dist, int32_t nthreads, int32_t use_grid,
                       double* out_fitness, double* out_rmse, int64_t* out_count) {
  if (ns < 0 || nt < 0 || nt > INT32_MAX || n_poses < 0 || !(max_corr_dist >= 0.0)) return ORA_ERR_ARG;
  float r_max = (float)max_corr_dist;
  if (use_grid && !(r_max > 0.0f && isfinite(r_max))) return ORA_ERR_ARG;
  int64_t nalloc = ns > 0 ? ns : 1;
  float* p = (float*)malloc(sizeof(float) * 3 * nalloc);
  int32_t* corr = (int32_t*)malloc(sizeof(int32_t) * nalloc);
  float* d2 = (float*)malloc(sizeof(float) * nalloc);
  ora_grid* g = use_grid ? ora_grid_build(tgt, nt, r_max) : NULL;
  if (!p || !corr || !d2 || (use_grid && !g)) {
    free(p);
    free(corr);
    free(d2);
    ora_grid_free(g);
    return ORA_ERR_OOM;
  }
  for (int32_t h = 0; h < n_poses; ++h) {
    ora_transform(src, ns, poses + 16 * (int64_t)h, p);
    if (g) ora_grid_nn(g, p, ns, nthreads, corr, d2);
    else ora_nn(p, ns, tgt, nt, r_max, nthreads, corr, d2);
    int64_t count = 0;
    double sum_d2 = 0.0;
    for (int64_t i = 0; i < ns; ++i)
      if (corr[i] >= 0) {
        sum_d2 += (double)d2[i];
        ++count;
      }
    out_count[h] = count;
    out_fitness[h] = ns > 0 ? (double)count / (double)ns : 0.0;
    out_rmse[h] = count > 0 ? sqrt(sum_d2 / (double)count) : 0.0;
  }
  free(p);
  free(corr);
  free(d2);
  ora_grid_free(g);
  return ORA_OK;
}
