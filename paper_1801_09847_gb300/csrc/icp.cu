// Point-to-plane ICP on the GPU: registration_icp(source, target,
// max_correspondence_distance, init, TransformationEstimationPointToPlane())
// of the Open3D paper (Sec. 3.3), as the Gauss-Newton iteration of Sec. 4,
// Eq. (1)-(2).  One kernel launch per iteration, k_icp_iter:
//   1. transform the (cell-sorted) source point, float32, fixed rounding order;
//   2. fixed-radius nearest neighbour over the target grid: the home cell first,
//      then every cell column whose slab can still hold a point at or below the
//      best squared distance so far, over the z-range that bound allows (exact:
//      every pruning bound carries a margin for float32 rounding, and ties are
//      kept, so the result is the minimum of (d2, original index));
//   3. r = (p - q) . n, J = [p x n ; n]; the 21 upper entries of J^T J, J^T r,
//      r^2, d2 and |C| summed per thread with TwoSum compensation, then across
//      the block by a fixed shuffle tree, into one float64 partial per block;
//   4. the last block to finish (atomic arrival counter, no waiting) sums the
//      partials in float64 in block order, solves (J^T J) xi = -J^T r by LDL^T
//      with the frozen-pivot rule, and updates T <- [Rz Ry Rx(xi), t] T on the
//      device.  The next launch reads the new pose.
// The pose never leaves the device between iterations.
#include <cmath>
#include <mutex>

#include "o3g_internal.cuh"

namespace o3g {

namespace {

constexpr int kThreads = 128;
constexpr int kPPT = 1;       // source points per thread
constexpr int kPartial = 32;  // doubles per block partial
constexpr int kNSum = 29;     // 21 (J^T J upper) + 6 (J^T r) + r^2 + d2
constexpr int kGroup = 32;    // block partials summed together by a group's last block

struct Pose {
  double m[16];
};

// Device-resident iteration state.
struct IcpState {
  double T[16];
  float R[9];
  float t[3];
  int iters;
  int done;        // 1: later iterations are skipped
  int degenerate;  // some pivot was frozen
  int few_corr;    // stopped with < 6 correspondences
  int nonfinite;   // the normal equations were not finite
  unsigned arrived;  // groups of the current launch whose sum is stored
  double A[36];
  double b[6];
  double stats[3];  // sum r^2, sum d2, |C|
  double fitness, rmse;
};

enum Mode : int { kIterate = 0, kEquations = 1, kEvaluate = 2, kCorrOnly = 3 };

__global__ void k_init_state(IcpState* st, Pose T) {
  if (threadIdx.x != 0) return;
  for (int k = 0; k < 16; ++k) st->T[k] = T.m[k];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) st->R[3 * r + c] = __double2float_rn(T.m[4 * r + c]);
    st->t[r] = __double2float_rn(T.m[4 * r + 3]);
  }
  st->iters = 0;
  st->done = 0;
  st->degenerate = 0;
  st->few_corr = 0;
  st->nonfinite = 0;
  st->arrived = 0u;
  st->fitness = 0.0;
  st->rmse = 0.0;
}

// Lower bound (with a rounding margin) of |c - x| over the cell slab
// [(lo + i) * cell, (lo + i + 1) * cell) along one axis.
__device__ __forceinline__ float slab_gap(float x, int i_abs, float cell, float margin) {
  const float a = __fmul_rn(static_cast<float>(i_abs), cell);
  const float b = __fmul_rn(static_cast<float>(i_abs + 1), cell);
  const float g = fmaxf(fmaxf(a - x, x - b), 0.f);
  return fmaxf(g - margin, 0.f);
}

// Scans sorted target positions [beg, end) and keeps the minimum of (d2, original index).
__device__ __forceinline__ void scan_run(const float4* __restrict__ pts, uint32_t beg, uint32_t end, float px,
                                         float py, float pz, float& best_d2, int& best_orig, int& best) {
  for (uint32_t k = beg; k < end; ++k) {
    const float4 q = pts[k];
    const float d2 = dist2_rn(px, py, pz, q);
    const int o = __float_as_int(q.w);
    if (d2 < best_d2 || (d2 == best_d2 && o < best_orig)) {
      best_d2 = d2;
      best_orig = o;
      best = static_cast<int>(k);
    }
  }
}

// Fixed-radius nearest neighbour of p among the grid points: the minimum of
// (d2, original index) over d2 <= r2.  Returns the sorted position or -1.
__device__ int nn_search(const GridView& g, float cell, float px, float py, float pz, float r, float r2,
                         float& best_d2) {
  int ax, bx, ay, by, az, bz;
  axis_range(px, r, g.inv_cell, g.lo_x, g.sx, ax, bx);
  axis_range(py, r, g.inv_cell, g.lo_y, g.sy, ay, by);
  axis_range(pz, r, g.inv_cell, g.lo_z, g.sz, az, bz);
  int best = -1, best_orig = 0x7fffffff;
  best_d2 = r2;
  if (ax > bx || ay > by || az > bz) return -1;
  // home cell first: it usually holds a close match, which then prunes the rest
  const int hx = cell_coord(px, g.inv_cell) - g.lo_x;
  const int hy = cell_coord(py, g.inv_cell) - g.lo_y;
  const int hz = cell_coord(pz, g.inv_cell) - g.lo_z;
  const bool home_in = hx >= ax && hx <= bx && hy >= ay && hy <= by && hz >= az && hz <= bz;
  if (home_in) {
    const int c = (hx * g.sy + hy) * g.sz + hz;
    scan_run(g.pts, g.cell_start[c], g.cell_start[c + 1], px, py, pz, best_d2, best_orig, best);
  }
  const float margin = __fadd_rn(__fmul_rn(__fadd_rn(cell, r), 1e-5f),
                                 __fmul_rn(fmaxf(fmaxf(fabsf(px), fabsf(py)), fabsf(pz)), 4e-6f));
  for (int x = ax; x <= bx; ++x) {
    const float gx = slab_gap(px, x + g.lo_x, cell, margin);
    const float gx2 = gx * gx;
    for (int y = ay; y <= by; ++y) {
      const float gy = slab_gap(py, y + g.lo_y, cell, margin);
      const float lim = __fmul_rn(best_d2, 1.0001f) - (gx2 + gy * gy);
      if (lim < 0.f) continue;
      // z-range that can still hold d2 <= best
      const float rz = __fadd_rn(sqrtf(lim), margin);
      const int zl = max(az, cell_coord(__fsub_rn(pz, rz), g.inv_cell) - g.lo_z);
      const int zh = min(bz, cell_coord(__fadd_rn(pz, rz), g.inv_cell) - g.lo_z);
      if (zl > zh) continue;
      const int col = (x * g.sy + y) * g.sz;
      if (home_in && x == hx && y == hy && zl <= hz && hz <= zh) {
        scan_run(g.pts, g.cell_start[col + zl], g.cell_start[col + hz], px, py, pz, best_d2, best_orig, best);
        scan_run(g.pts, g.cell_start[col + hz + 1], g.cell_start[col + zh + 1], px, py, pz, best_d2, best_orig,
                 best);
      } else {
        scan_run(g.pts, g.cell_start[col + zl], g.cell_start[col + zh + 1], px, py, pz, best_d2, best_orig, best);
      }
    }
  }
  return best;
}

// Error-free transformation: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

struct CompSum {
  float s[kNSum];
  float c[kNSum];
  __device__ void zero() {
#pragma unroll
    for (int k = 0; k < kNSum; ++k) s[k] = c[k] = 0.f;
  }
  __device__ __forceinline__ void add(int k, float v) {
    float e;
    two_sum(s[k], v, s[k], e);
    c[k] += e;
  }
};

// Block reduction of the compensated sums (fixed shuffle tree, then warps in
// order) into one float64 partial: [0..28] = sums, [29] = |C|.
__device__ void block_reduce_store(CompSum& acc, int cnt, double* __restrict__ out) {
  __shared__ float ws[kThreads / 32][kNSum];
  __shared__ float wc[kThreads / 32][kNSum];
  __shared__ int wn[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kNSum; ++k) {
    float s = acc.s[k], c = acc.c[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float s2 = __shfl_down_sync(0xffffffffu, s, o);
      float c2 = __shfl_down_sync(0xffffffffu, c, o);
      float e;
      two_sum(s, s2, s, e);
      c = c + c2 + e;
    }
    if (lane == 0) {
      ws[warp][k] = s;
      wc[warp][k] = c;
    }
  }
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  if (lane == 0) wn[warp] = cnt;
  __syncthreads();
  const int t = threadIdx.x;
  if (t < kNSum) {
    float s = ws[0][t], c = wc[0][t];
    for (int w = 1; w < kThreads / 32; ++w) {
      float e;
      two_sum(s, ws[w][t], s, e);
      c = c + wc[w][t] + e;
    }
    out[t] = static_cast<double>(s) + static_cast<double>(c);
  } else if (t == kNSum) {
    int n = 0;
    for (int w = 0; w < kThreads / 32; ++w) n += wn[w];
    out[t] = static_cast<double>(n);
  } else if (t < kPartial) {
    out[t] = 0.0;
  }
}

// sin and cos of a small angle by their Taylor series (|x| <= 0.25: the first
// omitted terms, x^15/15! and x^14/14!, are below 1e-19), else the library call.
__device__ __forceinline__ void sincos_step(double x, double* s, double* c) {
  if (fabs(x) > 0.25) {
    sincos(x, s, c);
    return;
  }
  const double x2 = x * x;
  // sin x = x + x^3 (-1/3! + x^2/5! - x^4/7! + x^6/9! - x^8/11! + x^10/13!), Horner in x^2
  double ps = 1.0 / 6227020800.0;         // 1/13!
  ps = ps * x2 - 1.0 / 39916800.0;        // -1/11!
  ps = ps * x2 + 1.0 / 362880.0;          // 1/9!
  ps = ps * x2 - 1.0 / 5040.0;            // -1/7!
  ps = ps * x2 + 1.0 / 120.0;             // 1/5!
  ps = ps * x2 - 1.0 / 6.0;               // -1/3!
  *s = x + x * x2 * ps;
  // cos x = 1 - x^2 (1/2! - x^2/4! + x^4/6! - x^6/8! + x^8/10! - x^10/12! + x^12/14!)
  double pc = 1.0 / 87178291200.0;        // 1/14!
  pc = pc * x2 - 1.0 / 479001600.0;       // -1/12!
  pc = pc * x2 + 1.0 / 3628800.0;         // 1/10!
  pc = pc * x2 - 1.0 / 40320.0;           // -1/8!
  pc = pc * x2 + 1.0 / 720.0;             // 1/6!
  pc = pc * x2 - 1.0 / 24.0;              // -1/4!
  pc = pc * x2 + 0.5;                     // 1/2!
  *c = 1.0 - x2 * pc;
}

// Float64 sums of `count` partials of kPartial doubles each (rows `first`,
// `first + 1`, ...), in row order: 128 threads = 32 columns x 4 interleaved
// row subsets, combined in subset order.  Result in out[0..kPartial).
__device__ void sum_partials(const double* __restrict__ rows, int first, int count, double* out) {
  __shared__ double sub[4][kPartial];
  const int col = threadIdx.x & 31, q = threadIdx.x >> 5;
  double acc = 0.0;
  for (int b = q; b < count; b += 4) acc += __ldcg(rows + static_cast<size_t>(first + b) * kPartial + col);
  sub[q][col] = acc;
  __syncthreads();
  if (threadIdx.x < kPartial) out[col] = ((sub[0][col] + sub[1][col]) + sub[2][col]) + sub[3][col];
  __syncthreads();
}

// The Gauss-Newton update on one warp, all in float64: LDL^T of the 6x6
// (right-looking, no pivoting; a pivot <= 1e-12 * max_j A_jj freezes its
// unknown: xi_k = 0 and no elimination through it), xi = -(A)^-1 b by forward
// and back substitution, dR = Rz(gamma) Ry(beta) Rx(alpha), T <- [dR, t] T.
__device__ void solve_update(const double* sums, IcpState* __restrict__ st, double eps) {
  __shared__ double M[6][6];
  __shared__ double inv[6], xi[6], sn[3], cs[3], dR[9], Tn[12];
  __shared__ int frozen_any;
  const int lane = threadIdx.x;  // called by warp 0 only
  // unpack the upper triangle (row-major order of the 21 sums)
  if (lane < 21) {
    int a = 0, k = lane;
    while (k >= 6 - a) {
      k -= 6 - a;
      ++a;
    }
    const int c = a + k;
    M[a][c] = sums[lane];
    M[c][a] = sums[lane];
  }
  if (lane == 0) frozen_any = 0;
  __syncwarp();
  double mx = M[0][0];
  for (int j = 1; j < 6; ++j) mx = fmax(mx, M[j][j]);
  const double thr = 1e-12 * mx;
  for (int k = 0; k < 6; ++k) {
    const double d = M[k][k];
    const bool fz = !(d > thr);
    if (lane == 0) {
      inv[k] = fz ? 0.0 : 1.0 / d;
      if (fz) frozen_any = 1;
    }
    __syncwarp();
    const double ik = inv[k];
    // column k of L, then the trailing update, lanes over the lower triangle of rows/cols > k
    if (lane > k && lane < 6) M[lane][k] = M[lane][k] * ik;
    __syncwarp();
    const int m = 5 - k;  // trailing size
    if (!fz && lane < m * m) {
      const int i = k + 1 + lane / m, j = k + 1 + lane % m;
      if (j <= i) M[i][j] -= M[i][k] * d * M[j][k];
    }
    __syncwarp();
  }
  if (lane == 0) {
    double y[6];
    for (int i = 0; i < 6; ++i) {
      double v = -sums[21 + i];
      for (int m = 0; m < i; ++m) v -= M[i][m] * y[m];
      y[i] = v;
    }
    for (int i = 5; i >= 0; --i) {
      double v = y[i] * inv[i];
      for (int m = i + 1; m < 6; ++m) v -= M[m][i] * xi[m];
      xi[i] = v;
    }
  }
  __syncwarp();
  if (lane < 3) sincos_step(xi[lane], &sn[lane], &cs[lane]);
  __syncwarp();
  if (lane < 9) {
    const double sa = sn[0], ca = cs[0], sb = sn[1], cb = cs[1], sg = sn[2], cg = cs[2];
    double v;
    switch (lane) {
      case 0: v = cg * cb; break;
      case 1: v = cg * sb * sa - sg * ca; break;
      case 2: v = cg * sb * ca + sg * sa; break;
      case 3: v = sg * cb; break;
      case 4: v = sg * sb * sa + cg * ca; break;
      case 5: v = sg * sb * ca - cg * sa; break;
      case 6: v = -sb; break;
      case 7: v = cb * sa; break;
      default: v = cb * ca; break;
    }
    dR[lane] = v;
  }
  __syncwarp();
  if (lane < 12) {
    const int r = lane / 4, c = lane % 4;
    double v = dR[3 * r + 0] * st->T[c] + dR[3 * r + 1] * st->T[4 + c] + dR[3 * r + 2] * st->T[8 + c];
    if (c == 3) v += xi[3 + r];
    Tn[lane] = v;
  }
  __syncwarp();
  if (lane < 12) {
    st->T[lane] = Tn[lane];
    const int r = lane / 4, c = lane % 4;
    if (c < 3) st->R[3 * r + c] = __double2float_rn(Tn[lane]);
    else st->t[r] = __double2float_rn(Tn[lane]);
  }
  if (lane == 0) {
    if (frozen_any) st->degenerate = 1;
    st->iters += 1;
    const double w2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
    const double v2 = xi[3] * xi[3] + xi[4] * xi[4] + xi[5] * xi[5];
    if (eps > 0.0 && fmax(w2, v2) < eps * eps) st->done = 1;
  }
}

// Run by the last block of a launch once every group sum is stored: the float64
// total in group order, then per mode the update, the stored normal equations,
// or fitness / rmse.
__device__ void finish(const double* __restrict__ gsums, int ngroups, IcpState* __restrict__ st, double eps,
                       int mode, int ns) {
  __shared__ double sums[kPartial];
  sum_partials(gsums, 0, ngroups, sums);
  if (threadIdx.x == 0) st->arrived = 0u;  // ready for the next launch
  const double count = sums[29];
  if (mode == kEvaluate) {
    if (threadIdx.x == 0) {
      st->fitness = ns > 0 ? count / static_cast<double>(ns) : 0.0;
      st->rmse = count > 0.0 ? sqrt(sums[28] / count) : 0.0;
    }
    return;
  }
  if (threadIdx.x == 0) {
    bool finite = true;
    for (int k = 0; k < 27; ++k) finite = finite && isfinite(sums[k]);
    int k = 0;
    for (int a = 0; a < 6; ++a)
      for (int c = a; c < 6; ++c) {
        st->A[6 * a + c] = sums[k];
        st->A[6 * c + a] = sums[k];
        ++k;
      }
    for (int a = 0; a < 6; ++a) st->b[a] = sums[21 + a];
    st->stats[0] = sums[27];
    st->stats[1] = sums[28];
    st->stats[2] = count;
    if (mode == kIterate) {
      if (!finite) {
        st->nonfinite = 1;
        st->done = 1;
      } else if (count < 6.0) {
        st->few_corr = 1;
        st->done = 1;
      }
    }
  }
  if (mode != kIterate) return;
  __syncthreads();
  if (st->done || threadIdx.x >= 32) return;
  solve_update(sums, st, eps);
}

// One ICP step over the cell-sorted source src4 (x, y, z, original index).
// mode kIterate: skipped once st->done is set; otherwise the other modes run
// regardless.  kCorrOnly writes corr/d2 (by original source index) and no sums.
__global__ void __launch_bounds__(kThreads) k_icp_iter(GridView g, float cell, const float4* __restrict__ src4,
                                                       int ns, IcpState* __restrict__ st, float r,
                                                       double* __restrict__ partials, double* __restrict__ gsums,
                                                       unsigned* __restrict__ group_cnt, double eps, int mode,
                                                       int32_t* __restrict__ corr_out, float* __restrict__ d2_out) {
  if (mode == kIterate && st->done) return;
  float R[9], t[3];
#pragma unroll
  for (int k = 0; k < 9; ++k) R[k] = st->R[k];
#pragma unroll
  for (int k = 0; k < 3; ++k) t[k] = st->t[k];
  const float r2 = __fmul_rn(r, r);
  CompSum acc;
  acc.zero();
  int cnt = 0;
  const int base = blockIdx.x * kThreads * kPPT + threadIdx.x;
#pragma unroll
  for (int j = 0; j < kPPT; ++j) {
    const int i = base + j * kThreads;
    if (i >= ns) break;
    const float4 s = src4[i];
    const float3 p = xform_rn(R, t, s.x, s.y, s.z);
    float bd2;
    const int bp = nn_search(g, cell, p.x, p.y, p.z, r, r2, bd2);
    if (mode == kCorrOnly) {
      const int o = __float_as_int(s.w);
      corr_out[o] = bp >= 0 ? __float_as_int(g.pts[bp].w) : -1;
      d2_out[o] = bp >= 0 ? bd2 : 0.f;
      continue;
    }
    if (bp >= 0) {
      const float4 q = g.pts[bp];
      const float4 n = g.nrm[bp];
      const float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
      const float res = dx * n.x + dy * n.y + dz * n.z;
      float J[6];
      J[0] = p.y * n.z - p.z * n.y;
      J[1] = p.z * n.x - p.x * n.z;
      J[2] = p.x * n.y - p.y * n.x;
      J[3] = n.x;
      J[4] = n.y;
      J[5] = n.z;
      int k = 0;
#pragma unroll
      for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int b = a; b < 6; ++b) acc.add(k++, J[a] * J[b]);
#pragma unroll
      for (int a = 0; a < 6; ++a) acc.add(21 + a, J[a] * res);
      acc.add(27, res * res);
      acc.add(28, bd2);
      ++cnt;
    }
  }
  if (mode == kCorrOnly) return;
  block_reduce_store(acc, cnt, partials + static_cast<size_t>(blockIdx.x) * kPartial);
  // The last block of each group of kGroup blocks sums the group (float64, block
  // order); the last group to finish sums the groups and finishes the launch.
  __shared__ bool last;
  const int grp = blockIdx.x / kGroup;
  const int ngroups = (gridDim.x + kGroup - 1) / kGroup;
  const int in_group = min(kGroup, static_cast<int>(gridDim.x) - grp * kGroup);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&group_cnt[grp], 1u) == static_cast<unsigned>(in_group - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ double gsum[kPartial];
  sum_partials(partials, grp * kGroup, in_group, gsum);
  if (threadIdx.x < kPartial) gsums[static_cast<size_t>(grp) * kPartial + threadIdx.x] = gsum[threadIdx.x];
  if (threadIdx.x == 0) group_cnt[grp] = 0u;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&st->arrived, 1u) == static_cast<unsigned>(ngroups - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  finish(gsums, ngroups, st, eps, mode, ns);
}

inline int iter_blocks(int64_t ns) {
  int64_t b = (ns + kThreads * kPPT - 1) / (kThreads * kPPT);
  return static_cast<int>(b < 1 ? 1 : b);
}

bool pose_ok(const double* T) {
  if (!T) return false;
  for (int k = 0; k < 16; ++k)
    if (!std::isfinite(T[k])) return false;
  return true;
}

Pose to_pose(const double* T) {
  Pose p;
  for (int k = 0; k < 16; ++k) p.m[k] = T[k];
  return p;
}

int32_t check_src(const char* fn, const float* d_src, int64_t ns, int32_t stride) {
  if (ns < 0 || ns > 0x7fffffffLL - kThreads * kPPT || (ns > 0 && !d_src) || stride < 3) {
    set_error("%s: invalid source cloud (n=%lld stride=%d)", fn, static_cast<long long>(ns), stride);
    return O3G_ERR_ARG;
  }
  return O3G_OK;
}

// Everything one ICP-style call needs on the device: the cell-sorted source,
// the iteration state and the block partials.
struct Work {
  SortedCloud src;
  DevBuf state;
  DevBuf partials;  // nblk block partials, then ngroups group sums
  DevBuf counters;  // ngroups arrival counters
  int nblk = 1, ngroups = 1;
  explicit Work(cudaStream_t s) : src(s), state(s), partials(s), counters(s) {}
  int32_t prepare(const float* d_src, int64_t ns, int32_t stride, float cell, const double* T, cudaStream_t s) {
    O3G_TRY_STATUS(sort_cloud(d_src, ns, stride, s, &src));
    nblk = iter_blocks(ns);
    ngroups = (nblk + kGroup - 1) / kGroup;
    O3G_TRY(state.alloc(sizeof(IcpState)));
    O3G_TRY(partials.alloc(sizeof(double) * kPartial * (nblk + ngroups)));
    O3G_TRY(counters.alloc(sizeof(unsigned) * ngroups));
    O3G_TRY(cudaMemsetAsync(counters.p, 0, sizeof(unsigned) * ngroups, s));
    k_init_state<<<1, 32, 0, s>>>(state.as<IcpState>(), to_pose(T));
    count_launch();
    return O3G_OK;
  }
  int32_t launch(const o3g_grid* g, int ns, float r, double eps, int mode, int32_t* corr, float* d2,
                 cudaStream_t s) {
    double* pp = partials.as<double>();
    k_icp_iter<<<nblk, kThreads, 0, s>>>(g->view(), g->cell, src.pts, ns, state.as<IcpState>(), r, pp,
                                         pp + static_cast<size_t>(kPartial) * nblk, counters.as<unsigned>(), eps,
                                         mode, corr, d2);
    count_launch();
    return O3G_OK;
  }
};

}  // namespace

int32_t icp_run(const o3g_grid* g, const float* d_src, int64_t ns, int32_t stride, const double* init_T,
                double max_corr_dist, int32_t max_iter, double eps, double* out_T, double* out_fitness,
                double* out_rmse, int32_t* out_iters, cudaStream_t s) {
  const char* fn = "o3g_icp_point_to_plane_grid";
  if (!g || !out_T || !out_fitness || !out_rmse || max_iter < 0 || !(max_corr_dist >= 0.0) ||
      !std::isfinite(max_corr_dist)) {
    set_error("%s: invalid argument", fn);
    return O3G_ERR_ARG;
  }
  O3G_TRY_STATUS(check_src(fn, d_src, ns, stride));
  if (!g->has_normals) {
    set_error("%s: the target grid carries no normals (attach or estimate them first)", fn);
    return O3G_ERR_ARG;
  }
  if (!pose_ok(init_T)) {
    set_error("%s: init_T is null or not finite", fn);
    return O3G_ERR_NONFINITE;
  }
  const float r = static_cast<float>(max_corr_dist);
  Work w(s);
  O3G_TRY_STATUS(w.prepare(d_src, ns, stride, g->cell, init_T, s));
  const int n = static_cast<int>(ns);
  for (int it = 0; it < max_iter; ++it) {
    TimedRegion tr(O3G_KERNEL_ICP_CORR, s);
    w.launch(g, n, r, eps, kIterate, nullptr, nullptr, s);
  }
  w.launch(g, n, r, eps, kEvaluate, nullptr, nullptr, s);
  O3G_TRY(cudaGetLastError());
  IcpState h;
  int aux[8];
  O3G_TRY(cudaMemcpyAsync(&h, w.state.p, sizeof(IcpState), cudaMemcpyDeviceToHost, s));
  O3G_TRY(cudaMemcpyAsync(aux, w.src.aux.p, sizeof(aux), cudaMemcpyDeviceToHost, s));
  O3G_TRY(cudaStreamSynchronize(s));
  if (aux[6]) {
    set_error("%s: non-finite source coordinate", fn);
    return O3G_ERR_NONFINITE;
  }
  if (h.nonfinite) {
    set_error("%s: the normal equations became non-finite (check the target normals)", fn);
    return O3G_ERR_NONFINITE;
  }
  for (int k = 0; k < 16; ++k) out_T[k] = h.T[k];
  *out_fitness = h.fitness;
  *out_rmse = h.rmse;
  if (out_iters) *out_iters = h.iters;
  if (h.few_corr) return O3G_WARN_FEW_CORR;
  if (h.degenerate) return O3G_WARN_DEGENERATE;
  return O3G_OK;
}

}  // namespace o3g

using namespace o3g;

extern "C" int32_t o3g_correspondences(const o3g_grid* g, const float* d_src, int64_t ns, int32_t stride,
                                       const double* T, float max_corr_dist, int32_t* d_corr, float* d_d2,
                                       void* stream) {
  const char* fn = "o3g_correspondences";
  if (!g || (ns > 0 && (!d_corr || !d_d2)) || !(max_corr_dist >= 0.f) || !std::isfinite(max_corr_dist)) {
    set_error("%s: invalid argument", fn);
    return O3G_ERR_ARG;
  }
  O3G_TRY_STATUS(check_src(fn, d_src, ns, stride));
  if (!pose_ok(T)) {
    set_error("%s: T is null or not finite", fn);
    return O3G_ERR_NONFINITE;
  }
  if (ns == 0) return O3G_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Work w(s);
  O3G_TRY_STATUS(w.prepare(d_src, ns, stride, g->cell, T, s));
  w.launch(g, static_cast<int>(ns), max_corr_dist, 0.0, kCorrOnly, d_corr, d_d2, s);
  O3G_TRY(cudaGetLastError());
  return O3G_OK;
}

extern "C" int32_t o3g_normal_equations(const o3g_grid* g, const float* d_src, int64_t ns, int32_t stride,
                                        const double* T, float max_corr_dist, double* out_A, double* out_b,
                                        double* out_stats, void* stream) {
  const char* fn = "o3g_normal_equations";
  if (!g || !out_A || !out_b || !out_stats || !(max_corr_dist >= 0.f) || !std::isfinite(max_corr_dist)) {
    set_error("%s: invalid argument", fn);
    return O3G_ERR_ARG;
  }
  O3G_TRY_STATUS(check_src(fn, d_src, ns, stride));
  if (!g->has_normals) {
    set_error("%s: the target grid carries no normals", fn);
    return O3G_ERR_ARG;
  }
  if (!pose_ok(T)) {
    set_error("%s: T is null or not finite", fn);
    return O3G_ERR_NONFINITE;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Work w(s);
  O3G_TRY_STATUS(w.prepare(d_src, ns, stride, g->cell, T, s));
  w.launch(g, static_cast<int>(ns), max_corr_dist, 0.0, kEquations, nullptr, nullptr, s);
  O3G_TRY(cudaGetLastError());
  IcpState h;
  O3G_TRY(cudaMemcpyAsync(&h, w.state.p, sizeof(IcpState), cudaMemcpyDeviceToHost, s));
  O3G_TRY(cudaStreamSynchronize(s));
  for (int k = 0; k < 36; ++k) out_A[k] = h.A[k];
  for (int k = 0; k < 6; ++k) out_b[k] = h.b[k];
  for (int k = 0; k < 3; ++k) out_stats[k] = h.stats[k];
  return O3G_OK;
}

extern "C" int32_t o3g_icp_point_to_plane_grid(const o3g_grid* g, const float* d_src, int64_t ns, int32_t stride,
                                               const double* init_T, double max_corr_dist, int32_t max_iter,
                                               double eps, double* out_T, double* out_fitness, double* out_rmse,
                                               int32_t* out_iters, void* stream) {
  return icp_run(g, d_src, ns, stride, init_T, max_corr_dist, max_iter, eps, out_T, out_fitness, out_rmse, out_iters,
                 static_cast<cudaStream_t>(stream));
}

extern "C" int32_t o3g_icp_point_to_plane(const float* d_src, int64_t ns, int32_t src_stride, const float* d_tgt,
                                          int64_t nt, int32_t tgt_stride, const float* d_tgt_nrm, int64_t n_nrm,
                                          int32_t nrm_stride, const double* init_T, double max_corr_dist,
                                          int32_t max_iter, double* out_T, double* out_fitness, double* out_rmse) {
  if (n_nrm != nt) {
    set_error("o3g_icp_point_to_plane: %lld target normals for %lld target points (must match one to one)",
              static_cast<long long>(n_nrm), static_cast<long long>(nt));
    return O3G_ERR_ARG;
  }
  if (!(max_corr_dist > 0.0) || !std::isfinite(max_corr_dist)) {
    set_error("o3g_icp_point_to_plane: max_corr_dist must be positive and finite");
    return O3G_ERR_ARG;
  }
  o3g_grid* g = nullptr;
  O3G_TRY_STATUS(o3g_build_grid(d_tgt, nt, tgt_stride, static_cast<float>(max_corr_dist), nullptr, &g));
  int32_t st = o3g_grid_set_normals(g, d_tgt_nrm, n_nrm, nrm_stride, nullptr);
  if (st >= 0)
    st = icp_run(g, d_src, ns, src_stride, init_T, max_corr_dist, max_iter, 0.0, out_T, out_fitness, out_rmse, nullptr,
                 nullptr);
  o3g_free_grid(g);
  return st;
}

// ---------------------------------------------------------------------------
// Allocation-free ICP: the same iteration kernel, with every scratch buffer
// carved out of one static device array instead of the memory pool.  For
// callers that cannot allocate once running (see o3g.h).

namespace o3g {
namespace {

constexpr size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }
constexpr int kNaMaxBlocks = (O3G_NOALLOC_MAX_POINTS + kThreads * kPPT - 1) / (kThreads * kPPT);
constexpr int kNaMaxGroups = (kNaMaxBlocks + kGroup - 1) / kGroup;
constexpr size_t kNaOffSrc = 0;
constexpr size_t kNaOffState = align256(kNaOffSrc + sizeof(float4) * static_cast<size_t>(O3G_NOALLOC_MAX_POINTS));
constexpr size_t kNaOffPartials = align256(kNaOffState + sizeof(IcpState));
constexpr size_t kNaOffCounters =
    align256(kNaOffPartials + sizeof(double) * kPartial * static_cast<size_t>(kNaMaxBlocks + kNaMaxGroups));
constexpr size_t kNaOffFlag = align256(kNaOffCounters + sizeof(unsigned) * kNaMaxGroups);
constexpr size_t kNaBytes = align256(kNaOffFlag + sizeof(int));
static_assert(kNaBytes == 4736256, "update the size stated in o3g.h");

// The working memory of o3g_icp_point_to_plane_grid_noalloc, shared by every call.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

std::mutex g_noalloc_mutex;
constexpr int kNaMaxDevices = 64;
void* g_noalloc_addr[kNaMaxDevices] = {};

// Source rows (caller order) -> float4 (x, y, z, index bits); flags non-finite coordinates.
__global__ void __launch_bounds__(kThreads) k_pack_src(const float* __restrict__ src, int n, int stride,
                                                       float4* __restrict__ out, int* __restrict__ bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* p = src + static_cast<int64_t>(i) * stride;
  const float x = p[0], y = p[1], z = p[2];
  if (!isfinite(x) || !isfinite(y) || !isfinite(z)) *bad = 1;
  out[i] = make_float4(x, y, z, __int_as_float(i));
}

// Device address of the static array on the current device (looked up once per device).
int32_t noalloc_scratch(unsigned char** out) {
  int dev = 0;
  O3G_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNaMaxDevices) {
    set_error("o3g_icp_point_to_plane_grid_noalloc: device %d out of range", dev);
    return O3G_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    O3G_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_noalloc_addr[dev]);
  return O3G_OK;
}

}  // namespace
}  // namespace o3g

extern "C" int32_t o3g_icp_point_to_plane_grid_noalloc(const o3g_grid* g, const float* d_src, int64_t ns,
                                                       int32_t stride, const double* init_T, double max_corr_dist,
                                                       int32_t max_iter, double eps, double* out_T,
                                                       double* out_fitness, double* out_rmse, int32_t* out_iters,
                                                       void* stream) {
  using namespace o3g;
  const char* fn = "o3g_icp_point_to_plane_grid_noalloc";
  if (!g || !out_T || !out_fitness || !out_rmse || max_iter < 0 || !(max_corr_dist >= 0.0) ||
      !std::isfinite(max_corr_dist)) {
    set_error("%s: invalid argument", fn);
    return O3G_ERR_ARG;
  }
  O3G_TRY_STATUS(check_src(fn, d_src, ns, stride));
  if (ns > O3G_NOALLOC_MAX_POINTS) {
    set_error("%s: %lld source points exceed the fixed working memory (at most %d points)", fn,
              static_cast<long long>(ns), O3G_NOALLOC_MAX_POINTS);
    return O3G_ERR_ARG;
  }
  if (!g->has_normals) {
    set_error("%s: the target grid carries no normals (attach or estimate them first)", fn);
    return O3G_ERR_ARG;
  }
  if (!pose_ok(init_T)) {
    set_error("%s: init_T is null or not finite", fn);
    return O3G_ERR_NONFINITE;
  }
  unsigned char* base = nullptr;
  O3G_TRY_STATUS(noalloc_scratch(&base));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float4* src4 = reinterpret_cast<float4*>(base + kNaOffSrc);
  IcpState* st = reinterpret_cast<IcpState*>(base + kNaOffState);
  double* partials = reinterpret_cast<double*>(base + kNaOffPartials);
  unsigned* counters = reinterpret_cast<unsigned*>(base + kNaOffCounters);
  int* bad = reinterpret_cast<int*>(base + kNaOffFlag);
  const int n = static_cast<int>(ns);
  const int nblk = iter_blocks(ns);
  const int ngroups = (nblk + kGroup - 1) / kGroup;
  // the arrival counters and the input flag must start at zero; the state is rewritten by k_init_state
  O3G_TRY(cudaMemsetAsync(counters, 0, sizeof(unsigned) * ngroups, s));
  O3G_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
  if (n > 0) {
    k_pack_src<<<(n + kThreads - 1) / kThreads, kThreads, 0, s>>>(d_src, n, stride, src4, bad);
    count_launch();
  }
  k_init_state<<<1, 32, 0, s>>>(st, to_pose(init_T));
  count_launch();
  const float r = static_cast<float>(max_corr_dist);
  const GridView gv = g->view();
  double* gsums = partials + static_cast<size_t>(kPartial) * nblk;
  for (int it = 0; it <= max_iter; ++it) {
    const int mode = it < max_iter ? kIterate : kEvaluate;
    k_icp_iter<<<nblk, kThreads, 0, s>>>(gv, g->cell, src4, n, st, r, partials, gsums, counters, eps, mode, nullptr,
                                         nullptr);
    count_launch();
  }
  O3G_TRY(cudaGetLastError());
  IcpState h;
  int h_bad = 0;
  O3G_TRY(cudaMemcpyAsync(&h, st, sizeof(IcpState), cudaMemcpyDeviceToHost, s));
  O3G_TRY(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  O3G_TRY(cudaStreamSynchronize(s));
  if (h_bad) {
    set_error("%s: non-finite source coordinate", fn);
    return O3G_ERR_NONFINITE;
  }
  if (h.nonfinite) {
    set_error("%s: the normal equations became non-finite (check the target normals)", fn);
    return O3G_ERR_NONFINITE;
  }
  for (int k = 0; k < 16; ++k) out_T[k] = h.T[k];
  *out_fitness = h.fitness;
  *out_rmse = h.rmse;
  if (out_iters) *out_iters = h.iters;
  if (h.few_corr) return O3G_WARN_FEW_CORR;
  if (h.degenerate) return O3G_WARN_DEGENERATE;
  return O3G_OK;
}
