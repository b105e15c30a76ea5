// Internal declarations shared by the translation units of libo3g.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "o3g.h"

namespace o3g {

// ----------------------------------------------------------------- errors

void set_error(const char* fmt, ...);
int32_t cuda_fail(cudaError_t e, const char* what);

#define O3G_TRY(call)                                          \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return ::o3g::cuda_fail(e_, #call); \
  } while (0)

#define O3G_TRY_STATUS(expr)        \
  do {                              \
    int32_t s_ = (expr);            \
    if (s_ < 0) return s_;          \
  } while (0)

// --------------------------------------------------------- device memory

// Stream-ordered allocation from the library's private pool on the current device.
cudaError_t dmalloc(void** p, size_t bytes, cudaStream_t s);
void dfree(void* p, cudaStream_t s);

// RAII holder for pool allocations that must be released on every return path.
struct DevBuf {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  explicit DevBuf(cudaStream_t st) : s(st) {}
  ~DevBuf() {
    if (p) dfree(p, s);
  }
  cudaError_t alloc(size_t bytes) { return dmalloc(&p, bytes ? bytes : 16, s); }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
};

constexpr int kNumSMs = 152;  // GB300

// ------------------------------------------------------ instrumentation

// Counts one kernel launch (o3g_launch_count).
void count_launch(int n = 1);
// Event bracket around a launch of kernel `kind` on stream s when timing is on.
struct TimedRegion {
  int kind;
  cudaStream_t s;
  void* ev0 = nullptr;
  TimedRegion(int k, cudaStream_t st);
  ~TimedRegion();
};

// ------------------------------------------- cross-file entry points

int32_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t m, cudaStream_t s);

// A cloud copied into a spatially coherent order (30-bit Morton code over its
// bounding box, stable sort) as float4 (x, y, z, original index bits), so that
// consecutive threads work on nearby points.  aux[6] is set to 1 if some
// coordinate was not finite.  No host synchronisation.
struct SortedCloud {
  DevBuf buf;
  DevBuf aux;
  float4* pts = nullptr;
  explicit SortedCloud(cudaStream_t s) : buf(s), aux(s) {}
};
int32_t sort_cloud(const float* d_xyz, int64_t n, int32_t stride, cudaStream_t s, SortedCloud* out);
int32_t sort_clouds_batch(const float* const* d_ptrs, const int32_t* d_strides, const int64_t* d_offsets,
                          int n_pairs, int64_t total, cudaStream_t s, float4* out, int* aux);
int32_t radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* tmp_k, uint32_t* tmp_v, int n, int bits,
                         cudaStream_t s, uint32_t* hist0 = nullptr);

// ------------------------------------------------------------ the grid

// Kernel-side view of a uniform grid: points sorted by linear cell index
// (z fastest), and cell_start[c] = number of points whose cell index is < c.
struct GridView {
  const float4* pts;         // sorted points; .w holds the original index (int bits)
  const float4* nrm;         // sorted normals (.w = 0), or null; nrm[n].x bounds their length
  const uint32_t* cell_start;  // cells + 1 entries
  const uint32_t* col_z;     // per (x, y) column: lowest | highest occupied z cell << 16 (empty: 0xffff)
  int lo_x, lo_y, lo_z;      // smallest occupied cell coordinate per axis
  int sx, sy, sz;            // cell span per axis
  float inv_cell;
  float cell;                // cell edge (inv_cell = 1 / cell, rounded)
  int n;
};

// Cell coordinate of one coordinate value.  Used identically when building
// and when querying, so the two always agree.  Clamped to +-2^20.
__device__ __forceinline__ int cell_coord(float x, float inv_cell) {
  float v = floorf(__fmul_rn(x, inv_cell));
  v = fminf(fmaxf(v, -1048576.0f), 1048575.0f);
  return static_cast<int>(v);
}

// Range of grid cells (relative, clamped to the grid) along one axis that can
// hold a point whose float32 squared distance to coordinate p is <= fl(r)^2.
// The margin covers the rounding of the distance and of p -+ r.
__device__ __forceinline__ void axis_range(float p, float r, float inv_cell, int lo, int span, int& a, int& b) {
  float m = __fadd_rn(__fmul_rn(r, 1.0001f), __fmul_rn(fabsf(p), 1e-6f));
  a = max(cell_coord(__fsub_rn(p, m), inv_cell) - lo, 0);
  b = min(cell_coord(__fadd_rn(p, m), inv_cell) - lo, span - 1);
}

// Narrows [zl, zh] to the occupied z-cells of column col_xy; false if none remain.
__device__ __forceinline__ bool column_z(const GridView& g, int col_xy, int& zl, int& zh) {
  const uint32_t e = g.col_z[col_xy];
  zl = max(zl, static_cast<int>(e & 0xffffu));
  zh = min(zh, static_cast<int>(e >> 16));
  return zl <= zh;
}

// Lower bound (with a rounding margin) of |c - x| over the cell slab
// [(lo + i) * cell, (lo + i + 1) * cell) along one axis.
__device__ __forceinline__ float slab_gap(float x, int i_abs, float cell, float margin) {
  const float a = __fmul_rn(static_cast<float>(i_abs), cell);
  const float b = __fmul_rn(static_cast<float>(i_abs + 1), cell);
  const float g = fmaxf(fmaxf(a - x, x - b), 0.f);
  return fmaxf(g - margin, 0.f);
}

// Rounding margin of the exact searches: covers the float32 rounding of the
// distance, of the bound and of the cell arithmetic for a query at p.
__device__ __forceinline__ float search_margin(float cell, float r, float px, float py, float pz) {
  return __fadd_rn(__fmul_rn(__fadd_rn(cell, r), 1e-5f),
                   __fmul_rn(fmaxf(fmaxf(fabsf(px), fabsf(py)), fabsf(pz)), 4e-6f));
}

// sqrt(x) for x >= 0 from the hardware reciprocal square root (a few ulp): the
// search bounds add a relative margin far larger than that error.
__device__ __forceinline__ float fast_sqrt(float x) {
  const float y = fmaxf(x, 1e-30f);
  return y * rsqrtf(y);
}

// d2 = (dx*dx + dy*dy) + dz*dz with d = p - q, every operation rounded on its own.
__device__ __forceinline__ float dist2_rn(float px, float py, float pz, float4 q) {
  float dx = __fsub_rn(px, q.x), dy = __fsub_rn(py, q.y), dz = __fsub_rn(pz, q.z);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// p = R s + t per row as ((R0 sx + R1 sy) + R2 sz) + t, no contraction.
__device__ __forceinline__ float3 xform_rn(const float* R, const float* t, float sx, float sy, float sz) {
  float3 p;
  p.x = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(R[0], sx), __fmul_rn(R[1], sy)), __fmul_rn(R[2], sz)), t[0]);
  p.y = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(R[3], sx), __fmul_rn(R[4], sy)), __fmul_rn(R[5], sz)), t[1]);
  p.z = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(R[6], sx), __fmul_rn(R[7], sy)), __fmul_rn(R[8], sz)), t[2]);
  return p;
}

}  // namespace o3g

struct o3g_grid;

namespace o3g {
// ICP on a target grid (point-to-plane, or point-to-point); `pre`, when given,
// is the source already sorted (sort_cloud of d_src, complete before work on s).
int32_t icp_run(const o3g_grid* g, const float* d_src, int64_t ns, int32_t stride, const double* init_T,
                double max_corr_dist, int32_t max_iter, double eps, double* out_T, double* out_fitness,
                double* out_rmse, int32_t* out_iters, cudaStream_t s, int32_t precision = O3G_PREC_F32_COMPENSATED,
                bool point_to_point = false, const SortedCloud* pre = nullptr, int32_t* d_corr = nullptr,
                float* d_d2 = nullptr);
// A library-owned non-blocking stream per device for work beside the caller's stream.
cudaError_t side_stream(cudaStream_t* out);
int32_t estimate_normals_impl(o3g_grid* g, float radius, int32_t max_nn, const float* viewpoint, float* d_out,
                              int32_t out_stride, cudaStream_t s);
}  // namespace o3g

// The opaque handle of the C ABI.
struct o3g_grid {
  int64_t n = 0;
  float cell = 0.f, inv_cell = 0.f;
  int lo[3] = {0, 0, 0};
  int span[3] = {1, 1, 1};
  float box_lo[3] = {0.f, 0.f, 0.f};  // coordinate bounding box of the points
  float box_hi[3] = {0.f, 0.f, 0.f};
  int64_t cells = 1;
  float4* pts = nullptr;
  float4* nrm = nullptr;  // n + 1 entries: the sorted normals, then (length bound, 0, 0, 0)
  uint32_t* cell_start = nullptr;
  uint32_t* col_z = nullptr;  // per column: lowest | highest occupied z cell << 16
  int32_t* pos_of = nullptr;  // original index -> sorted position
  bool has_normals = false;
  cudaStream_t stream = nullptr;

  o3g::GridView view() const {
    o3g::GridView v;
    v.pts = pts;
    v.nrm = has_normals ? nrm : nullptr;
    v.cell_start = cell_start;
    v.col_z = col_z;
    v.lo_x = lo[0];
    v.lo_y = lo[1];
    v.lo_z = lo[2];
    v.sx = span[0];
    v.sy = span[1];
    v.sz = span[2];
    v.inv_cell = inv_cell;
    v.cell = cell;
    v.n = static_cast<int>(n);
    return v;
  }
};
