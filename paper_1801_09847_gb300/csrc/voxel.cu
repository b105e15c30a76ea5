// Voxel downsampling (voxel_down_sample, Sec. 3.1 and Fig. 1: the thinning
// that precedes normal estimation and registration in every workflow).
//   voxel index  (floor(x / v), floor(y / v), floor(z / v)), each quotient one
//                correctly rounded float32 division; points with a non-finite
//                coordinate are dropped; an index outside [-2^30, 2^30] is an
//                argument error
//   order        voxels in increasing (ix, iy, iz), x most significant
//   centroid     float64 sum of the voxel's points in increasing input index,
//                divided by the count, rounded to float32
// Steps: voxel coordinates and their bounding box (one host round-trip to size
// the keys), a stable LSD radix sort of the point indices by a packed
// lexicographic key (or by z, then y, then x, then validity when the packed key
// would not fit 32 bits; invalid points sort last either way), segment heads by comparing
// neighbours and an exclusive scan, then one thread per voxel sums its points
// in sorted order, which within a voxel is input order (the sort is stable).
#include <climits>
#include <cmath>

#include "o3g_internal.cuh"

namespace o3g {
namespace {

constexpr int kThreads = 256;
constexpr float kMaxIndex = 1073741824.0f;  // 2^30

inline int blocks(int64_t n) { return static_cast<int>((n + kThreads - 1) / kThreads); }

// aux: 0-2 min (ix, iy, iz), 3-5 max, 6 range error, 7 valid points
__global__ void k_vox_init(int* aux) {
  if (threadIdx.x < 3) aux[threadIdx.x] = INT_MAX;
  else if (threadIdx.x < 6) aux[threadIdx.x] = INT_MIN;
  else if (threadIdx.x < 8) aux[threadIdx.x] = 0;
}

__global__ void __launch_bounds__(kThreads) k_vox_coords(const float* __restrict__ xyz, int n, int stride, float v,
                                                         int* __restrict__ vx, int* __restrict__ vy,
                                                         int* __restrict__ vz, int* __restrict__ aux) {
  const int i = blockIdx.x * kThreads + threadIdx.x;
  bool valid = false;
  int c[3] = {0, 0, 0};
  if (i < n) {
    const float* p = xyz + static_cast<int64_t>(i) * stride;
    const float x = p[0], y = p[1], z = p[2];
    if (isfinite(x) && isfinite(y) && isfinite(z)) {
      const float q[3] = {floorf(__fdiv_rn(x, v)), floorf(__fdiv_rn(y, v)), floorf(__fdiv_rn(z, v))};
      bool in_range = true;
#pragma unroll
      for (int k = 0; k < 3; ++k) in_range = in_range && q[k] >= -kMaxIndex && q[k] <= kMaxIndex;
      if (in_range) {
        valid = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) c[k] = static_cast<int>(q[k]);
      } else {
        atomicOr(&aux[6], 1);
      }
    }
    vx[i] = valid ? c[0] : INT_MIN;
    vy[i] = c[1];
    vz[i] = c[2];
  }
  const unsigned full = 0xffffffffu;
  const int lx = __reduce_min_sync(full, valid ? c[0] : INT_MAX), ly = __reduce_min_sync(full, valid ? c[1] : INT_MAX);
  const int lz = __reduce_min_sync(full, valid ? c[2] : INT_MAX);
  const int ux = __reduce_max_sync(full, valid ? c[0] : INT_MIN), uy = __reduce_max_sync(full, valid ? c[1] : INT_MIN);
  const int uz = __reduce_max_sync(full, valid ? c[2] : INT_MIN);
  const unsigned nv = __popc(__ballot_sync(full, valid));
  if ((threadIdx.x & 31) == 0 && nv) {
    atomicMin(&aux[0], lx);
    atomicMin(&aux[1], ly);
    atomicMin(&aux[2], lz);
    atomicMax(&aux[3], ux);
    atomicMax(&aux[4], uy);
    atomicMax(&aux[5], uz);
    atomicAdd(&aux[7], static_cast<int>(nv));
  }
}

// Packed key (x most significant); invalid points get bit `total` set.
__global__ void __launch_bounds__(kThreads) k_vox_packed_key(const int* __restrict__ vx, const int* __restrict__ vy,
                                                             const int* __restrict__ vz, int n, int3 lo, int by,
                                                             int bz, int total, uint32_t* __restrict__ keys,
                                                             uint32_t* __restrict__ idx) {
  const int i = blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  const int x = vx[i];
  uint32_t k;
  if (x == INT_MIN) {
    k = 1u << total;
  } else {
    k = (static_cast<uint32_t>(x - lo.x) << (by + bz)) | (static_cast<uint32_t>(vy[i] - lo.y) << bz) |
        static_cast<uint32_t>(vz[i] - lo.z);
  }
  keys[i] = k;
  idx[i] = static_cast<uint32_t>(i);
}

// One pass of the multi-pass order: the key of point idx[j] along one axis,
// relative to the box corner (invalid points 0), or with axis == nullptr the
// validity bit (invalid points 1, so a last pass puts them at the end).
__global__ void __launch_bounds__(kThreads) k_vox_axis_key(const int* __restrict__ vx, const int* __restrict__ axis,
                                                           int lo, const uint32_t* __restrict__ idx, int n,
                                                           uint32_t* __restrict__ keys) {
  const int j = blockIdx.x * kThreads + threadIdx.x;
  if (j >= n) return;
  const int i = static_cast<int>(idx[j]);
  const bool valid = vx[i] != INT_MIN;
  if (!axis) keys[j] = valid ? 0u : 1u;
  else keys[j] = valid ? static_cast<uint32_t>(static_cast<int64_t>(axis[i]) - lo) : 0u;
}

__global__ void __launch_bounds__(kThreads) k_iota(uint32_t* __restrict__ idx, int n) {
  const int j = blockIdx.x * kThreads + threadIdx.x;
  if (j < n) idx[j] = static_cast<uint32_t>(j);
}

// head[j] = 1 where sorted point j is valid and starts a new voxel.
__global__ void __launch_bounds__(kThreads) k_vox_heads(const int* __restrict__ vx, const int* __restrict__ vy,
                                                        const int* __restrict__ vz, const uint32_t* __restrict__ idx,
                                                        int n, uint32_t* __restrict__ head) {
  const int j = blockIdx.x * kThreads + threadIdx.x;
  if (j >= n) return;
  const int i = static_cast<int>(idx[j]);
  uint32_t h = 0u;
  if (vx[i] != INT_MIN) {
    if (j == 0) {
      h = 1u;
    } else {
      const int k = static_cast<int>(idx[j - 1]);
      h = (vx[k] != vx[i] || vy[k] != vy[i] || vz[k] != vz[i]) ? 1u : 0u;
    }
  }
  head[j] = h;
}

__global__ void __launch_bounds__(kThreads) k_vox_starts(const uint32_t* __restrict__ head,
                                                         const uint32_t* __restrict__ seg, int n,
                                                         uint32_t* __restrict__ start) {
  const int j = blockIdx.x * kThreads + threadIdx.x;
  if (j < n && head[j]) start[seg[j]] = static_cast<uint32_t>(j);
}

// Voxel s: float64 sum of its points in sorted (= input) order, mean, float32.
__global__ void __launch_bounds__(kThreads) k_vox_mean(const float* __restrict__ xyz, int stride,
                                                       const uint32_t* __restrict__ idx,
                                                       const uint32_t* __restrict__ start, int m, int n_valid,
                                                       float* __restrict__ out, int32_t* __restrict__ counts) {
  const int s = blockIdx.x * kThreads + threadIdx.x;
  if (s >= m) return;
  const int a = static_cast<int>(start[s]);
  const int b = s + 1 < m ? static_cast<int>(start[s + 1]) : n_valid;
  double sx = 0.0, sy = 0.0, sz = 0.0;
  for (int j = a; j < b; ++j) {
    const float* p = xyz + static_cast<int64_t>(idx[j]) * stride;
    sx += static_cast<double>(p[0]);
    sy += static_cast<double>(p[1]);
    sz += static_cast<double>(p[2]);
  }
  const double c = static_cast<double>(b - a);
  out[3 * static_cast<int64_t>(s) + 0] = __double2float_rn(sx / c);
  out[3 * static_cast<int64_t>(s) + 1] = __double2float_rn(sy / c);
  out[3 * static_cast<int64_t>(s) + 2] = __double2float_rn(sz / c);
  if (counts) counts[s] = b - a;
}

int bits_for(int64_t span) {  // bits to hold 0 .. span - 1 (span <= 2^31 + 1)
  int b = 0;
  while (b < 32 && (int64_t{1} << b) < span) ++b;
  return b;
}

}  // namespace
}  // namespace o3g

using namespace o3g;

extern "C" int32_t o3g_voxel_down_sample(const float* d_xyz, int64_t n64, int32_t stride, float voxel,
                                         float* d_out, int32_t* d_counts, int64_t* out_n, void* stream) {
  const char* fn = "o3g_voxel_down_sample";
  if (!out_n || n64 < 0 || n64 > INT_MAX - kThreads || stride < 3 || (n64 > 0 && (!d_xyz || !d_out)) ||
      !(voxel > 0.f) || !std::isfinite(voxel)) {
    set_error("%s: invalid argument (n=%lld stride=%d voxel=%g)", fn, static_cast<long long>(n64), stride,
              static_cast<double>(voxel));
    return O3G_ERR_ARG;
  }
  if (n64 == 0) {
    *out_n = 0;
    return O3G_OK;
  }
  const int n = static_cast<int>(n64);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TimedRegion tr(O3G_KERNEL_VOXEL, s);
  DevBuf coords(s), aux(s), keys(s), idx(s), tk(s), tv(s), head(s), seg(s);
  O3G_TRY(coords.alloc(sizeof(int) * 3 * static_cast<size_t>(n)));
  O3G_TRY(aux.alloc(sizeof(int) * 8));
  int* vx = coords.as<int>();
  int* vy = vx + n;
  int* vz = vy + n;
  k_vox_init<<<1, 32, 0, s>>>(aux.as<int>());
  k_vox_coords<<<blocks(n), kThreads, 0, s>>>(d_xyz, n, stride, voxel, vx, vy, vz, aux.as<int>());
  count_launch(2);
  int h[8];
  O3G_TRY(cudaMemcpyAsync(h, aux.p, sizeof(h), cudaMemcpyDeviceToHost, s));
  O3G_TRY(cudaStreamSynchronize(s));
  if (h[6]) {
    set_error("%s: a voxel index is outside [-2^30, 2^30] (voxel %g too small for the coordinates)", fn,
              static_cast<double>(voxel));
    return O3G_ERR_ARG;
  }
  const int n_valid = h[7];
  if (n_valid == 0) {
    *out_n = 0;
    return O3G_OK;
  }
  const int bx = bits_for(int64_t{h[3]} - h[0] + 1), by = bits_for(int64_t{h[4]} - h[1] + 1),
            bz = bits_for(int64_t{h[5]} - h[2] + 1);
  O3G_TRY(keys.alloc(sizeof(uint32_t) * n));
  O3G_TRY(idx.alloc(sizeof(uint32_t) * n));
  O3G_TRY(tk.alloc(sizeof(uint32_t) * n));
  O3G_TRY(tv.alloc(sizeof(uint32_t) * n));
  uint32_t* K = keys.as<uint32_t>();
  uint32_t* I = idx.as<uint32_t>();
  if (bx + by + bz + 1 <= 32) {
    k_vox_packed_key<<<blocks(n), kThreads, 0, s>>>(vx, vy, vz, n, make_int3(h[0], h[1], h[2]), by, bz,
                                                     bx + by + bz, K, I);
    count_launch();
    O3G_TRY_STATUS(radix_sort_pairs(K, I, tk.as<uint32_t>(), tv.as<uint32_t>(), n, bx + by + bz + 1, s));
  } else {
    // stable passes by z, then y, then x, then validity: lexicographic
    // (x, y, z) order with the invalid points at the end
    k_iota<<<blocks(n), kThreads, 0, s>>>(I, n);
    count_launch();
    const int* axes[4] = {vz, vy, vx, nullptr};
    const int los[4] = {h[2], h[1], h[0], 0};
    const int nbits[4] = {bz, by, bx, 1};
    for (int pass = 0; pass < 4; ++pass) {
      k_vox_axis_key<<<blocks(n), kThreads, 0, s>>>(vx, axes[pass], los[pass], I, n, K);
      count_launch();
      O3G_TRY_STATUS(radix_sort_pairs(K, I, tk.as<uint32_t>(), tv.as<uint32_t>(), n, nbits[pass], s));
    }
  }
  O3G_TRY(head.alloc(sizeof(uint32_t) * n));
  O3G_TRY(seg.alloc(sizeof(uint32_t) * n));
  k_vox_heads<<<blocks(n), kThreads, 0, s>>>(vx, vy, vz, I, n, head.as<uint32_t>());
  count_launch();
  O3G_TRY_STATUS(exclusive_scan_u32(head.as<uint32_t>(), seg.as<uint32_t>(), n, s));
  uint32_t last[2];
  O3G_TRY(cudaMemcpyAsync(&last[0], seg.as<uint32_t>() + (n - 1), sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  O3G_TRY(cudaMemcpyAsync(&last[1], head.as<uint32_t>() + (n - 1), sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  O3G_TRY(cudaStreamSynchronize(s));
  const int m = static_cast<int>(last[0] + last[1]);
  // segment starts reuse the key buffer (no longer needed)
  k_vox_starts<<<blocks(n), kThreads, 0, s>>>(head.as<uint32_t>(), seg.as<uint32_t>(), n, K);
  k_vox_mean<<<blocks(m), kThreads, 0, s>>>(d_xyz, stride, I, K, m, n_valid, d_out, d_counts);
  count_launch(2);
  O3G_TRY(cudaGetLastError());
  O3G_TRY(cudaStreamSynchronize(s));
  *out_n = m;
  return O3G_OK;
}
