// Uniform grid over a point cloud, built by a stable sort on the linear cell
// index.  Replaces the kd-tree that Open3D uses for nearest-neighbour search
// (Sec. 2: FLANN) with a layout suited to fixed-radius queries on the GPU:
//   1. bounding box of the cell coordinates (one host round-trip, to size it);
//   2. key = linear cell index over that box (z fastest), value = point index;
//   3. stable LSD radix sort of (key, value), 8-bit digits;
//   4. cell_start[c] = number of points with key < c (dense, cells + 1 entries);
//   5. gather the points into sorted order as float4 (x, y, z, original index).
// A query box then reads each (x, y) column of cells as ONE contiguous run of
// the sorted points: [cell_start[col + z_lo], cell_start[col + z_hi + 1]).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>

#include "o3g_internal.cuh"

namespace o3g {

namespace {

constexpr int kThreads = 256;

// --------------------------------------------------------------- bbox

// bb: cell coordinate minima (0-2) and maxima (3-5), the non-finite flag (6),
// and the coordinate minima (7-9) and maxima (10-12) as float_key values.
__global__ void k_bbox_init(int* bb) {
  const int t = threadIdx.x;
  if (t < 3 || (t >= 7 && t < 10)) bb[t] = INT_MAX;
  else if (t < 6 || (t >= 10 && t < 13)) bb[t] = INT_MIN;
  else if (t == 6) bb[6] = 0;
}

// An int ordered like the float it encodes (non-NaN); its own inverse.
__host__ __device__ __forceinline__ int float_key(int bits) { return bits ^ ((bits >> 31) & 0x7fffffff); }

__global__ void __launch_bounds__(kThreads) k_bbox(const float* __restrict__ xyz, int n, int stride, float inv,
                                                   int* __restrict__ bb) {
  int mn0 = INT_MAX, mn1 = INT_MAX, mn2 = INT_MAX;
  int mx0 = INT_MIN, mx1 = INT_MIN, mx2 = INT_MIN;
  int fn[3] = {INT_MAX, INT_MAX, INT_MAX}, fx[3] = {INT_MIN, INT_MIN, INT_MIN};
  int bad = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float* p = xyz + static_cast<int64_t>(i) * stride;
    float x = p[0], y = p[1], z = p[2];
    if (!isfinite(x) || !isfinite(y) || !isfinite(z)) {
      bad = 1;
      continue;
    }
    int cx = cell_coord(x, inv), cy = cell_coord(y, inv), cz = cell_coord(z, inv);
    mn0 = min(mn0, cx);
    mn1 = min(mn1, cy);
    mn2 = min(mn2, cz);
    mx0 = max(mx0, cx);
    mx1 = max(mx1, cy);
    mx2 = max(mx2, cz);
    const int kx = float_key(__float_as_int(x)), ky = float_key(__float_as_int(y)), kz = float_key(__float_as_int(z));
    fn[0] = min(fn[0], kx);
    fn[1] = min(fn[1], ky);
    fn[2] = min(fn[2], kz);
    fx[0] = max(fx[0], kx);
    fx[1] = max(fx[1], ky);
    fx[2] = max(fx[2], kz);
  }
  // warp, then block reduction; one atomic per value per block
  const unsigned full = 0xffffffffu;
  int v[13] = {mn0, mn1, mn2, mx0, mx1, mx2, bad, fn[0], fn[1], fn[2], fx[0], fx[1], fx[2]};
#pragma unroll
  for (int k = 0; k < 13; ++k) {
    if (k < 3 || (k >= 7 && k < 10)) v[k] = __reduce_min_sync(full, v[k]);
    else if (k == 6) v[k] = __reduce_or_sync(full, v[k]);
    else v[k] = __reduce_max_sync(full, v[k]);
  }
  __shared__ int part[kThreads / 32][13];
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < 13; ++k) part[warp][k] = v[k];
  __syncthreads();
  const int k = threadIdx.x;
  if (k < 13) {
    int r = part[0][k];
    for (int w = 1; w < kThreads / 32; ++w) {
      const int x = part[w][k];
      r = (k < 3 || (k >= 7 && k < 10)) ? min(r, x) : (k == 6 ? (r | x) : max(r, x));
    }
    // an empty block (all of its points non-finite or none) leaves the extremes untouched
    if (k == 6) {
      if (r) atomicOr(bb + 6, 1);
    } else if (k < 3 || (k >= 7 && k < 10)) {
      if (r != INT_MAX) atomicMin(bb + k, r);
    } else if (r != INT_MIN) {
      atomicMax(bb + k, r);
    }
  }
}

// ---------------------------------------------------------------- keys

// Linear cell key of point i.
__device__ __forceinline__ uint32_t cell_key(const float* __restrict__ xyz, int i, int stride, float inv, int lx, int ly,
                                             int lz, uint32_t sy, uint32_t sz) {
  const float* p = xyz + static_cast<int64_t>(i) * stride;
  uint32_t cx = static_cast<uint32_t>(cell_coord(p[0], inv) - lx);
  uint32_t cy = static_cast<uint32_t>(cell_coord(p[1], inv) - ly);
  uint32_t cz = static_cast<uint32_t>(cell_coord(p[2], inv) - lz);
  return (cx * sy + cy) * sz + cz;
}

// -------------------------------------------------------- exclusive scan

constexpr int kScanItems = 8;
constexpr int kScanTile = kThreads * kScanItems;

// Exclusive scan of one value per thread across the block; *total = block sum.
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_sums[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_sums[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kThreads / 32) warp_sums[lane] = w;  // inclusive
  }
  __syncthreads();
  uint32_t warp_off = warp == 0 ? 0 : warp_sums[warp - 1];
  *total = warp_sums[kThreads / 32 - 1];
  __syncthreads();
  return warp_off + inc - v;
}

__global__ void __launch_bounds__(kThreads) k_scan_reduce(const uint32_t* __restrict__ in, int64_t m,
                                                          uint32_t* __restrict__ bsum) {
  int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile + static_cast<int64_t>(threadIdx.x) * kScanItems;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < m) s += in[base + k];
  uint32_t total;
  block_exclusive_scan(s, &total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// Single block: in-place exclusive scan of nb block sums.
__global__ void __launch_bounds__(kThreads) k_scan_top(uint32_t* __restrict__ bsum, int nb) {
  uint32_t carry = 0;
  for (int c0 = 0; c0 < nb; c0 += kScanTile) {
    int base = c0 + threadIdx.x * kScanItems;
    uint32_t v[kScanItems], s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      v[k] = base + k < nb ? bsum[base + k] : 0;
      s += v[k];
    }
    uint32_t total;
    uint32_t off = block_exclusive_scan(s, &total) + carry;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      if (base + k < nb) bsum[base + k] = off;
      off += v[k];
    }
    carry += total;
  }
}

__global__ void __launch_bounds__(kThreads) k_scan_down(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                        int64_t m, const uint32_t* __restrict__ bsum) {
  int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile + static_cast<int64_t>(threadIdx.x) * kScanItems;
  uint32_t v[kScanItems], s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = base + k < m ? in[base + k] : 0;
    s += v[k];
  }
  uint32_t total;
  uint32_t off = block_exclusive_scan(s, &total) + bsum[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < m) out[base + k] = off;
    off += v[k];
  }
}

// ---------------------------------------------------------- radix sort

constexpr int kRsRounds = 8;
constexpr int kRsTile = kThreads * kRsRounds;
constexpr int kWarps = kThreads / 32;
// Sorts of at most this many tiles skip the separate scan of the per-tile digit
// counts: each scatter block sums the counts it needs itself (every block reads
// all nblk x 256 counts once, which beats three more launches while nblk is small).
constexpr int kRsInlineBlocks = 160;

// Per-tile digit counts: digit-major (count of digit d in tile b at d * nblk +
// b, the order whose exclusive scan gives every tile's offsets) or, with
// kTileMajor, at b * 256 + d for the scatter to sum itself.
template <bool kTileMajor>
__device__ __forceinline__ void store_hist(uint32_t* __restrict__ hist, int nblk, uint32_t count) {
  if (kTileMajor) hist[static_cast<size_t>(blockIdx.x) * 256 + threadIdx.x] = count;
  else hist[static_cast<size_t>(threadIdx.x) * nblk + blockIdx.x] = count;
}

template <bool kTileMajor>
__global__ void __launch_bounds__(kThreads) k_rs_hist(const uint32_t* __restrict__ keys, int n, int shift,
                                                      uint32_t* __restrict__ hist, int nblk) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int base = blockIdx.x * kRsTile;
#pragma unroll
  for (int r = 0; r < kRsRounds; ++r) {
    int i = base + r * kThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  store_hist<kTileMajor>(hist, nblk, h[threadIdx.x]);
}

// The grid build's first step: cell keys (and identity values) of tile b, with
// the tile's counts of the first sort digit.
template <bool kTileMajor>
__global__ void __launch_bounds__(kThreads) k_keys_hist(const float* __restrict__ xyz, int n, int stride, float inv,
                                                        int lx, int ly, int lz, uint32_t sy, uint32_t sz,
                                                        uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                        uint32_t* __restrict__ hist, int nblk) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int base = blockIdx.x * kRsTile;
#pragma unroll
  for (int r = 0; r < kRsRounds; ++r) {
    int i = base + r * kThreads + threadIdx.x;
    if (i < n) {
      const uint32_t k = cell_key(xyz, i, stride, inv, lx, ly, lz, sy, sz);
      keys[i] = k;
      vals[i] = static_cast<uint32_t>(i);
      atomicAdd(&h[k & 255u], 1u);
    }
  }
  __syncthreads();
  store_hist<kTileMajor>(hist, nblk, h[threadIdx.x]);
}

// Stable scatter of one tile: elements keep their input order within a digit.
// Rounds walk the tile in order; inside a round, warps in order; inside a warp,
// lanes in order (rank among equal digits via __match_any_sync).  The tile's
// first output position for each digit comes from the scanned digit-major
// counts or, with kInline, from the tile-major counts: all tiles' counts of
// smaller digits plus the earlier tiles' counts of the same digit.
template <bool kInline>
__global__ void __launch_bounds__(kThreads) k_rs_scatter(const uint32_t* __restrict__ kin,
                                                         const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
                                                         uint32_t* __restrict__ vout, int n, int shift,
                                                         const uint32_t* __restrict__ offs, int nblk) {
  __shared__ uint32_t base[256];
  __shared__ uint32_t wcnt[kWarps][256];
  __shared__ uint32_t total[256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  if (kInline) {
    uint32_t all = 0, before = 0;
    for (int b = 0; b < nblk; ++b) {
      const uint32_t c = offs[static_cast<size_t>(b) * 256 + tid];
      all += c;
      before += b < static_cast<int>(blockIdx.x) ? c : 0u;
    }
    uint32_t sum;
    base[tid] = block_exclusive_scan(all, &sum) + before;
  } else {
    base[tid] = offs[static_cast<size_t>(tid) * nblk + blockIdx.x];
  }
  const int tile0 = blockIdx.x * kRsTile;
  for (int r = 0; r < kRsRounds; ++r) {
#pragma unroll
    for (int w = 0; w < kWarps; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    int i = tile0 + r * kThreads + tid;
    bool valid = i < n;
    uint32_t k = valid ? kin[i] : 0u, v = valid ? vin[i] : 0u;
    uint32_t d = (k >> shift) & 255u;
    uint32_t peers = __match_any_sync(0xffffffffu, valid ? d : 256u);
    uint32_t rank = __popc(peers & lt);
    if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t run = 0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        uint32_t c = wcnt[w][tid];
        wcnt[w][tid] = run;
        run += c;
      }
      total[tid] = run;
    }
    __syncthreads();
    if (valid) {
      uint32_t pos = base[d] + wcnt[warp][d] + rank;
      kout[pos] = k;
      vout[pos] = v;
    }
    __syncthreads();
    base[tid] += total[tid];
  }
}

// ------------------------------------------------------ cell table, gather

// cell_start[c] = the number of points whose key is < c (the first position
// with key >= c), c = 0 .. cells.  Small tables: one binary search over all n
// keys per cell (k_cell_start_direct).  Large tables (more cells than
// kChunkedMinCells, where every thread of a full wave has several cells): a
// block takes kCellsPerThread * kThreads consecutive cells, two threads find
// the positions of the chunk's first cell and of the cell after it, every cell
// of the chunk starts between those two, and each thread finds its cells'
// starts by binary searches inside that narrow range (cached; coalesced
// writes).  Measured: the 2M-point fragment's 8.5M-cell grid 0.316 -> 0.278 ms;
// on the RGB-D frame's 53,200-cell table (52 chunks) the direct form stays
// faster (0.077 against 0.090 ms).
constexpr int kCellsPerThread = 8;
constexpr int64_t kChunkedMinCells = int64_t{4} * kNumSMs * 16 * kThreads;
__global__ void __launch_bounds__(kThreads) k_cell_start_direct(const uint32_t* __restrict__ skeys, int n,
                                                                uint32_t* __restrict__ cell_start, int64_t cells) {
  for (int64_t c = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; c <= cells;
       c += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int lo = 0, hi = n;  // first position with key >= c
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (static_cast<int64_t>(skeys[mid]) < c) lo = mid + 1;
      else hi = mid;
    }
    cell_start[c] = static_cast<uint32_t>(lo);
  }
}
__device__ __forceinline__ int key_lower_bound(const uint32_t* __restrict__ skeys, int lo, int hi, int64_t c) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (static_cast<int64_t>(skeys[mid]) < c) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}
__global__ void __launch_bounds__(kThreads) k_cell_start(const uint32_t* __restrict__ skeys, int n,
                                                         uint32_t* __restrict__ cell_start, int64_t cells) {
  __shared__ int range[2];
  const int64_t chunk = static_cast<int64_t>(kThreads) * kCellsPerThread;
  for (int64_t c0 = static_cast<int64_t>(blockIdx.x) * chunk; c0 <= cells;
       c0 += static_cast<int64_t>(gridDim.x) * chunk) {
    if (threadIdx.x < 2) range[threadIdx.x] = key_lower_bound(skeys, 0, n, threadIdx.x == 0 ? c0 : c0 + chunk);
    __syncthreads();
    const int rlo = range[0], rhi = range[1];
    for (int k = 0; k < kCellsPerThread; ++k) {
      const int64_t c = c0 + static_cast<int64_t>(k) * kThreads + threadIdx.x;
      if (c > cells) break;
      cell_start[c] = static_cast<uint32_t>(key_lower_bound(skeys, rlo, rhi, c));
    }
    __syncthreads();  // range is rewritten for the next chunk
  }
}

// Per (x, y) column: the lowest and highest occupied z-cell, from cell_start by
// binary search (cell_start is non-decreasing along the column).  Empty columns
// get lowest = 0xffff, highest = 0, an empty range.
__device__ __forceinline__ void col_extent(const uint32_t* __restrict__ cell_start, int c, int sz,
                                           uint32_t* __restrict__ col_z) {
  const uint32_t* cs = cell_start + static_cast<int64_t>(c) * sz;
  const uint32_t first = cs[0], last = cs[sz];
  if (first == last) {
    col_z[c] = 0xffffu;
    return;
  }
  int lo = 0, hi = sz - 1;  // lowest z with cs[z + 1] > first
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (cs[mid + 1] > first) hi = mid;
    else lo = mid + 1;
  }
  const int zmin = lo;
  lo = 0;
  hi = sz - 1;  // highest z with cs[z] < last
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cs[mid] < last) lo = mid;
    else hi = mid - 1;
  }
  col_z[c] = static_cast<uint32_t>(zmin) | (static_cast<uint32_t>(lo) << 16);
}

__global__ void k_empty_col(uint32_t* col_z) { col_z[0] = 0xffffu; }

// The grid's last step, two independent parts in one launch: blocks below nbz
// find the occupied z-range of every (x, y) column (grid-stride), the others
// copy the points into cell order (point k of the sorted order is input point
// perm[k]), record where each input point went and zero the normals' length
// bound (no normals yet).
__global__ void __launch_bounds__(kThreads) k_col_extent_gather(const uint32_t* __restrict__ cell_start, int ncol,
                                                                int sz, uint32_t* __restrict__ col_z, int nbz,
                                                                const float* __restrict__ xyz, int n, int stride,
                                                                const uint32_t* __restrict__ perm,
                                                                float4* __restrict__ pts,
                                                                int32_t* __restrict__ pos_of,
                                                                float4* __restrict__ nrm) {
  if (static_cast<int>(blockIdx.x) < nbz) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncol; c += nbz * blockDim.x)
      col_extent(cell_start, c, sz, col_z);
    return;
  }
  int k = (blockIdx.x - nbz) * blockDim.x + threadIdx.x;
  if (k == 0) nrm[n] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (k >= n) return;
  uint32_t o = perm[k];
  const float* p = xyz + static_cast<int64_t>(o) * stride;
  pts[k] = make_float4(p[0], p[1], p[2], __int_as_float(static_cast<int>(o)));
  pos_of[o] = k;
}

__global__ void __launch_bounds__(kThreads) k_set_normals(const float* __restrict__ nrm, int stride,
                                                          const float4* __restrict__ pts, int n,
                                                          float4* __restrict__ out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  float len = 0.f;
  if (k < n) {
    int o = __float_as_int(pts[k].w);
    const float* q = nrm + static_cast<int64_t>(o) * stride;
    out[k] = make_float4(q[0], q[1], q[2], 0.f);
    len = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
    if (!isfinite(len)) len = 0.f;  // such a normal, where a correspondence uses it, makes its terms non-finite
  }
  // out[n].x (zeroed before the launch): the largest finite normal length, the
  // bound the ICP sums are scaled by (non-negative floats order like their bits
  // as ints).
  const int bits = static_cast<int>(__reduce_max_sync(0xffffffffu, static_cast<unsigned>(__float_as_int(len))));
  if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int*>(&out[n].x), bits);
}

inline int blocks_for(int64_t n, int per_block) {
  int64_t b = (n + per_block - 1) / per_block;
  return static_cast<int>(b < 1 ? 1 : b);
}

// ------------------------------------------ spatially coherent point order

// Order-preserving map of a float to an int (for atomicMin / atomicMax).
__device__ __forceinline__ int ordered_int(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ordered_float(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

__device__ __forceinline__ void k_fbox_init_one(int* aux) {
  for (int k = 0; k < 3; ++k) aux[k] = INT_MAX;
  for (int k = 3; k < 6; ++k) aux[k] = INT_MIN;
  aux[6] = 0;
}

__global__ void k_fbox_init(int* aux) {
  if (threadIdx.x == 0) k_fbox_init_one(aux);
}

__global__ void __launch_bounds__(kThreads) k_fbox(const float* __restrict__ xyz, int n, int stride,
                                                   int* __restrict__ aux) {
  int mn[3] = {INT_MAX, INT_MAX, INT_MAX}, mx[3] = {INT_MIN, INT_MIN, INT_MIN};
  int bad = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float* p = xyz + static_cast<int64_t>(i) * stride;
    const float v[3] = {p[0], p[1], p[2]};
    if (!isfinite(v[0]) || !isfinite(v[1]) || !isfinite(v[2])) {
      bad = 1;
      continue;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      mn[a] = min(mn[a], ordered_int(v[a]));
      mx[a] = max(mx[a], ordered_int(v[a]));
    }
  }
  // warp, then block reduction; one atomic per value per block
  int v[7] = {mn[0], mn[1], mn[2], mx[0], mx[1], mx[2], bad};
#pragma unroll
  for (int k = 0; k < 7; ++k)
    v[k] = k < 3 ? __reduce_min_sync(0xffffffffu, v[k])
                 : (k < 6 ? __reduce_max_sync(0xffffffffu, v[k]) : __reduce_or_sync(0xffffffffu, v[k]));
  __shared__ int part[kThreads / 32][7];
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < 7; ++k) part[threadIdx.x >> 5][k] = v[k];
  __syncthreads();
  const int k = threadIdx.x;
  if (k < 7) {
    int r = part[0][k];
    for (int w = 1; w < kThreads / 32; ++w) {
      const int x = part[w][k];
      r = k < 3 ? min(r, x) : (k < 6 ? max(r, x) : (r | x));
    }
    if (k < 3) {
      if (r != INT_MAX) atomicMin(aux + k, r);
    } else if (k < 6) {
      if (r != INT_MIN) atomicMax(aux + k, r);
    } else if (r) {
      atomicOr(aux + 6, 1);
    }
  }
}

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// 30-bit Morton code of the point quantised to 1024 steps per axis of the box in aux.
__device__ __forceinline__ uint32_t morton_of(const float* p, const int* aux) {
  uint32_t q[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float lo = aux[a] == INT_MAX ? 0.f : ordered_float(aux[a]);
    const float hi = aux[3 + a] == INT_MIN ? 0.f : ordered_float(aux[3 + a]);
    const float ext = fmaxf(hi - lo, 1e-30f);
    const float u = fminf(fmaxf((p[a] - lo) * (1023.0f / ext), 0.f), 1023.f);  // NaN -> 0
    q[a] = static_cast<uint32_t>(u);
  }
  return spread10(q[0]) | (spread10(q[1]) << 1) | (spread10(q[2]) << 2);
}

__global__ void __launch_bounds__(kThreads) k_morton(const float* __restrict__ xyz, int n, int stride,
                                                     const int* __restrict__ aux, uint32_t* __restrict__ keys,
                                                     uint32_t* __restrict__ vals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = morton_of(xyz + static_cast<int64_t>(i) * stride, aux);
  vals[i] = static_cast<uint32_t>(i);
}

__global__ void __launch_bounds__(kThreads) k_gather4(const float* __restrict__ xyz, int n, int stride,
                                                      const uint32_t* __restrict__ perm, float4* __restrict__ pts) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint32_t o = perm[k];
  const float* p = xyz + static_cast<int64_t>(o) * stride;
  pts[k] = make_float4(p[0], p[1], p[2], __int_as_float(static_cast<int>(o)));
}

}  // namespace

namespace {

// Pair of global point g: last p with offsets[p] <= g (offsets has n_pairs + 1 entries).
__device__ __forceinline__ int pair_of(const int64_t* __restrict__ offsets, int n_pairs, int64_t g) {
  int lo = 0, hi = n_pairs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (offsets[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Batch: per point, its pair's bounding box (ordered ints, as k_fbox) and the
// non-finite flag; aux is n_pairs x 8 ints initialised like k_fbox_init.  A warp
// whose points all belong to one pair reduces first and updates once.
__global__ void __launch_bounds__(kThreads) k_bbox_batch(const float* const* __restrict__ ptrs,
                                                         const int32_t* __restrict__ strides,
                                                         const int64_t* __restrict__ offsets, int n_pairs,
                                                         int64_t total, int* __restrict__ aux) {
  const unsigned full = 0xffffffffu;
  for (int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x; base < total;
       base += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t gi = base + threadIdx.x;
    const bool valid = gi < total;
    const int p = valid ? pair_of(offsets, n_pairs, gi) : -1;
    int mn[3] = {INT_MAX, INT_MAX, INT_MAX}, mx[3] = {INT_MIN, INT_MIN, INT_MIN};
    int bad = 0;
    if (valid) {
      const float* q = ptrs[p] + (gi - offsets[p]) * strides[p];
      const float v[3] = {q[0], q[1], q[2]};
      if (!isfinite(v[0]) || !isfinite(v[1]) || !isfinite(v[2])) {
        bad = 1;
      } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) mn[k] = mx[k] = ordered_int(v[k]);
      }
    }
    const int p0 = __shfl_sync(full, p, 0);
    if (__all_sync(full, p == p0 || p < 0)) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        mn[k] = __reduce_min_sync(full, mn[k]);
        mx[k] = __reduce_max_sync(full, mx[k]);
      }
      bad = __reduce_or_sync(full, bad);
      if ((threadIdx.x & 31) == 0 && p0 >= 0) {
        int* a = aux + 8 * p0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          if (mn[k] != INT_MAX) atomicMin(a + k, mn[k]);
          if (mx[k] != INT_MIN) atomicMax(a + 3 + k, mx[k]);
        }
        if (bad) atomicOr(a + 6, 1);
      }
    } else if (p >= 0) {
      int* a = aux + 8 * p;
      if (bad) {
        atomicOr(a + 6, 1);
      } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          atomicMin(a + k, mn[k]);
          atomicMax(a + 3 + k, mx[k]);
        }
      }
    }
  }
}

__global__ void k_bbox_batch_init(int* aux, int n_pairs) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_pairs; p += gridDim.x * blockDim.x) k_fbox_init_one(aux + 8 * p);
}

// Batch: Morton key of each point over its own pair's box (as k_morton), value = global index.
__global__ void __launch_bounds__(kThreads) k_morton_batch(const float* const* __restrict__ ptrs,
                                                           const int32_t* __restrict__ strides,
                                                           const int64_t* __restrict__ offsets, int n_pairs,
                                                           int total, const int* __restrict__ aux,
                                                           uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= total) return;
  const int p = pair_of(offsets, n_pairs, gi);
  const float* q = ptrs[p] + (gi - offsets[p]) * strides[p];
  keys[gi] = morton_of(q, aux + 8 * p);
  vals[gi] = static_cast<uint32_t>(gi);
}

// Batch: pair id of each (already Morton-sorted) element, for the second stable sort.
__global__ void __launch_bounds__(kThreads) k_pair_keys(const uint32_t* __restrict__ vals,
                                                        const int64_t* __restrict__ offsets, int n_pairs, int total,
                                                        uint32_t* __restrict__ keys) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= total) return;
  keys[k] = static_cast<uint32_t>(pair_of(offsets, n_pairs, vals[k]));
}

// Batch: sorted float4 (x, y, z, index within its pair).
__global__ void __launch_bounds__(kThreads) k_gather4_batch(const float* const* __restrict__ ptrs,
                                                            const int32_t* __restrict__ strides,
                                                            const int64_t* __restrict__ offsets, int n_pairs,
                                                            int total, const uint32_t* __restrict__ perm,
                                                            float4* __restrict__ pts) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= total) return;
  const int gi = static_cast<int>(perm[k]);
  const int p = pair_of(offsets, n_pairs, gi);
  const int local = gi - static_cast<int>(offsets[p]);
  const float* q = ptrs[p] + static_cast<int64_t>(local) * strides[p];
  pts[k] = make_float4(q[0], q[1], q[2], __int_as_float(local));
}

}  // namespace

// All clouds of a batch sorted at once: the concatenation ordered by (pair,
// Morton code over the pair's own box, index) - within each pair exactly the
// order sort_cloud gives that cloud alone (both sorts are stable).  d_ptrs,
// d_strides, d_offsets are device arrays (n_pairs, n_pairs, n_pairs + 1);
// aux receives n_pairs x 8 ints (aux[8p + 6] != 0: non-finite coordinate).
int32_t sort_clouds_batch(const float* const* d_ptrs, const int32_t* d_strides, const int64_t* d_offsets,
                          int n_pairs, int64_t total64, cudaStream_t s, float4* out, int* aux) {
  const int total = static_cast<int>(total64);
  k_bbox_batch_init<<<blocks_for(n_pairs, kThreads), kThreads, 0, s>>>(aux, n_pairs);
  count_launch();
  if (total == 0) return O3G_OK;
  int nb = blocks_for(total, kThreads);
  if (nb > kNumSMs * 8) nb = kNumSMs * 8;
  k_bbox_batch<<<nb, kThreads, 0, s>>>(d_ptrs, d_strides, d_offsets, n_pairs, total, aux);
  DevBuf keys(s), vals(s), tk(s), tv(s);
  O3G_TRY(keys.alloc(sizeof(uint32_t) * total));
  O3G_TRY(vals.alloc(sizeof(uint32_t) * total));
  O3G_TRY(tk.alloc(sizeof(uint32_t) * total));
  O3G_TRY(tv.alloc(sizeof(uint32_t) * total));
  k_morton_batch<<<blocks_for(total, kThreads), kThreads, 0, s>>>(d_ptrs, d_strides, d_offsets, n_pairs, total, aux,
                                                                  keys.as<uint32_t>(), vals.as<uint32_t>());
  count_launch(2);
  O3G_TRY(cudaGetLastError());
  O3G_TRY_STATUS(radix_sort_pairs(keys.as<uint32_t>(), vals.as<uint32_t>(), tk.as<uint32_t>(), tv.as<uint32_t>(),
                                  total, 30, s));
  int pair_bits = 0;
  while ((1 << pair_bits) < n_pairs) ++pair_bits;
  if (pair_bits > 0) {
    k_pair_keys<<<blocks_for(total, kThreads), kThreads, 0, s>>>(vals.as<uint32_t>(), d_offsets, n_pairs, total,
                                                                 keys.as<uint32_t>());
    count_launch();
    O3G_TRY_STATUS(radix_sort_pairs(keys.as<uint32_t>(), vals.as<uint32_t>(), tk.as<uint32_t>(), tv.as<uint32_t>(),
                                    total, pair_bits, s));
  }
  k_gather4_batch<<<blocks_for(total, kThreads), kThreads, 0, s>>>(d_ptrs, d_strides, d_offsets, n_pairs, total,
                                                                   vals.as<uint32_t>(), out);
  count_launch();
  O3G_TRY(cudaGetLastError());
  return O3G_OK;
}

int32_t sort_cloud(const float* d_xyz, int64_t n64, int32_t stride, cudaStream_t s, SortedCloud* out) {
  const int n = static_cast<int>(n64);
  O3G_TRY(out->buf.alloc(sizeof(float4) * (n > 0 ? n : 1)));
  O3G_TRY(out->aux.alloc(8 * sizeof(int)));
  out->pts = out->buf.as<float4>();
  k_fbox_init<<<1, 32, 0, s>>>(out->aux.as<int>());
  count_launch();
  if (n == 0) return O3G_OK;
  int nb = blocks_for(n, kThreads);
  if (nb > kNumSMs * 2) nb = kNumSMs * 2;
  k_fbox<<<nb, kThreads, 0, s>>>(d_xyz, n, stride, out->aux.as<int>());
  DevBuf keys(s), vals(s), tk(s), tv(s);
  O3G_TRY(keys.alloc(sizeof(uint32_t) * n));
  O3G_TRY(vals.alloc(sizeof(uint32_t) * n));
  O3G_TRY(tk.alloc(sizeof(uint32_t) * n));
  O3G_TRY(tv.alloc(sizeof(uint32_t) * n));
  k_morton<<<blocks_for(n, kThreads), kThreads, 0, s>>>(d_xyz, n, stride, out->aux.as<int>(), keys.as<uint32_t>(),
                                                        vals.as<uint32_t>());
  count_launch(2);
  O3G_TRY(cudaGetLastError());
  O3G_TRY_STATUS(radix_sort_pairs(keys.as<uint32_t>(), vals.as<uint32_t>(), tk.as<uint32_t>(), tv.as<uint32_t>(), n,
                                  30, s));
  k_gather4<<<blocks_for(n, kThreads), kThreads, 0, s>>>(d_xyz, n, stride, vals.as<uint32_t>(), out->pts);
  count_launch();
  O3G_TRY(cudaGetLastError());
  return O3G_OK;
}

// Exclusive scan of m uint32 values (in may equal out).
int32_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t m, cudaStream_t s) {
  if (m <= 0) return O3G_OK;
  int nb = blocks_for(m, kScanTile);
  DevBuf bsum(s);
  O3G_TRY(bsum.alloc(sizeof(uint32_t) * nb));
  k_scan_reduce<<<nb, kThreads, 0, s>>>(in, m, bsum.as<uint32_t>());
  k_scan_top<<<1, kThreads, 0, s>>>(bsum.as<uint32_t>(), nb);
  k_scan_down<<<nb, kThreads, 0, s>>>(in, out, m, bsum.as<uint32_t>());
  count_launch(3);
  O3G_TRY(cudaGetLastError());
  return O3G_OK;
}

int rs_tiles(int n) { return blocks_for(n, kRsTile); }
bool rs_inline(int nblk) { return nblk <= kRsInlineBlocks; }

// Stable sort of (keys, vals) by the low `bits` bits of the keys.  The sorted
// pairs end in (keys, vals); tmp_k/tmp_v are scratch of the same size.  With
// hist0 non-null, the first pass's per-tile digit counts are already there
// (256 x rs_tiles(n) entries, tile-major when rs_inline, digit-major
// otherwise) and the buffer serves all passes.
int32_t radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* tmp_k, uint32_t* tmp_v, int n, int bits,
                         cudaStream_t s, uint32_t* hist0) {
  if (n <= 1 || bits <= 0) return O3G_OK;
  const int nblk = rs_tiles(n);
  const bool inl = rs_inline(nblk);
  DevBuf own(s);
  uint32_t* hist = hist0;
  if (!hist) {
    O3G_TRY(own.alloc(sizeof(uint32_t) * 256 * static_cast<size_t>(nblk)));
    hist = own.as<uint32_t>();
  }
  uint32_t *ka = keys, *va = vals, *kb = tmp_k, *vb = tmp_v;
  int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    int shift = 8 * p;
    if (p > 0 || !hist0) {
      if (inl) k_rs_hist<true><<<nblk, kThreads, 0, s>>>(ka, n, shift, hist, nblk);
      else k_rs_hist<false><<<nblk, kThreads, 0, s>>>(ka, n, shift, hist, nblk);
      count_launch();
    }
    if (inl) {
      k_rs_scatter<true><<<nblk, kThreads, 0, s>>>(ka, va, kb, vb, n, shift, hist, nblk);
    } else {
      O3G_TRY_STATUS(exclusive_scan_u32(hist, hist, 256LL * nblk, s));
      k_rs_scatter<false><<<nblk, kThreads, 0, s>>>(ka, va, kb, vb, n, shift, hist, nblk);
    }
    count_launch();
    O3G_TRY(cudaGetLastError());
    uint32_t* t = ka;
    ka = kb;
    kb = t;
    t = va;
    va = vb;
    vb = t;
  }
  if (ka != keys) {
    O3G_TRY(cudaMemcpyAsync(keys, ka, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    O3G_TRY(cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
  }
  return O3G_OK;
}

static void release(o3g_grid* g) {
  dfree(g->pts, g->stream);
  dfree(g->nrm, g->stream);
  dfree(g->cell_start, g->stream);
  dfree(g->pos_of, g->stream);
  dfree(g->col_z, g->stream);
  g->col_z = nullptr;
  g->pts = nullptr;
  g->nrm = nullptr;
  g->cell_start = nullptr;
  g->pos_of = nullptr;
}

static int32_t build_impl(const float* d_xyz, int64_t n64, int stride, float cell, cudaStream_t s, o3g_grid* g) {
  const int n = static_cast<int>(n64);
  g->n = n64;
  g->stream = s;
  if (n == 0) {
    g->cell = cell;
    g->inv_cell = 1.0f / cell;
    g->cells = 1;
    O3G_TRY(dmalloc(reinterpret_cast<void**>(&g->cell_start), 2 * sizeof(uint32_t), s));
    O3G_TRY(cudaMemsetAsync(g->cell_start, 0, 2 * sizeof(uint32_t), s));
    O3G_TRY(dmalloc(reinterpret_cast<void**>(&g->pts), sizeof(float4), s));
    O3G_TRY(dmalloc(reinterpret_cast<void**>(&g->nrm), sizeof(float4), s));
    O3G_TRY(cudaMemsetAsync(g->nrm, 0, sizeof(float4), s));
    O3G_TRY(dmalloc(reinterpret_cast<void**>(&g->pos_of), sizeof(int32_t), s));
    O3G_TRY(dmalloc(reinterpret_cast<void**>(&g->col_z), sizeof(uint32_t), s));
    O3G_TRY(cudaMemsetAsync(g->col_z, 0, sizeof(uint32_t), s));
    k_empty_col<<<1, 1, 0, s>>>(g->col_z);
    count_launch();
    return O3G_OK;
  }
  // 1. bounding box; enlarge the cell while the dense table would be too big.
  DevBuf bb(s);
  O3G_TRY(bb.alloc(16 * sizeof(int)));
  const int64_t cap = std::min<int64_t>(32LL * n + (1LL << 20), (1LL << 31) - 2);
  int h[13];
  int64_t span[3], cells = 0;
  float inv = 0.f;
  for (int attempt = 0;; ++attempt) {
    inv = 1.0f / cell;
    if (!(inv > 0.f) || !std::isfinite(inv)) {
      set_error("o3g_build_grid: cell size %g gives no usable grid", static_cast<double>(cell));
      return O3G_ERR_ARG;
    }
    k_bbox_init<<<1, 32, 0, s>>>(bb.as<int>());
    int nb = blocks_for(n, kThreads);
    if (nb > kNumSMs * 2) nb = kNumSMs * 2;
    k_bbox<<<nb, kThreads, 0, s>>>(d_xyz, n, stride, inv, bb.as<int>());
    count_launch(2);
    O3G_TRY(cudaGetLastError());
    O3G_TRY(cudaMemcpyAsync(h, bb.p, 13 * sizeof(int), cudaMemcpyDeviceToHost, s));
    O3G_TRY(cudaStreamSynchronize(s));
    if (h[6]) {
      set_error("o3g_build_grid: non-finite point coordinate");
      return O3G_ERR_NONFINITE;
    }
    cells = 1;
    for (int a = 0; a < 3; ++a) {
      span[a] = static_cast<int64_t>(h[3 + a]) - h[a] + 1;
      cells *= span[a];
    }
    if (cells <= cap) break;
    if (attempt >= 24) {
      set_error("o3g_build_grid: could not bound the grid size");
      return O3G_ERR_ARG;
    }
    cell = static_cast<float>(cell * std::cbrt(static_cast<double>(cells) / static_cast<double>(cap)) * 1.05);
  }
  g->cell = cell;
  g->inv_cell = inv;
  for (int a = 0; a < 3; ++a) {
    g->lo[a] = h[a];
    g->span[a] = static_cast<int>(span[a]);
    int lo_bits = float_key(h[7 + a]), hi_bits = float_key(h[10 + a]);
    std::memcpy(&g->box_lo[a], &lo_bits, sizeof(float));
    std::memcpy(&g->box_hi[a], &hi_bits, sizeof(float));
  }
  g->cells = cells;

  // 2-3. keys and stable sort
  DevBuf keys(s), vals(s), tk(s), tv(s);
  O3G_TRY(keys.alloc(sizeof(uint32_t) * n));
  O3G_TRY(vals.alloc(sizeof(uint32_t) * n));
  O3G_TRY(tk.alloc(sizeof(uint32_t) * n));
  O3G_TRY(tv.alloc(sizeof(uint32_t) * n));
  const int nblk = rs_tiles(n);
  DevBuf hist(s);
  O3G_TRY(hist.alloc(sizeof(uint32_t) * 256 * static_cast<size_t>(nblk)));
  const uint32_t sy = static_cast<uint32_t>(span[1]), sz = static_cast<uint32_t>(span[2]);
  if (rs_inline(nblk))
    k_keys_hist<true><<<nblk, kThreads, 0, s>>>(d_xyz, n, stride, inv, h[0], h[1], h[2], sy, sz, keys.as<uint32_t>(),
                                                vals.as<uint32_t>(), hist.as<uint32_t>(), nblk);
  else
    k_keys_hist<false><<<nblk, kThreads, 0, s>>>(d_xyz, n, stride, inv, h[0], h[1], h[2], sy, sz, keys.as<uint32_t>(),
                                                 vals.as<uint32_t>(), hist.as<uint32_t>(), nblk);
  count_launch();
  O3G_TRY(cudaGetLastError());
  int bits = 0;
  while (bits < 32 && (static_cast<uint64_t>(cells - 1) >> bits) != 0) ++bits;
  O3G_TRY_STATUS(radix_sort_pairs(keys.as<uint32_t>(), vals.as<uint32_t>(), tk.as<uint32_t>(), tv.as<uint32_t>(), n,
                                  bits, s, hist.as<uint32_t>()));

  // 4-5. cell table and sorted points
  O3G_TRY(dmalloc(reinterpret_cast<void**>(&g->cell_start), sizeof(uint32_t) * (cells + 1), s));
  O3G_TRY(dmalloc(reinterpret_cast<void**>(&g->pts), sizeof(float4) * n, s));
  O3G_TRY(dmalloc(reinterpret_cast<void**>(&g->nrm), sizeof(float4) * (n + 1), s));
  O3G_TRY(dmalloc(reinterpret_cast<void**>(&g->pos_of), sizeof(int32_t) * n, s));
  const bool chunked = cells + 1 > kChunkedMinCells;
  int nbc = blocks_for(cells + 1, chunked ? kThreads * kCellsPerThread : kThreads);
  if (nbc > kNumSMs * 16) nbc = kNumSMs * 16;
  if (chunked) k_cell_start<<<nbc, kThreads, 0, s>>>(keys.as<uint32_t>(), n, g->cell_start, cells);
  else k_cell_start_direct<<<nbc, kThreads, 0, s>>>(keys.as<uint32_t>(), n, g->cell_start, cells);
  const int ncol = g->span[0] * g->span[1];
  O3G_TRY(dmalloc(reinterpret_cast<void**>(&g->col_z), sizeof(uint32_t) * ncol, s));
  int nbz = blocks_for(ncol, kThreads);
  if (nbz > kNumSMs * 16) nbz = kNumSMs * 16;
  k_col_extent_gather<<<nbz + blocks_for(n, kThreads), kThreads, 0, s>>>(
      g->cell_start, ncol, g->span[2], g->col_z, nbz, d_xyz, n, stride, vals.as<uint32_t>(), g->pts, g->pos_of,
      g->nrm);
  count_launch(2);
  O3G_TRY(cudaGetLastError());
  return O3G_OK;
}

}  // namespace o3g

using namespace o3g;

extern "C" int32_t o3g_build_grid(const float* d_xyz, int64_t n, int32_t stride, float cell_size, void* stream,
                                  o3g_grid** out) {
  if (!out) {
    set_error("o3g_build_grid: out is null");
    return O3G_ERR_ARG;
  }
  *out = nullptr;
  if (n < 0 || n > INT32_MAX - kRsTile || (n > 0 && !d_xyz) || stride < 3 || !(cell_size > 0.f) ||
      !std::isfinite(cell_size)) {
    set_error("o3g_build_grid: invalid argument (n=%lld stride=%d cell=%g)", static_cast<long long>(n), stride,
              static_cast<double>(cell_size));
    return O3G_ERR_ARG;
  }
  o3g_grid* g = new (std::nothrow) o3g_grid();
  if (!g) {
    set_error("o3g_build_grid: host allocation failed");
    return O3G_ERR_OOM;
  }
  int32_t st;
  {
    TimedRegion tr(O3G_KERNEL_GRID, static_cast<cudaStream_t>(stream));
    st = build_impl(d_xyz, n, stride, cell_size, static_cast<cudaStream_t>(stream), g);
  }
  if (st < 0) {
    release(g);
    delete g;
    return st;
  }
  *out = g;
  return O3G_OK;
}

extern "C" int32_t o3g_free_grid(o3g_grid* g) {
  if (!g) return O3G_OK;
  release(g);
  delete g;
  return O3G_OK;
}

extern "C" int32_t o3g_grid_info(const o3g_grid* g, int64_t* n, float* cell_size) {
  if (!g) {
    set_error("o3g_grid_info: grid is null");
    return O3G_ERR_ARG;
  }
  if (n) *n = g->n;
  if (cell_size) *cell_size = g->cell;
  return O3G_OK;
}

extern "C" int32_t o3g_grid_set_normals(o3g_grid* g, const float* d_nrm, int64_t n, int32_t stride, void* stream) {
  if (!g || (n > 0 && !d_nrm) || stride < 3) {
    set_error("o3g_grid_set_normals: invalid argument");
    return O3G_ERR_ARG;
  }
  if (n != g->n) {
    set_error("o3g_grid_set_normals: %lld normals for %lld points (normals must match the points one to one)",
              static_cast<long long>(n), static_cast<long long>(g->n));
    return O3G_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n > 0) {
    O3G_TRY(cudaMemsetAsync(g->nrm + n, 0, sizeof(float4), s));
    k_set_normals<<<blocks_for(n, kThreads), kThreads, 0, s>>>(d_nrm, stride, g->pts, static_cast<int>(n), g->nrm);
    count_launch();
    O3G_TRY(cudaGetLastError());
  }
  g->has_normals = true;
  return O3G_OK;
}
