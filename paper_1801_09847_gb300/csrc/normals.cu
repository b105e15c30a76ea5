// Hybrid kNN search and normal estimation on the GPU:
// estimate_normals(pc, KDTreeSearchParamHybrid(radius, max_nn)) of the Open3D
// paper (Fig. 1, Sec. 3.3), parallel across data samples (Sec. 4).
//
// Per point: the at most max_nn grid points with float32 d2 <= fl(radius)^2,
// smallest first in (d2, original index) order; the covariance of that
// neighbourhood about its mean (float32, offsets taken from the query point
// first); its smallest-eigenvalue eigenvector; orientation toward the
// viewpoint.  max_nn <= 32 (the paper's 30 included) runs one warp per point:
// coalesced candidate loads, the box's column runs found by all lanes at once,
// an exact selection through a histogram of d2, and a closed-form eigenvector.
// Larger max_nn runs one thread per point with an insertion-sorted list in
// local memory and cyclic Jacobi rotations.
#include <cmath>

#include <vector>

#include "o3g_internal.cuh"

namespace o3g {

namespace {

constexpr int kThreads = 128;

// Inserts the grid points within r of q into keys/pos (ascending 64-bit keys
// (d2 bits << 32 | original index)); returns how many were kept (<= max_nn).
template <int KMAX>
__device__ int knn_select(const GridView& g, float qx, float qy, float qz, float r, int max_nn, uint64_t* keys,
                          int* pos) {
  const float r2 = __fmul_rn(r, r);
  int ax, bx, ay, by, az, bz;
  axis_range(qx, r, g.inv_cell, g.lo_x, g.sx, ax, bx);
  axis_range(qy, r, g.inv_cell, g.lo_y, g.sy, ay, by);
  axis_range(qz, r, g.inv_cell, g.lo_z, g.sz, az, bz);
  int m = 0;
  if (az > bz) return 0;
  for (int x = ax; x <= bx; ++x) {
    for (int y = ay; y <= by; ++y) {
      int zl = az, zh = bz;
      if (!column_z(g, x * g.sy + y, zl, zh)) continue;
      const int col = (x * g.sy + y) * g.sz;
      const uint32_t beg = g.cell_start[col + zl], end = g.cell_start[col + zh + 1];
      for (uint32_t k = beg; k < end; ++k) {
        const float4 q = g.pts[k];
        const float d2 = dist2_rn(qx, qy, qz, q);
        if (!(d2 <= r2)) continue;
        const uint64_t key = (static_cast<uint64_t>(__float_as_uint(d2)) << 32) |
                             static_cast<uint32_t>(__float_as_int(q.w));
        if (m == max_nn && key >= keys[m - 1]) continue;
        int j = m < max_nn ? m++ : m - 1;
        while (j > 0 && keys[j - 1] > key) {
          keys[j] = keys[j - 1];
          pos[j] = pos[j - 1];
          --j;
        }
        keys[j] = key;
        pos[j] = static_cast<int>(k);
      }
    }
  }
  return m;
}

// One Jacobi rotation in the (p, q) plane of the symmetric a (row-major 3x3),
// accumulated into V, chosen so that the new a_pq is zero.
template <int P, int Q>
__device__ __forceinline__ void jacobi_rotate(float a[3][3], float V[3][3]) {
  const float apq = a[P][Q];
  if (apq == 0.f) return;
  const float theta = (a[Q][Q] - a[P][P]) / (2.f * apq);
  const float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
  const float c = rsqrtf(t * t + 1.f);
  const float s = t * c;
  constexpr int R = 3 - P - Q;
  const float arp = a[R][P], arq = a[R][Q];
  a[P][P] -= t * apq;
  a[Q][Q] += t * apq;
  a[P][Q] = a[Q][P] = 0.f;
  a[R][P] = a[P][R] = c * arp - s * arq;
  a[R][Q] = a[Q][R] = s * arp + c * arq;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float vp = V[k][P], vq = V[k][Q];
    V[k][P] = c * vp - s * vq;
    V[k][Q] = s * vp + c * vq;
  }
}

// Unit eigenvector of the smallest eigenvalue of the symmetric a.
__device__ float3 smallest_eigvec(float a[3][3]) {
  float V[3][3] = {{1.f, 0.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 0.f, 1.f}};
  for (int sweep = 0; sweep < 10; ++sweep) {
    const float off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    const float dg = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
    if (!(off > 1e-14f * dg)) break;
    jacobi_rotate<0, 1>(a, V);
    jacobi_rotate<0, 2>(a, V);
    jacobi_rotate<1, 2>(a, V);
  }
  int k = 0;
  if (a[1][1] < a[k][k]) k = 1;
  if (a[2][2] < a[k][k]) k = 2;
  float3 n = make_float3(V[0][k], V[1][k], V[2][k]);
  const float inv = rsqrtf(n.x * n.x + n.y * n.y + n.z * n.z);
  n.x *= inv;
  n.y *= inv;
  n.z *= inv;
  return n;
}

// Unit eigenvector of the smallest eigenvalue of the symmetric a, closed form:
// the eigenvalues of a 3x3 symmetric matrix from its characteristic cubic in
// trigonometric form (lambda = m + 2 s cos(phi + 2 pi k / 3) with m = tr/3,
// s^2 = |a - m I|_F^2 / 6, cos(3 phi) = det((a - m I) / s) / 2), then the null
// vector of a - lambda_min I as the largest cross product of two of its rows.
// When the smallest eigenvalue is (nearly) repeated, any unit vector orthogonal
// to the remaining direction is a smallest eigenvector; one such is returned.
__device__ float3 smallest_eigvec_closed(const float a[3][3]) {
  const float m = (a[0][0] + a[1][1] + a[2][2]) * (1.f / 3.f);
  const float b00 = a[0][0] - m, b11 = a[1][1] - m, b22 = a[2][2] - m;
  const float b01 = a[0][1], b02 = a[0][2], b12 = a[1][2];
  const float off = b01 * b01 + b02 * b02 + b12 * b12;
  const float s2 = (b00 * b00 + b11 * b11 + b22 * b22 + 2.f * off) * (1.f / 6.f);
  if (!(s2 > 0.f)) return make_float3(0.f, 0.f, 1.f);  // a = m I: every direction is an eigenvector
  const float s = sqrtf(s2);
  const float is = 1.f / s;
  const float c00 = b00 * is, c11 = b11 * is, c22 = b22 * is, c01 = b01 * is, c02 = b02 * is, c12 = b12 * is;
  const float det = c00 * (c11 * c22 - c12 * c12) - c01 * (c01 * c22 - c12 * c02) + c02 * (c01 * c12 - c11 * c02);
  const float h = fminf(fmaxf(0.5f * det, -1.f), 1.f);
  const float phi = acosf(h) * (1.f / 3.f);
  const float lmin = m + 2.f * s * cosf(phi + 2.0943951023931957f);  // + 2 pi / 3: the smallest root
  const float3 r0 = make_float3(a[0][0] - lmin, a[0][1], a[0][2]);
  const float3 r1 = make_float3(a[1][0], a[1][1] - lmin, a[1][2]);
  const float3 r2 = make_float3(a[2][0], a[2][1], a[2][2] - lmin);
  auto cross = [](float3 u, float3 v) {
    return make_float3(u.y * v.z - u.z * v.y, u.z * v.x - u.x * v.z, u.x * v.y - u.y * v.x);
  };
  auto dot = [](float3 u, float3 v) { return u.x * v.x + u.y * v.y + u.z * v.z; };
  const float3 x01 = cross(r0, r1), x02 = cross(r0, r2), x12 = cross(r1, r2);
  const float d01 = dot(x01, x01), d02 = dot(x02, x02), d12 = dot(x12, x12);
  float3 n = x01;
  float dn = d01;
  if (d02 > dn) { n = x02; dn = d02; }
  if (d12 > dn) { n = x12; dn = d12; }
  const float rr = fmaxf(fmaxf(dot(r0, r0), dot(r1, r1)), dot(r2, r2));
  if (!(dn > 1e-12f * rr * rr)) {
    // rank <= 1: take the largest row and any direction orthogonal to it
    float3 r = r0;
    if (dot(r1, r1) > dot(r, r)) r = r1;
    if (dot(r2, r2) > dot(r, r)) r = r2;
    const float ax = fabsf(r.x), ay = fabsf(r.y), az = fabsf(r.z);
    const float3 e = (ax <= ay && ax <= az) ? make_float3(1.f, 0.f, 0.f)
                     : (ay <= az)           ? make_float3(0.f, 1.f, 0.f)
                                            : make_float3(0.f, 0.f, 1.f);
    n = cross(r, e);
    dn = dot(n, n);
    if (!(dn > 0.f)) return make_float3(0.f, 0.f, 1.f);
  }
  const float inv = rsqrtf(dn);
  return make_float3(n.x * inv, n.y * inv, n.z * inv);
}

// ---------------------------------------------------------------------------
// Warp-cooperative hybrid search (max_nn <= 32): one warp per query.  Lanes
// load consecutive points of a cell column (coalesced) and append the keys of
// those within the radius to the warp's buffer in shared memory; keys are
// (d2 bits << 32 | original index), so their order is (d2, index) and the
// result is the exact set the definition gives.  The max_nn smallest are then
// selected in two steps: a histogram of d2 finds the bin that holds the
// max_nn-th smallest key, and only the keys up to that bin (typically max_nn to
// max_nn + 2) are kept.  kNN queries sort them (one bitonic network across the
// lanes); normals need only the set, so they rank just the few keys of that
// last bin.  A buffer that fills up is cut down to its max_nn smallest keys the
// same way, and from then on only keys below the max_nn-th are appended.
constexpr uint64_t kNoKey = ~0ull;
constexpr int kStageCap = 256;  // keys buffered per warp
constexpr int kBins = 128;      // histogram bins of the selection, four per lane

struct alignas(16) WarpStage {
  uint64_t key[kStageCap];
  uint32_t hist[kBins];
};

__device__ __forceinline__ uint64_t shfl_xor64(uint64_t v, int m) {
  return __shfl_xor_sync(0xffffffffu, v, m);
}

// Ascending bitonic sort of one key per lane.
__device__ __forceinline__ uint64_t warp_sort32(uint64_t v, int lane) {
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const uint64_t o = shfl_xor64(v, j);
      const bool up = (lane & k) == 0;
      const bool low = (lane & j) == 0;
      v = (low == up) ? (v < o ? v : o) : (v < o ? o : v);
    }
  }
  return v;
}

// list (ascending) <- the 32 smallest of list and batch (ascending).
__device__ __forceinline__ uint64_t warp_merge32(uint64_t list, uint64_t batch, int lane) {
  const uint64_t rev = __shfl_sync(0xffffffffu, batch, 31 - lane);
  uint64_t v = list < rev ? list : rev;  // bitonic
#pragma unroll
  for (int j = 16; j > 0; j >>= 1) {
    const uint64_t o = shfl_xor64(v, j);
    v = ((lane & j) == 0) ? (v < o ? v : o) : (v < o ? o : v);
  }
  return v;
}

__device__ __forceinline__ float key_d2(uint64_t key) {
  return __uint_as_float(static_cast<uint32_t>(key >> 32));
}

// Histogram bin of a key: non-decreasing in the key (a correctly rounded
// product of non-negative floats, truncated and clamped, keeps their order).
__device__ __forceinline__ int key_bin(uint64_t key, float scale) {
  return min(static_cast<int>(__fmul_rn(key_d2(key), scale)), kBins - 1);
}

// The k (<= 32) smallest of the m keys s.key[0, m), ascending, lane j holding
// the j-th (kNoKey past the end); every key has d2 <= hi.  With more than 32
// keys, a histogram of d2 over [0, hi] gives the bin b of the k-th smallest;
// since bins follow the key order, the k smallest are among the keys of bins
// <= b, which are moved to the front of the buffer.  While more than 32 remain,
// the same is repeated over the range of those bins (a few rounds at most),
// then the rest is sorted.  Should more than 32 keys still be left (ties), they
// are sorted and merged 32 at a time.  Any scale gives non-decreasing bins, so
// the range only decides how fast the keys thin out.  With ordered false the
// result may instead be the same set unsorted: lanes below m hold the selected
// keys or kNoKey, in buffer order.  All lanes must call this.
__device__ uint64_t warp_select(WarpStage& s, int m, int k, float hi, int lane, bool ordered = true) {
  const unsigned full = 0xffffffffu;
  __syncwarp();
  float scale = __fdiv_rn(static_cast<float>(kBins), hi);
  int last_b = -1;
  uint32_t last_nb = 0;
  float last_scale = 0.f;
  for (int round = 0; m > 32 && round < 3 && scale <= 3.0e38f; ++round) {  // hi = 0: no histogram
    reinterpret_cast<uint4*>(s.hist)[lane] = make_uint4(0u, 0u, 0u, 0u);
    __syncwarp();
    for (int i = lane; i < m; i += 32) atomicAdd(&s.hist[key_bin(s.key[i], scale)], 1u);
    __syncwarp();
    const uint4 c = reinterpret_cast<const uint4*>(s.hist)[lane];
    const uint32_t own = c.x + c.y + c.z + c.w;
    uint32_t incl = own;  // keys in the bins of lanes 0..lane
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(full, incl, o);
      if (lane >= o) incl += v;
    }
    const uint32_t uk = static_cast<uint32_t>(k);
    const int src = __ffs(__ballot_sync(full, incl >= uk)) - 1;  // incl of lane 31 is m > k
    const uint32_t e0 = incl - own + c.x, e1 = e0 + c.y, e2 = e1 + c.z;
    const int sub = e0 >= uk ? 0 : e1 >= uk ? 1 : e2 >= uk ? 2 : 3;
    const int b = 4 * src + __shfl_sync(full, sub, src);
    last_nb = __shfl_sync(full, sub == 0 ? c.x : sub == 1 ? c.y : sub == 2 ? c.z : c.w, src);
    last_b = b;
    last_scale = scale;
    int w = 0;
    for (int base = 0; base < m; base += 32) {  // in place: writes stay below base + 32
      const int i = base + lane;
      const uint64_t key = i < m ? s.key[i] : kNoKey;
      const bool sel = i < m && key_bin(key, scale) <= b;
      const uint32_t mask = __ballot_sync(full, sel);
      if (sel) s.key[w + __popc(mask & ((1u << lane) - 1u))] = key;
      w += __popc(mask);
    }
    __syncwarp();
    m = w;
    if (b == kBins - 1) break;  // nothing was dropped, and the range would not narrow
    scale = __fmul_rn(scale, __fdiv_rn(static_cast<float>(kBins), static_cast<float>(b + 1)));
  }
  if (!ordered && last_b >= 0 && m <= 32) {
    // the keys of bins below last_b are all in; of the last_nb keys in bin
    // last_b, the (k - those below) smallest, by their rank within the bin
    const uint64_t v = lane < m ? s.key[lane] : kNoKey;
    const bool inb = lane < m && key_bin(v, last_scale) == last_b;
    const uint32_t need = static_cast<uint32_t>(k) - (static_cast<uint32_t>(m) - last_nb);
    bool keep = lane < m;
    if (last_nb > need) {
      uint32_t mb = __ballot_sync(full, inb), rank = 0;
      while (mb) {
        const int j = __ffs(mb) - 1;
        mb &= mb - 1u;
        const uint64_t o = __shfl_sync(full, v, j);
        rank += o < v ? 1u : 0u;
      }
      keep = keep && (!inb || rank < need);
    }
    return keep ? v : kNoKey;
  }
  if (m <= 32) {
    const uint64_t v = warp_sort32(lane < m ? s.key[lane] : kNoKey, lane);
    return lane < k ? v : kNoKey;
  }
  uint64_t list = kNoKey;
  for (int base = 0; base < m; base += 32) {
    const uint64_t v = warp_sort32(base + lane < m ? s.key[base + lane] : kNoKey, lane);
    list = warp_merge32(list, v, lane);
  }
  return lane < k ? list : kNoKey;
}

// Returns lane `lane`'s entry of the <= max_nn nearest keys: lane j holds the
// j-th when ordered, otherwise the set sits on some lanes (kNoKey on the rest).
__device__ uint64_t warp_knn(const GridView& g, float qx, float qy, float qz, float r, int max_nn, WarpStage& s,
                             bool ordered = true) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  const float r2 = __fmul_rn(r, r);
  int ax, bx, ay, by, az, bz;
  axis_range(qx, r, g.inv_cell, g.lo_x, g.sx, ax, bx);
  axis_range(qy, r, g.inv_cell, g.lo_y, g.sy, ay, by);
  axis_range(qz, r, g.inv_cell, g.lo_z, g.sz, az, bz);
  if (ax > bx || ay > by || az > bz) return kNoKey;
  uint64_t thr = kNoKey;  // once the buffer was cut down: its max_nn-th key (keys must be < thr to matter)
  float hi = r2;          // every buffered key has d2 <= hi
  int m = 0;              // keys in the buffer
  // The box's (x, y) columns, 32 at a time: lane c finds the run of sorted
  // points of column c over the z-range the radius allows there (the ball's
  // extent above the column's nearest point, with the exact search's rounding
  // margins; a column the ball misses has none), two loads for all columns at
  // once, then the warp scans the runs one after another.
  const float margin = search_margin(g.cell, r, qx, qy, qz);
  const uint32_t ny = by - ay + 1, ncols = (bx - ax + 1) * ny;  // <= the grid's cells < 2^31
  for (uint32_t c0 = 0; c0 < ncols; c0 += 32) {
    uint32_t rb = 0, re = 0;
    const uint32_t c = c0 + lane;
    if (c < ncols) {
      const int x = ax + static_cast<int>(c / ny), y = ay + static_cast<int>(c % ny);
      const float gx = slab_gap(qx, x + g.lo_x, g.cell, margin), gy = slab_gap(qy, y + g.lo_y, g.cell, margin);
      const float lim = __fmul_rn(r2, 1.0001f) - (gx * gx + gy * gy);
      int zl = 1, zh = 0;
      if (lim >= 0.f) {
        const float rz = __fadd_rn(fast_sqrt(lim), margin);
        zl = max(az, cell_coord(__fsub_rn(qz, rz), g.inv_cell) - g.lo_z);
        zh = min(bz, cell_coord(__fadd_rn(qz, rz), g.inv_cell) - g.lo_z);
      }
      if (zl <= zh && column_z(g, x * g.sy + y, zl, zh)) {
        const int col = (x * g.sy + y) * g.sz;
        rb = g.cell_start[col + zl];
        re = g.cell_start[col + zh + 1];
      }
    }
    uint32_t runs = __ballot_sync(0xffffffffu, rb < re);
    while (runs) {
      const int src = __ffs(runs) - 1;
      runs &= runs - 1u;
      const uint32_t beg = __shfl_sync(0xffffffffu, rb, src), end = __shfl_sync(0xffffffffu, re, src);
      for (uint32_t k0 = beg; k0 < end; k0 += 32) {
        const uint32_t k = k0 + lane;
        uint64_t key = kNoKey;
        if (k < end) {
          const float4 q = g.pts[k];
          const float d2 = dist2_rn(qx, qy, qz, q);
          if (d2 <= r2)
            key = (static_cast<uint64_t>(__float_as_uint(d2)) << 32) | static_cast<uint32_t>(__float_as_int(q.w));
        }
        bool keep = key < thr;
        uint32_t mask = __ballot_sync(0xffffffffu, keep);
        if (mask == 0u) continue;
        if (m + __popc(mask) > kStageCap) {  // m > kStageCap - 32 >= max_nn: the cut keeps max_nn keys
          const uint64_t v = warp_select(s, m, max_nn, hi, lane);
          __syncwarp();
          if (lane < max_nn) s.key[lane] = v;
          m = max_nn;
          thr = __shfl_sync(0xffffffffu, v, max_nn - 1);
          hi = key_d2(thr);
          keep = key < thr;
          mask = __ballot_sync(0xffffffffu, keep);
        }
        if (keep) s.key[m + __popc(mask & lt)] = key;
        m += __popc(mask);
      }
    }
  }
  return warp_select(s, m, max_nn, hi, lane, ordered);
}

constexpr int kWarpsPerBlock = kThreads / 32;

// Warp-sum of a float (fixed shuffle tree; every lane gets the total).
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Normal of sorted point k of grid g, computed by one whole warp (stage: that
// warp's key buffer).  The sums run over the lanes in a fixed order, so the
// result depends only on the grid and the point.  Lane 0 stores it.
__device__ void warp_normal(const GridView& g, const int32_t* __restrict__ pos_of, int k, float radius, int max_nn,
                            float vx, float vy, float vz, float4* __restrict__ nrm_sorted, float* __restrict__ out,
                            int out_stride, WarpStage& stage) {
  const int lane = threadIdx.x & 31;
  const float4 q = g.pts[k];
  const uint64_t key = warp_knn(g, q.x, q.y, q.z, radius, max_nn, stage, false);
  const bool have = key != kNoKey;
  const int m = __popc(__ballot_sync(0xffffffffu, have));
  float3 n = make_float3(0.f, 0.f, 1.f);
  if (m >= 3) {
    float ox = 0.f, oy = 0.f, oz = 0.f;
    if (have) {
      const float4 p = g.pts[pos_of[static_cast<uint32_t>(key & 0xffffffffu)]];
      ox = p.x - q.x;
      oy = p.y - q.y;
      oz = p.z - q.z;
    }
    const float inv_m = 1.f / static_cast<float>(m);
    const float mx = warp_sum(ox) * inv_m, my = warp_sum(oy) * inv_m, mz = warp_sum(oz) * inv_m;
    const float dx = have ? ox - mx : 0.f, dy = have ? oy - my : 0.f, dz = have ? oz - mz : 0.f;
    float a[3][3];
    a[0][0] = warp_sum(dx * dx) * inv_m;
    a[0][1] = a[1][0] = warp_sum(dx * dy) * inv_m;
    a[0][2] = a[2][0] = warp_sum(dx * dz) * inv_m;
    a[1][1] = warp_sum(dy * dy) * inv_m;
    a[1][2] = a[2][1] = warp_sum(dy * dz) * inv_m;
    a[2][2] = warp_sum(dz * dz) * inv_m;
    if (lane != 0) return;
    n = smallest_eigvec_closed(a);
    const float facing = n.x * (vx - q.x) + n.y * (vy - q.y) + n.z * (vz - q.z);
    if (facing < 0.f) {
      n.x = -n.x;
      n.y = -n.y;
      n.z = -n.z;
    }
  } else if (lane != 0) {
    return;
  }
  nrm_sorted[k] = make_float4(n.x, n.y, n.z, 0.f);
  if (out) {
    float* o = out + static_cast<int64_t>(__float_as_int(q.w)) * out_stride;
    o[0] = n.x;
    o[1] = n.y;
    o[2] = n.z;
  }
}

__global__ void __launch_bounds__(kThreads, 10) k_normals_warp(GridView g, const int32_t* __restrict__ pos_of,
                                                           float radius, int max_nn, float vx, float vy, float vz,
                                                           float4* __restrict__ nrm_sorted, float* __restrict__ out,
                                                           int out_stride) {
  __shared__ WarpStage stage_all[kWarpsPerBlock];
  const int warp = threadIdx.x >> 5;
  const int k = blockIdx.x * kWarpsPerBlock + warp;
  if (k == 0 && threadIdx.x == 0) nrm_sorted[g.n] = make_float4(1.f, 0.f, 0.f, 0.f);  // length bound: unit normals
  if (k >= g.n) return;
  warp_normal(g, pos_of, k, radius, max_nn, vx, vy, vz, nrm_sorted, out, out_stride, stage_all[warp]);
}

// One cloud of a batched normals or kNN launch.
struct NormalsJob {
  GridView g;
  const int32_t* pos_of;
  float4* nrm_sorted;
  float* out;        // normals: by original index, or null;  kNN: unused
  const float* qry;  // kNN: query rows (stride floats each)
  int32_t* idx;      // kNN outputs
  float* dd;
  int32_t* cnt;
  int n;             // points (normals) or queries (kNN)
  int stride;        // out stride (normals) or query stride (kNN)
  float radius, vx, vy, vz;
};

// Job of global warp w: the last job whose first warp is <= w (binary search
// over the jobs' first warps, ascending).
__device__ __forceinline__ int job_of(const int64_t* __restrict__ first, int njobs, int64_t w) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= w) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Normals of many clouds in one launch: warp w takes point w - first[j] of
// job j, so every point gets exactly the computation the one-cloud launch gives it.
__global__ void __launch_bounds__(kThreads, 9) k_normals_batch(const NormalsJob* __restrict__ jobs,
                                                            const int64_t* __restrict__ first, int njobs,
                                                            int64_t total, int max_nn) {
  __shared__ WarpStage stage_all[kWarpsPerBlock];
  const int warp = threadIdx.x >> 5;
  const int64_t w = static_cast<int64_t>(blockIdx.x) * kWarpsPerBlock + warp;
  if (w >= total) return;
  const int j = job_of(first, njobs, w);
  const NormalsJob& J = jobs[j];
  const int k = static_cast<int>(w - first[j]);
  if (k >= J.n) return;
  if (k == 0 && (threadIdx.x & 31) == 0) J.nrm_sorted[J.n] = make_float4(1.f, 0.f, 0.f, 0.f);  // length bound
  warp_normal(J.g, J.pos_of, k, J.radius, max_nn, J.vx, J.vy, J.vz, J.nrm_sorted, J.out, J.stride,
              stage_all[warp]);
}

// Hybrid kNN of query i, computed by one whole warp.
__device__ void warp_query(const GridView& g, const float* __restrict__ qry, int i, int stride, float radius,
                           int max_nn, int32_t* __restrict__ idx, float* __restrict__ dd, int32_t* __restrict__ cnt,
                           WarpStage& stage) {
  const int lane = threadIdx.x & 31;
  const float* q = qry + static_cast<int64_t>(i) * stride;
  const uint64_t key = warp_knn(g, q[0], q[1], q[2], radius, max_nn, stage);
  const bool have = key != kNoKey;
  const int m = __popc(__ballot_sync(0xffffffffu, have));
  if (lane < max_nn) {
    idx[static_cast<int64_t>(i) * max_nn + lane] = have ? static_cast<int32_t>(key & 0xffffffffu) : -1;
    dd[static_cast<int64_t>(i) * max_nn + lane] = have ? __uint_as_float(static_cast<uint32_t>(key >> 32)) : 0.f;
  }
  if (lane == 0) cnt[i] = m;
}

__global__ void __launch_bounds__(kThreads) k_knn_warp(GridView g, const float* __restrict__ qry, int nq, int stride,
                                                       float radius, int max_nn, int32_t* __restrict__ idx,
                                                       float* __restrict__ dd, int32_t* __restrict__ cnt) {
  __shared__ WarpStage stage_all[kWarpsPerBlock];
  const int warp = threadIdx.x >> 5;
  const int i = blockIdx.x * kWarpsPerBlock + warp;
  if (i >= nq) return;
  warp_query(g, qry, i, stride, radius, max_nn, idx, dd, cnt, stage_all[warp]);
}

// Hybrid kNN queries against many grids in one launch (warp w: query
// w - first[j] of job j).
__global__ void __launch_bounds__(kThreads) k_knn_batch(const NormalsJob* __restrict__ jobs,
                                                        const int64_t* __restrict__ first, int njobs, int64_t total,
                                                        int max_nn) {
  __shared__ WarpStage stage_all[kWarpsPerBlock];
  const int warp = threadIdx.x >> 5;
  const int64_t w = static_cast<int64_t>(blockIdx.x) * kWarpsPerBlock + warp;
  if (w >= total) return;
  const int j = job_of(first, njobs, w);
  const NormalsJob& J = jobs[j];
  const int i = static_cast<int>(w - first[j]);
  if (i >= J.n) return;
  warp_query(J.g, J.qry, i, J.stride, J.radius, max_nn, J.idx, J.dd, J.cnt, stage_all[warp]);
}

template <int KMAX>
__global__ void __launch_bounds__(kThreads) k_normals(GridView g, float radius, int max_nn, float vx, float vy,
                                                      float vz, float4* __restrict__ nrm_sorted,
                                                      float* __restrict__ out, int out_stride) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) nrm_sorted[g.n] = make_float4(1.f, 0.f, 0.f, 0.f);  // length bound: unit normals
  if (k >= g.n) return;
  uint64_t keys[KMAX];
  int pos[KMAX];
  const float4 q = g.pts[k];
  const int m = knn_select<KMAX>(g, q.x, q.y, q.z, radius, max_nn, keys, pos);
  float3 n = make_float3(0.f, 0.f, 1.f);
  if (m >= 3) {
    float sx = 0.f, sy = 0.f, sz = 0.f;
    for (int j = 0; j < m; ++j) {
      const float4 p = g.pts[pos[j]];
      sx += p.x - q.x;
      sy += p.y - q.y;
      sz += p.z - q.z;
    }
    const float inv_m = 1.f / static_cast<float>(m);
    const float mx = sx * inv_m, my = sy * inv_m, mz = sz * inv_m;
    float c00 = 0.f, c01 = 0.f, c02 = 0.f, c11 = 0.f, c12 = 0.f, c22 = 0.f;
    for (int j = 0; j < m; ++j) {
      const float4 p = g.pts[pos[j]];
      const float dx = (p.x - q.x) - mx, dy = (p.y - q.y) - my, dz = (p.z - q.z) - mz;
      c00 += dx * dx;
      c01 += dx * dy;
      c02 += dx * dz;
      c11 += dy * dy;
      c12 += dy * dz;
      c22 += dz * dz;
    }
    float a[3][3] = {{c00 * inv_m, c01 * inv_m, c02 * inv_m},
                     {c01 * inv_m, c11 * inv_m, c12 * inv_m},
                     {c02 * inv_m, c12 * inv_m, c22 * inv_m}};
    n = smallest_eigvec(a);
    const float facing = n.x * (vx - q.x) + n.y * (vy - q.y) + n.z * (vz - q.z);
    if (facing < 0.f) {
      n.x = -n.x;
      n.y = -n.y;
      n.z = -n.z;
    }
  }
  nrm_sorted[k] = make_float4(n.x, n.y, n.z, 0.f);
  if (out) {
    float* o = out + static_cast<int64_t>(__float_as_int(q.w)) * out_stride;
    o[0] = n.x;
    o[1] = n.y;
    o[2] = n.z;
  }
}

template <int KMAX>
__global__ void __launch_bounds__(kThreads) k_knn(GridView g, const float* __restrict__ qry, int nq, int stride,
                                                  float radius, int max_nn, int32_t* __restrict__ idx,
                                                  float* __restrict__ dd, int32_t* __restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  uint64_t keys[KMAX];
  int pos[KMAX];
  const float* q = qry + static_cast<int64_t>(i) * stride;
  const int m = knn_select<KMAX>(g, q[0], q[1], q[2], radius, max_nn, keys, pos);
  int32_t* oi = idx + static_cast<int64_t>(i) * max_nn;
  float* od = dd + static_cast<int64_t>(i) * max_nn;
  for (int j = 0; j < max_nn; ++j) {
    oi[j] = j < m ? static_cast<int32_t>(keys[j] & 0xffffffffu) : -1;
    od[j] = j < m ? __uint_as_float(static_cast<uint32_t>(keys[j] >> 32)) : 0.f;
  }
  cnt[i] = m;
}

int blocks_for(int64_t n) {
  int64_t b = (n + kThreads - 1) / kThreads;
  return static_cast<int>(b < 1 ? 1 : b);
}

int warp_blocks(int64_t n) {
  int64_t b = (n + kWarpsPerBlock - 1) / kWarpsPerBlock;
  return static_cast<int>(b < 1 ? 1 : b);
}

}  // namespace

int32_t estimate_normals_impl(o3g_grid* g, float radius, int32_t max_nn, const float* viewpoint, float* d_out,
                              int32_t out_stride, cudaStream_t s) {
  const char* fn = "o3g_estimate_normals";
  if (!g || !(radius >= 0.f) || !std::isfinite(radius) || max_nn < 1 || max_nn > O3G_MAX_NN ||
      (d_out && out_stride < 3)) {
    set_error("%s: invalid argument", fn);
    return O3G_ERR_ARG;
  }
  float v[3] = {0.f, 0.f, 0.f};
  if (viewpoint)
    for (int a = 0; a < 3; ++a) v[a] = viewpoint[a];
  if (!std::isfinite(v[0]) || !std::isfinite(v[1]) || !std::isfinite(v[2])) {
    set_error("%s: viewpoint is not finite", fn);
    return O3G_ERR_NONFINITE;
  }
  if (g->n > 0) {
    const GridView gv = g->view();
    TimedRegion tr(O3G_KERNEL_NORMALS, s);
    count_launch();
    if (max_nn <= 32)
      k_normals_warp<<<warp_blocks(g->n), kThreads, 0, s>>>(gv, g->pos_of, radius, max_nn, v[0], v[1], v[2], g->nrm,
                                                            d_out, out_stride);
    else
      k_normals<O3G_MAX_NN><<<blocks_for(g->n), kThreads, 0, s>>>(gv, radius, max_nn, v[0], v[1], v[2], g->nrm,
                                                                  d_out, out_stride);
    O3G_TRY(cudaGetLastError());
  }
  g->has_normals = true;
  return O3G_OK;
}

}  // namespace o3g

using namespace o3g;

extern "C" int32_t o3g_estimate_normals(o3g_grid* g, float radius, int32_t max_nn, const float* viewpoint,
                                        float* d_nrm_out, int32_t nrm_stride, void* stream) {
  return estimate_normals_impl(g, radius, max_nn, viewpoint, d_nrm_out, nrm_stride, static_cast<cudaStream_t>(stream));
}

extern "C" int32_t o3g_knn_hybrid(const o3g_grid* g, const float* d_qry, int64_t nq, int32_t stride, float radius,
                                  int32_t max_nn, int32_t* d_idx, float* d_d2, int32_t* d_cnt, void* stream) {
  if (!g || nq < 0 || nq > 0x7fffffffLL - kThreads || (nq > 0 && (!d_qry || !d_idx || !d_d2 || !d_cnt)) ||
      stride < 3 || !(radius >= 0.f) || !std::isfinite(radius) || max_nn < 1 || max_nn > O3G_MAX_NN) {
    set_error("o3g_knn_hybrid: invalid argument");
    return O3G_ERR_ARG;
  }
  if (nq == 0) return O3G_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const GridView gv = g->view();
  count_launch();
  if (max_nn <= 32)
    k_knn_warp<<<warp_blocks(nq), kThreads, 0, s>>>(gv, d_qry, static_cast<int>(nq), stride, radius, max_nn, d_idx,
                                                    d_d2, d_cnt);
  else
    k_knn<O3G_MAX_NN><<<blocks_for(nq), kThreads, 0, s>>>(gv, d_qry, static_cast<int>(nq), stride, radius, max_nn,
                                                          d_idx, d_d2, d_cnt);
  O3G_TRY(cudaGetLastError());
  return O3G_OK;
}

namespace {

// Launches one batched warp kernel over the jobs (first warp of each job from
// their sizes), synchronously on s.
template <class Launch>
int32_t run_jobs(std::vector<NormalsJob>& jobs, int max_nn, cudaStream_t s, Launch launch) {
  std::vector<int64_t> first(jobs.size());
  int64_t total = 0;
  for (size_t j = 0; j < jobs.size(); ++j) {
    first[j] = total;
    total += jobs[j].n;
  }
  if (total == 0) return O3G_OK;
  DevBuf d_jobs(s), d_first(s);
  O3G_TRY(d_jobs.alloc(sizeof(NormalsJob) * jobs.size()));
  O3G_TRY(d_first.alloc(sizeof(int64_t) * first.size()));
  O3G_TRY(cudaMemcpyAsync(d_jobs.p, jobs.data(), sizeof(NormalsJob) * jobs.size(), cudaMemcpyHostToDevice, s));
  O3G_TRY(cudaMemcpyAsync(d_first.p, first.data(), sizeof(int64_t) * first.size(), cudaMemcpyHostToDevice, s));
  launch(d_jobs.as<NormalsJob>(), d_first.as<int64_t>(), static_cast<int>(jobs.size()), total,
         warp_blocks(total));
  count_launch();
  O3G_TRY(cudaGetLastError());
  O3G_TRY(cudaStreamSynchronize(s));
  return O3G_OK;
}

}  // namespace

extern "C" int32_t o3g_estimate_normals_batch(int32_t n_grids, o3g_grid* const* grids, const float* radius,
                                              int32_t max_nn, const float* viewpoints, float* const* d_out,
                                              const int32_t* out_strides, void* stream) {
  const char* fn = "o3g_estimate_normals_batch";
  if (n_grids < 0 || (n_grids > 0 && (!grids || !radius)) || max_nn < 1 || max_nn > O3G_MAX_NN) {
    set_error("%s: invalid argument", fn);
    return O3G_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<NormalsJob> jobs(static_cast<size_t>(n_grids));
  for (int c = 0; c < n_grids; ++c) {
    const int stride = out_strides ? out_strides[c] : 3;
    if (!grids[c] || !(radius[c] >= 0.f) || !std::isfinite(radius[c]) || (d_out && d_out[c] && stride < 3)) {
      set_error("%s: invalid grid, radius or output stride for cloud %d", fn, c);
      return O3G_ERR_ARG;
    }
    const float* v = viewpoints ? viewpoints + 3 * c : nullptr;
    if (v && !(std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]))) {
      set_error("%s: viewpoint %d is not finite", fn, c);
      return O3G_ERR_NONFINITE;
    }
    NormalsJob& J = jobs[c];
    J = NormalsJob{};
    J.g = grids[c]->view();
    J.pos_of = grids[c]->pos_of;
    J.nrm_sorted = grids[c]->nrm;
    J.out = d_out ? d_out[c] : nullptr;
    J.n = static_cast<int>(grids[c]->n);
    J.stride = stride;
    J.radius = radius[c];
    J.vx = v ? v[0] : 0.f;
    J.vy = v ? v[1] : 0.f;
    J.vz = v ? v[2] : 0.f;
  }
  if (max_nn > 32) {  // the thread-per-point form, one launch per cloud
    for (int c = 0; c < n_grids; ++c)
      O3G_TRY_STATUS(estimate_normals_impl(grids[c], radius[c], max_nn, viewpoints ? viewpoints + 3 * c : nullptr,
                                           jobs[c].out, jobs[c].stride, s));
    O3G_TRY(cudaStreamSynchronize(s));
    return O3G_OK;
  }
  {
    TimedRegion tr(O3G_KERNEL_NORMALS, s);
    O3G_TRY_STATUS(run_jobs(jobs, max_nn, s, [&](const NormalsJob* dj, const int64_t* df, int nj, int64_t total,
                                                 int blocks) {
      k_normals_batch<<<blocks, kThreads, 0, s>>>(dj, df, nj, total, max_nn);
    }));
  }
  for (int c = 0; c < n_grids; ++c) grids[c]->has_normals = true;
  return O3G_OK;
}

extern "C" int32_t o3g_knn_hybrid_batch(int32_t n_grids, const o3g_grid* const* grids, const float* const* d_qry,
                                        const int64_t* nq, const int32_t* strides, const float* radius,
                                        int32_t max_nn, int32_t* const* d_idx, float* const* d_d2,
                                        int32_t* const* d_cnt, void* stream) {
  const char* fn = "o3g_knn_hybrid_batch";
  if (n_grids < 0 || (n_grids > 0 && (!grids || !d_qry || !nq || !strides || !radius || !d_idx || !d_d2 || !d_cnt)) ||
      max_nn < 1 || max_nn > O3G_MAX_NN) {
    set_error("%s: invalid argument", fn);
    return O3G_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<NormalsJob> jobs(static_cast<size_t>(n_grids));
  for (int c = 0; c < n_grids; ++c) {
    if (!grids[c] || nq[c] < 0 || nq[c] > 0x7fffffffLL - kThreads ||
        (nq[c] > 0 && (!d_qry[c] || !d_idx[c] || !d_d2[c] || !d_cnt[c])) || strides[c] < 3 || !(radius[c] >= 0.f) ||
        !std::isfinite(radius[c])) {
      set_error("%s: invalid arguments for query set %d", fn, c);
      return O3G_ERR_ARG;
    }
    NormalsJob& J = jobs[c];
    J = NormalsJob{};
    J.g = grids[c]->view();
    J.qry = d_qry[c];
    J.idx = d_idx[c];
    J.dd = d_d2[c];
    J.cnt = d_cnt[c];
    J.n = static_cast<int>(nq[c]);
    J.stride = strides[c];
    J.radius = radius[c];
  }
  if (max_nn > 32) {
    for (int c = 0; c < n_grids; ++c)
      O3G_TRY_STATUS(o3g_knn_hybrid(grids[c], d_qry[c], nq[c], strides[c], radius[c], max_nn, d_idx[c], d_d2[c],
                                    d_cnt[c], stream));
    O3G_TRY(cudaStreamSynchronize(s));
    return O3G_OK;
  }
  return run_jobs(jobs, max_nn, s, [&](const NormalsJob* dj, const int64_t* df, int nj, int64_t total, int blocks) {
    k_knn_batch<<<blocks, kThreads, 0, s>>>(dj, df, nj, total, max_nn);
  });
}
