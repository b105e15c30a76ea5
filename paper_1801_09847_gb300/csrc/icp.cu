// Point-to-plane ICP on the GPU: registration_icp(source, target,
// max_correspondence_distance, init, TransformationEstimationPointToPlane())
// of the Open3D paper (Sec. 3.3), as the Gauss-Newton iteration of Sec. 4,
// Eq. (1)-(2).  One kernel launch per iteration, k_icp_iter:
//   1. transform the (cell-sorted) source point, float32, fixed rounding order;
//   2. fixed-radius nearest neighbour over the target grid (exact: every
//      pruning bound carries a margin for float32 rounding, and ties are kept,
//      so the result is the minimum of (d2, original index)).  A point's
//      candidate list from an earlier iteration decides it alone while the list
//      still covers it (see ListSink); otherwise the search starts from the
//      last matches of the point and its warp neighbours and scans every cell
//      column whose slab can still hold a point within the bound, over the
//      z-range that bound allows (staged block-wide in shared memory in the
//      latency form, per thread from global memory in the throughput form);
//   3. r = (p - q) . n, J = [p x n ; n]; the 21 upper entries of J^T J, J^T r,
//      r^2, d2 and |C| as exact (value, error) pairs, summed over the tile's
//      rows in a fixed order into one compensated float32 pair per sum, which
//      is added as a 64-bit fixed-point integer (exact, order-free) to the
//      pair's accumulators;
//   4. the last tile to finish (atomic arrival counter, no waiting) converts the
//      totals to float64, solves (J^T J) xi = -J^T r with the frozen-pivot
//      rule (the pivots of LDL^T), and updates T <- [Rz Ry Rx(xi), t] T on the
//      device.  The next launch reads the new pose.
// The pose never leaves the device between iterations.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "o3g_internal.cuh"

namespace o3g {

namespace {

constexpr int kThreads = 128;
constexpr int kPartial = 32;  // sum columns of a block partial (column kBadCol: see add_fixed)
constexpr int kAccRows = 32;  // fixed-point accumulator rows of a pair (its tiles spread over them)
constexpr int kBadCol = 31;   // accumulator column counting partials outside their bound

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
  int lists_on;    // candidate lists are kept (the updates have become small; see ListSink)
  int phase;       // served pairs (mode kServe): 0 iterating, 1 evaluation next, 2 evaluated
  int cap;         // served pairs: the iteration limit
  unsigned arrived;  // tiles of the current launch whose sums are added
  double A[36];
  double b[6];
  double stats[3];  // sum r^2, sum d2, |C|
  double fitness, rmse;
};

// kServe: every pair advances by one stage of its own phase (see IcpState):
// an iteration, or the final evaluation after the last one.
enum Mode : int { kIterate = 0, kEquations = 1, kEvaluate = 2, kCorrOnly = 3, kServe = 4 };

// Which transformation estimate an iteration makes (Sec. 3.3).
enum Kind : int { kPointToPlane = 0, kPointToPoint = 1 };

// cap: the iteration limit a served pair stops at (its evaluation comes next at once when 0).
__global__ void k_init_state(IcpState* st, Pose T, int cap = 0x7fffffff) {
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
  st->lists_on = 0;
  st->phase = cap > 0 ? 0 : 1;
  st->cap = cap;
  st->arrived = 0u;
  st->fitness = 0.0;
  st->rmse = 0.0;
}


// Pose j of poses (n x 16 float64) into state j, as k_init_state.
__global__ void k_init_states(IcpState* st, const double* __restrict__ poses, int n) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const double* T = poses + 16 * j;
    IcpState& S = st[j];
    for (int k = 0; k < 16; ++k) S.T[k] = T[k];
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) S.R[3 * r + c] = __double2float_rn(T[4 * r + c]);
      S.t[r] = __double2float_rn(T[4 * r + 3]);
    }
    S.iters = 0;
    S.done = 0;
    S.degenerate = 0;
    S.few_corr = 0;
    S.nonfinite = 0;
    S.lists_on = 0;
    S.phase = 0;
    S.cap = 0x7fffffff;
    S.arrived = 0u;
    S.fitness = 0.0;
    S.rmse = 0.0;
  }
}


// Running fixed-radius nearest neighbour of one query: the minimum of
// (d2, original index) among the candidates seen so far with d2 <= r2.
struct Nearest {
  float d2;
  int orig;
  int pos;  // sorted target position, -1 if none
};

__device__ __forceinline__ void consider_d2(Nearest& nb, float d2, int orig, int pos) {
  if (d2 < nb.d2 || (d2 == nb.d2 && orig < nb.orig)) {
    nb.d2 = d2;
    nb.orig = orig;
    nb.pos = pos;
  }
}

__device__ __forceinline__ void consider(Nearest& nb, float4 q, int pos, float px, float py, float pz) {
  consider_d2(nb, dist2_rn(px, py, pz, q), __float_as_int(q.w), pos);
}

// Where the exact searches put their candidates.  NnSink keeps the nearest
// neighbour; its pruning bound is the best d2 so far.
struct NnSink {
  Nearest nb;
  __device__ __forceinline__ float bound() const { return nb.d2; }
  __device__ __forceinline__ bool seeded() const { return nb.pos >= 0; }
  __device__ __forceinline__ void offer(float4 q, int pos, float px, float py, float pz) {
    consider(nb, q, pos, px, py, pz);
  }
};

// Candidate lists.  While ICP iterates, each source point keeps a list of the
// targets near the place p_b where the list was built: every target within
// d1 + sigma of p_b (d1: the distance to its nearest target within r, or r
// when there is none; sigma = kSkin r), at most kList of them (the nearest),
// with a bound rho2 such that every target at dist2_rn(p_b, q) < rho2 is
// listed (a Verlet neighbour list with skin sigma, as molecular dynamics keeps
// them).  At a later position p with d = |p - p_b|: a target at d2 <= D from p
// lies within sqrt(D) + d of p_b, so when (sqrt(D) + d)^2, with margins for the
// float32 rounding of the three distances, is below rho2, every candidate of
// the exact search is listed and the list alone decides the correspondence
// (D = the best listed d2 within r2, or r2 when none is, which proves that no
// target is within r).  A list stays valid while its point moves less than
// about sigma; a point whose list no longer covers it searches the grid and
// rebuilds its list.
constexpr int kList = 8;
constexpr int kListVec = kList / 4;  // int4 words of one point's list
constexpr float kSkin = 0.1f;

// The bound a list rebuilt at p takes its candidates within: (sqrt(D) + sigma)^2,
// rounded up, for the best d2 D known when the rebuild starts (the nearest
// listed target of the old list within r2, else r2).
__device__ __forceinline__ float list_lim(float D, float sigma) {
  const float s = __fadd_rn(fast_sqrt(__fmul_rn(D, 1.0001f)), sigma);
  return __fmul_rn(__fmul_rn(s, s), 1.0001f);
}

// A list being rebuilt at p, with the nearest neighbour within r2 beside it:
// the kList nearest candidates by (d2, position) among those at d2 <= lim.
// While fewer are held every candidate within lim is taken; once kList are
// held, a nearer one replaces the farthest (and the pruning bound becomes the
// farthest held d2).  Every target left out is then at d2 >= the farthest held
// d2, so every target at d2 < rho2() is held.  The list depends only on the
// targets, p and lim, not on the order the search offers candidates in.
// Entries sit in shared-memory columns (entry k of thread t at [k][t]).
struct ListSink {
  Nearest nb;
  float (*d)[kThreads];
  int (*p)[kThreads];
  float lim;
  int m;       // entries held
  float maxv;  // m == kList: the farthest held (d2, position) is (maxv, p[maxk])
  int maxk;
  __device__ __forceinline__ float bound() const { return m < kList ? lim : maxv; }
  __device__ __forceinline__ bool seeded() const { return nb.pos >= 0; }
  __device__ __forceinline__ void rescan() {
    const int t = threadIdx.x;
    maxv = d[0][t];
    maxk = 0;
#pragma unroll
    for (int k = 1; k < kList; ++k)
      if (d[k][t] > maxv || (d[k][t] == maxv && p[k][t] > p[maxk][t])) {
        maxv = d[k][t];
        maxk = k;
      }
  }
  __device__ __forceinline__ void offer(float4 q, int pos, float px, float py, float pz) {
    const float v = dist2_rn(px, py, pz, q);
    consider_d2(nb, v, __float_as_int(q.w), pos);
    if (!(v <= lim)) return;
    const int t = threadIdx.x;
    if (m < kList) {
      d[m][t] = v;
      p[m][t] = pos;
      if (++m == kList) rescan();
    } else if (v < maxv || (v == maxv && pos < p[maxk][t])) {
      d[maxk][t] = v;
      p[maxk][t] = pos;
      rescan();
    }
  }
  // every target at d2 < rho2 from the build position is held
  __device__ __forceinline__ float rho2() const { return m < kList ? lim : maxv; }
};

// The state of one source point's list: (p_b, rho2), its kList entries (sorted
// target positions, -1: empty) ordered by (d2 from p_b, position), and for
// entries 1 .. kList-1 a code c_k with c_k sigma / kGapScale <= (distance of
// entry k from p_b) - (distance of entry 0 from p_b), saturating at 255.
// rho2 NaN (the initial all-ones bytes): no list.
struct ListRef {
  float4* pb;  // per source point
  int4* idx;   // kListVec per source point
  uint2* gap;  // per source point: c_1..c_4 in the bytes of .x, c_5..c_7 in .y
  int* hint;   // per source point: sorted target position of its last match, or -1
};
constexpr float kGapScale = 127.5f;  // codes in units of sigma / 127.5: 255 = two skins
// bytes per source point, a multiple of 16 (buffers of many pairs stay aligned)
constexpr size_t kListBytes = (sizeof(float4) * (1 + kListVec) + sizeof(uint2) + sizeof(int) + 15) / 16 * 16;

// Candidate lists pay where an iteration launch is bound by throughput rather
// than by the latency of one wave of tiles: a pair keeps them when it has at
// least kListMinPoints source points, once an update moves its points by less
// than a quarter of the skin.
constexpr int64_t kListMinPoints = 1 << 17;
inline float list_motion(int64_t ns, float r) { return ns >= kListMinPoints ? 0.25f * kSkin * r : -1.f; }

// The lists of n source points in one buffer of kListBytes * n bytes (all
// bytes 0xff at the start: no lists, no matches).
inline ListRef list_ref(void* base, int64_t n) {
  float4* pb = static_cast<float4*>(base);
  int4* idx = reinterpret_cast<int4*>(pb + n);
  uint2* gap = reinterpret_cast<uint2*>(idx + kListVec * n);
  return ListRef{pb, idx, gap, reinterpret_cast<int*>(gap + n)};
}

// Scans a query's list at its position p: the nearest listed target within r2
// goes into nb (a first bound for a rebuild), and the result says whether the
// list covers the query (see above).  With d = |p - p_b|, entry k lies at least
// (its distance from p_b) - d from p, and entry 0 at most (its distance) + d;
// so an entry whose code puts it farther from p_b than entry 0 by more than
// 2 d (plus a relative margin of 2e-4 of a bound on both distances, which keeps
// its float32 d2 strictly above entry 0's) can neither win nor tie, and is not
// loaded.  Entries 0-3 are scanned in every warp, 4-7 only in a warp where
// some lane needs one of them.  All lanes of the warp must call this (a lane
// without a list has only empty entries).
__device__ __forceinline__ bool list_scan(const GridView& g, float4 pb, const int4 (&l)[kListVec], uint2 gap,
                                          float sigma, float px, float py, float pz, Nearest& nb) {
  int e[kList];
#pragma unroll
  for (int k = 0; k < kListVec; ++k) {
    e[4 * k] = l[k].x;
    e[4 * k + 1] = l[k].y;
    e[4 * k + 2] = l[k].z;
    e[4 * k + 3] = l[k].w;
  }
  const float moved = dist2_rn(px, py, pz, pb);  // NaN without a list
  const float dm = fast_sqrt(__fmul_rn(moved, 1.0001f));
  const float thr = __fmul_rn(__fadd_rn(__fmul_rn(2.f, dm), __fmul_rn(2e-4f, __fadd_rn(fast_sqrt(__fmul_rn(pb.w, 1.0001f)), dm))),
                              1.0001f);
  const float unit = __fmul_rn(sigma, 1.f / kGapScale);
  unsigned need = e[0] >= 0 ? 1u : 0u;
#pragma unroll
  for (int k = 1; k < kList; ++k) {
    const unsigned c = ((k <= 4 ? gap.x : gap.y) >> (8 * ((k - 1) & 3))) & 0xffu;
    if (e[k] >= 0 && !(__fmul_rn(static_cast<float>(c), unit) > thr)) need |= 1u << k;
  }
  const unsigned any = __reduce_or_sync(0xffffffffu, need);
  {
    float4 q[kList / 2];
#pragma unroll
    for (int k = 0; k < kList / 2; ++k) q[k] = ((need >> k) & 1u) ? g.pts[e[k]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < kList / 2; ++k)
      if ((need >> k) & 1u) consider(nb, q[k], e[k], px, py, pz);
  }
  if (any >> (kList / 2)) {
    float4 q[kList / 2];
#pragma unroll
    for (int k = kList / 2; k < kList; ++k)
      q[k - kList / 2] = ((need >> k) & 1u) ? g.pts[e[k]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = kList / 2; k < kList; ++k)
      if ((need >> k) & 1u) consider(nb, q[k - kList / 2], e[k], px, py, pz);
  }
  const float s = __fadd_rn(fast_sqrt(__fmul_rn(nb.d2, 1.0001f)), dm);
  return __fadd_rn(__fmul_rn(__fmul_rn(s, s), 1.0001f), 1e-30f) < pb.w;
}

// Stores a rebuilt list of thread threadIdx.x for source point i: its entries
// sorted by (d2, position) (a 19-comparator merging network; empty entries
// last) and the gap codes of entries 1.. against entry 0, each rounded down
// from a lower bound on the true difference of the distances (relative
// margins of 1e-4 cover the float32 d2 and square roots).
__device__ __forceinline__ void list_store(const ListRef& L, int i, const ListSink& ls, float px, float py,
                                           float pz, float sigma) {
  float d[kList];
  int e[kList];
#pragma unroll
  for (int k = 0; k < kList; ++k) {
    d[k] = k < ls.m ? ls.d[k][threadIdx.x] : __int_as_float(0x7f800000);
    e[k] = k < ls.m ? ls.p[k][threadIdx.x] : 0x7fffffff;
  }
  constexpr int kNet[19][2] = {{0, 1}, {2, 3}, {4, 5}, {6, 7}, {0, 2}, {1, 3}, {4, 6}, {5, 7}, {1, 2}, {5, 6},
                               {0, 4}, {1, 5}, {2, 6}, {3, 7}, {2, 4}, {3, 5}, {1, 2}, {3, 4}, {5, 6}};
#pragma unroll
  for (int c = 0; c < 19; ++c) {
    const int a = kNet[c][0], b = kNet[c][1];
    if (d[a] > d[b] || (d[a] == d[b] && e[a] > e[b])) {
      const float td = d[a];
      d[a] = d[b];
      d[b] = td;
      const int te = e[a];
      e[a] = e[b];
      e[b] = te;
    }
  }
  const float r0 = fast_sqrt(__fmul_rn(d[0], 1.0002f));
  const float inv = __fdiv_rn(kGapScale, sigma);
  unsigned code[kList];
#pragma unroll
  for (int k = 1; k < kList; ++k) {
    const float gk = __fsub_rn(fast_sqrt(__fmul_rn(d[k], 0.9998f)), r0);
    const float c = __fmul_rn(__fmul_rn(gk, inv), 0.9999f);
    code[k] = k < ls.m && c > 0.f ? (c >= 255.f ? 255u : static_cast<unsigned>(c)) : 0u;
  }
#pragma unroll
  for (int k = 0; k < kList; ++k)
    if (k >= ls.m) e[k] = -1;
  __stcs(&L.pb[i], make_float4(px, py, pz, ls.rho2()));
#pragma unroll
  for (int k = 0; k < kListVec; ++k)
    __stcs(&L.idx[kListVec * i + k], make_int4(e[4 * k], e[4 * k + 1], e[4 * k + 2], e[4 * k + 3]));
  __stcs(&L.gap[i], make_uint2(code[1] | (code[2] << 8) | (code[3] << 16) | (code[4] << 24),
                               code[5] | (code[6] << 8) | (code[7] << 16)));
}

// Offers the sorted target positions [beg, end) to a sink in order.
template <class Sink>
__device__ __forceinline__ void offer_run(const GridView& g, uint32_t beg, uint32_t end, float px, float py, float pz,
                                          Sink& sk) {
#pragma unroll 4
  for (uint32_t j = beg; j < end; ++j) sk.offer(g.pts[j], static_cast<int>(j), px, py, pz);
}

// Candidates that give a first bound: this point's match in the previous
// iteration (`hint`, a sorted target position or -1) and those of its
// neighbours in the spatially sorted warp.  Each is an ordinary candidate, so it
// only tightens the bound, never changes the answer.  All lanes must call this.
__device__ __forceinline__ void first_bound(const GridView& g, float px, float py, float pz, int hint, Nearest& nb) {
  const unsigned full = 0xffffffffu;
  const int h[5] = {hint, __shfl_xor_sync(full, hint, 1), __shfl_xor_sync(full, hint, 2),
                    __shfl_xor_sync(full, hint, 3), __shfl_xor_sync(full, hint, 4)};
  float4 q[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) q[k] = h[k] >= 0 ? g.pts[h[k]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 5; ++k)
    if (h[k] >= 0) consider(nb, q[k], h[k], px, py, pz);
}

// The exact search from global memory: the home cell first when the sink has no
// bound yet, then every cell that can still hold a candidate within the sink's
// bound (box sized from the bound; each column over the z-range the bound
// allows; empty cells add nothing to a run, so the columns' occupied extents
// are not looked up: one dependent load fewer per column).  Every bound carries a
// margin for float32 rounding and ties are kept, so the nearest neighbour is
// exactly the brute-force minimum and a list holds exactly the nearest.
// R: the largest radius the sink asks for (its margins are sized by it).
template <class Sink>
__device__ void box_search_global(const GridView& g, float cell, float px, float py, float pz, float R, Sink& sk) {
  const float margin = search_margin(cell, R, px, py, pz);
  const int hx = cell_coord(px, g.inv_cell) - g.lo_x;
  const int hy = cell_coord(py, g.inv_cell) - g.lo_y;
  const int hz = cell_coord(pz, g.inv_cell) - g.lo_z;
  const bool home_in = hx >= 0 && hx < g.sx && hy >= 0 && hy < g.sy && hz >= 0 && hz < g.sz;
  bool home_done = false;
  if (!sk.seeded() && home_in) {
    const int c = (hx * g.sy + hy) * g.sz + hz;
    offer_run(g, g.cell_start[c], g.cell_start[c + 1], px, py, pz, sk);
    home_done = true;
  }
  const float reach = __fadd_rn(fast_sqrt(__fmul_rn(sk.bound(), 1.0001f)), margin);
  int ax, bx, ay, by, az, bz;
  axis_range(px, reach, g.inv_cell, g.lo_x, g.sx, ax, bx);
  axis_range(py, reach, g.inv_cell, g.lo_y, g.sy, ay, by);
  axis_range(pz, reach, g.inv_cell, g.lo_z, g.sz, az, bz);
  if (ax > bx || ay > by || az > bz) return;
  for (int x = ax; x <= bx; ++x) {
    const float gx = slab_gap(px, x + g.lo_x, cell, margin);
    for (int y = ay; y <= by; ++y) {
      const float gy = slab_gap(py, y + g.lo_y, cell, margin);
      const float lim = __fmul_rn(sk.bound(), 1.0001f) - (gx * gx + gy * gy);
      if (lim < 0.f) continue;
      const float rz = __fadd_rn(fast_sqrt(lim), margin);
      int zl = max(az, cell_coord(__fsub_rn(pz, rz), g.inv_cell) - g.lo_z);
      int zh = min(bz, cell_coord(__fadd_rn(pz, rz), g.inv_cell) - g.lo_z);
      if (zl > zh) continue;
      const int col = (x * g.sy + y) * g.sz;
      const uint32_t b0 = g.cell_start[col + zl], e1 = g.cell_start[col + zh + 1];
      if (home_done && x == hx && y == hy && zl <= hz && hz <= zh) {
        offer_run(g, b0, g.cell_start[col + hz], px, py, pz, sk);
        offer_run(g, g.cell_start[col + hz + 1], e1, px, py, pz, sk);
      } else {
        offer_run(g, b0, e1, px, py, pz, sk);
      }
    }
  }
}

// Block-wide search with the candidate cells staged in shared memory.  The
// block's queries are consecutive in Morton order, so the boxes their bounds
// allow overlap.  The block takes the bounding box of those boxes, and for each
// of its (x, y) columns the union of the z-ranges its threads will scan there;
// if that fits, it loads those columns' cell offsets (one round trip), copies
// every point of those z-ranges into shared memory (one warp per column,
// coalesced), and then each thread scans exactly its own cells there.  This
// replaces each thread's chain of dependent global loads with two block-wide
// round trips, and stages only cells some thread needs.  Returns false, with
// nothing changed, when the staged set does not fit: the caller then searches
// from global memory.  All threads of the block must call this.
constexpr int kStageZ = 15;  // z-cells per column

// The launch configurations.  Latency: every tile of a launch is resident at
// once (5 blocks per SM), and a large block stage keeps the searches off the
// slower chains of dependent global loads.  Throughput: more tiles than
// resident blocks; every search runs per thread from global memory (the
// latency of its dependent loads is hidden by 9 resident blocks per SM, with
// registers budgeted for them, and the block-wide staging's planning, copies
// and barriers are saved), and the stage only holds the rows of the reduction
// and the lists being rebuilt.  On the 2M-point fragment pair this measured
// 7.93 against 8.41 ms per registration, on the 256-pair batch 39.0 against
// 47.2 ms per call; on the one-wave RGB-D pair the latency form stays faster.
// Pose evaluation keeps a staged form for its many launches of cold searches.
struct CfgLatency {
  static constexpr int kPts = 1792, kCols = 128, kMinBlocks = 5;
  static constexpr bool kLists = false;  // one wave of tiles: lists do not pay (see kListMinPoints)
  static constexpr bool kStaged = true;
};
struct CfgThroughput {
  static constexpr int kPts = 640, kCols = 32, kMinBlocks = 9;
  static constexpr bool kLists = true;
  static constexpr bool kStaged = false;
};
struct CfgEval {
  static constexpr int kPts = 1024, kCols = 64, kMinBlocks = 7;
  static constexpr bool kLists = false;
  static constexpr bool kStaged = true;
};

// The lists being rebuilt in a tile (see ListSink) take the last kListPts
// points of the stage (a staged search then holds kListPts fewer candidates).
constexpr int kListPts = kList * kThreads * 2 * 4 / 16;

template <class Cfg>
struct Stage {
  static constexpr int kStagePts = Cfg::kPts, kStageCols = Cfg::kCols;
  static constexpr bool kLists = Cfg::kLists, kStaged = Cfg::kStaged;
  static_assert(!kLists || kStagePts >= kListPts, "the stage holds the lists being rebuilt");
  float4 pts[kStagePts];
  uint32_t off[kStageCols][kStageZ + 1];  // global cell_start of each z-cell of each column
  uint32_t base[kStageCols + 1];          // staged position of each column's first staged point
  int zlo[kStageCols], zhi[kStageCols];   // union of the threads' z-ranges per column (box-relative)
  int box[6];
  int total;
};

// The z-range [zl, zh] (grid-relative) a query at p must scan in column
// (x, y) for its current bound, or zl > zh when the column cannot hold a
// candidate.  The same expression serves the planning and the scan; the scan
// clamps its range to the planned one (see staged_search).
__device__ __forceinline__ void column_range(const GridView& g, float cell, float px, float py, float pz,
                                             float margin, float bound, int x, int y, int az, int bz, int& zl,
                                             int& zh) {
  const float gx = slab_gap(px, x + g.lo_x, cell, margin);
  const float gy = slab_gap(py, y + g.lo_y, cell, margin);
  const float lim = __fmul_rn(bound, 1.0001f) - (gx * gx + gy * gy);
  if (lim < 0.f) {
    zl = 1;
    zh = 0;
    return;
  }
  const float rz = __fadd_rn(fast_sqrt(lim), margin);
  zl = max(az, cell_coord(__fsub_rn(pz, rz), g.inv_cell) - g.lo_z);
  zh = min(bz, cell_coord(__fadd_rn(pz, rz), g.inv_cell) - g.lo_z);
}

template <class St, class Sink>
__device__ bool staged_search(const GridView& g, float cell, float px, float py, float pz, float r, bool live,
                              Sink& sk, St& S, int cap = St::kStagePts) {
  constexpr int kStageCols = St::kStageCols;
  const float margin = search_margin(cell, r, px, py, pz);
  const float reach = __fadd_rn(fast_sqrt(__fmul_rn(sk.bound(), 1.0001f)), margin);
  int ax = 0, bx = -1, ay = 0, by = -1, az = 0, bz = -1;
  if (live) {
    axis_range(px, reach, g.inv_cell, g.lo_x, g.sx, ax, bx);
    axis_range(py, reach, g.inv_cell, g.lo_y, g.sy, ay, by);
    axis_range(pz, reach, g.inv_cell, g.lo_z, g.sz, az, bz);
  }
  const bool any = ax <= bx && ay <= by && az <= bz;
  const unsigned full = 0xffffffffu;
  if (threadIdx.x < 3) S.box[threadIdx.x] = 0x7fffffff;
  else if (threadIdx.x < 6) S.box[threadIdx.x] = -1;
  __syncthreads();
  {
    const int lx = __reduce_min_sync(full, any ? ax : 0x7fffffff), ly = __reduce_min_sync(full, any ? ay : 0x7fffffff);
    const int lz = __reduce_min_sync(full, any ? az : 0x7fffffff);
    const int ux = __reduce_max_sync(full, any ? bx : -1), uy = __reduce_max_sync(full, any ? by : -1);
    const int uz = __reduce_max_sync(full, any ? bz : -1);
    if ((threadIdx.x & 31) == 0 && ux >= 0) {
      atomicMin(&S.box[0], lx);
      atomicMin(&S.box[1], ly);
      atomicMin(&S.box[2], lz);
      atomicMax(&S.box[3], ux);
      atomicMax(&S.box[4], uy);
      atomicMax(&S.box[5], uz);
    }
  }
  __syncthreads();
  const int AX = S.box[0], AY = S.box[1], AZ = S.box[2], BX = S.box[3], BY = S.box[4], BZ = S.box[5];
  if (BX < 0) return true;  // no query of the block can have a candidate
  const int NCY = BY - AY + 1, NCZ = BZ - AZ + 1;
  const int ncol = (BX - AX + 1) * NCY;
  if (ncol > kStageCols || NCZ > kStageZ) return false;
  // the union of the z-ranges each thread will scan, per column
  for (int t = threadIdx.x; t < ncol; t += blockDim.x) {
    S.zlo[t] = 0x7fffffff;
    S.zhi[t] = -1;
  }
  __syncthreads();
  if (any) {
    for (int x = ax; x <= bx; ++x)
      for (int y = ay; y <= by; ++y) {
        int zl, zh;
        column_range(g, cell, px, py, pz, margin, sk.bound(), x, y, az, bz, zl, zh);
        if (zl > zh) continue;
        const int t = (x - AX) * NCY + (y - AY);
        atomicMin(&S.zlo[t], zl - AZ);
        atomicMax(&S.zhi[t], zh - AZ);
      }
  }
  __syncthreads();
  // cell offsets of each column's planned range (all loads independent)
  for (int t = threadIdx.x; t < ncol; t += blockDim.x) {
    const int zl = S.zlo[t], zh = S.zhi[t];
    if (zl > zh) continue;
    const int col = ((AX + t / NCY) * g.sy + (AY + t % NCY)) * g.sz + AZ;
    for (int z = zl; z <= zh + 1; ++z) S.off[t][z] = g.cell_start[col + z];
  }
  __syncthreads();
  if (threadIdx.x < 32) {  // exclusive scan of the planned column lengths (kStageCols / 32 per lane)
    constexpr int kPer = kStageCols / 32;
    uint32_t len[kPer];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int t = kPer * threadIdx.x + k;
      len[k] = (t < ncol && S.zlo[t] <= S.zhi[t]) ? S.off[t][S.zhi[t] + 1] - S.off[t][S.zlo[t]] : 0u;
      sum += len[k];
    }
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(full, inc, o);
      if (threadIdx.x >= o) inc += y;
    }
    uint32_t run = inc - sum;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int t = kPer * threadIdx.x + k;
      if (t <= ncol) S.base[t] = run;
      run += len[k];
    }
    if (threadIdx.x == 31) S.total = static_cast<int>(inc);
  }
  __syncthreads();
  const int M = S.total;
  if (M > cap) return false;
  {  // copy: one warp per column, lanes over its points
    const int lane = threadIdx.x & 31;
    for (int t = threadIdx.x >> 5; t < ncol; t += blockDim.x >> 5) {
      if (S.zlo[t] > S.zhi[t]) continue;
      const uint32_t g0 = S.off[t][S.zlo[t]];
      const int len = static_cast<int>(S.off[t][S.zhi[t] + 1] - g0);
      const int b = static_cast<int>(S.base[t]);
      for (int k = lane; k < len; k += 32) S.pts[b + k] = g.pts[g0 + k];
    }
  }
  __syncthreads();
  if (!any) return true;
  for (int x = ax; x <= bx; ++x) {
    for (int y = ay; y <= by; ++y) {
      int zl, zh;
      column_range(g, cell, px, py, pz, margin, sk.bound(), x, y, az, bz, zl, zh);
      const int t = (x - AX) * NCY + (y - AY);
      // Clamp to the planned range: only its offsets were loaded.  The bound
      // has only shrunk since planning, but x * rsqrt(x) is not monotone to
      // the last ulp, so the recomputed range may reach one cell further; the
      // planned range, from the larger bound with its rounding margin, already
      // holds every point within the current bound.
      zl = max(zl, S.zlo[t] + AZ);
      zh = min(zh, S.zhi[t] + AZ);
      if (zl > zh) continue;
      const int shift = static_cast<int>(S.base[t]) - static_cast<int>(S.off[t][S.zlo[t]]);
      const uint32_t gb = S.off[t][zl - AZ], ge = S.off[t][zh + 1 - AZ];
      for (uint32_t k = gb; k < ge; ++k) sk.offer(S.pts[static_cast<int>(k) + shift], static_cast<int>(k), px, py, pz);
    }
  }
  return true;
}

// Error-free transformation: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}



// Rows of per-correspondence factors, one per thread of a tile (kRow floats;
// slot kOne holds 1, slot kZero 0).  Sum k of the block partial is, over the
// rows, x y + (the rounding error of x y) + x yl + xl y with (x, xl, y, yl) =
// the row slots kTerm[kind][k]: a product of two factors for the normal
// equations (J_a J_b, J_a r, r^2; the lows point at zeros), a factor times one
// for plain sums (d2, the match flag), and the exact product of two
// (high, low) pairs for the point-to-point moments.  Every term therefore
// enters as an exact (value, error) pair.
constexpr int kRow = 18, kOne = 16, kZero = 17;
static_assert(kOne == 16 && kZero == 17, "kTerm names the one and zero slots by number");
__constant__ unsigned char kTerm[2][32][4] = {
    {  // point-to-plane: J0..J5 in slots 0-5, r in 6, d2 in 7, match flag in 8
     {0, 0, 17, 17}, {0, 1, 17, 17}, {0, 2, 17, 17}, {0, 3, 17, 17}, {0, 4, 17, 17}, {0, 5, 17, 17},
     {1, 1, 17, 17}, {1, 2, 17, 17}, {1, 3, 17, 17}, {1, 4, 17, 17}, {1, 5, 17, 17},
     {2, 2, 17, 17}, {2, 3, 17, 17}, {2, 4, 17, 17}, {2, 5, 17, 17},
     {3, 3, 17, 17}, {3, 4, 17, 17}, {3, 5, 17, 17},
     {4, 4, 17, 17}, {4, 5, 17, 17},
     {5, 5, 17, 17},
     {0, 6, 17, 17}, {1, 6, 17, 17}, {2, 6, 17, 17}, {3, 6, 17, 17}, {4, 6, 17, 17}, {5, 6, 17, 17},
     {6, 6, 17, 17}, {7, 16, 17, 17}, {8, 16, 17, 17}, {17, 17, 17, 17}, {17, 17, 17, 17}},
    {  // point-to-point: a high 0-2, a low 3-5, b high 6-8, b low 9-11, |a|^2 12, |b|^2 13, d2 14, flag 15
     {0, 16, 3, 17}, {1, 16, 4, 17}, {2, 16, 5, 17}, {6, 16, 9, 17}, {7, 16, 10, 17}, {8, 16, 11, 17},
     {0, 6, 3, 9}, {0, 7, 3, 10}, {0, 8, 3, 11},
     {1, 6, 4, 9}, {1, 7, 4, 10}, {1, 8, 4, 11},
     {2, 6, 5, 9}, {2, 7, 5, 10}, {2, 8, 5, 11},
     {12, 16, 17, 17}, {13, 16, 17, 17},
     {17, 17, 17, 17}, {17, 17, 17, 17}, {17, 17, 17, 17}, {17, 17, 17, 17}, {17, 17, 17, 17},
     {17, 17, 17, 17}, {17, 17, 17, 17}, {17, 17, 17, 17}, {17, 17, 17, 17}, {17, 17, 17, 17},
     {17, 17, 17, 17}, {14, 16, 17, 17}, {15, 16, 17, 17}, {17, 17, 17, 17}, {17, 17, 17, 17}}};

// Compensated pair arithmetic: the exact value is s + c.
__device__ __forceinline__ void add_pair(float& s, float& c, float s2, float c2) {
  float e;
  two_sum(s, s2, s, e);
  c = c + c2 + e;
}

// Block partial of the 32 sums from the tile's rows.  Thread t forms sum
// t % 32 over rows 32 (t / 32) .. 32 (t / 32) + 31 in order, as a compensated
// float32 pair; the four quarters are then added in order and the pair
// rounded to float64.  A fixed sequence, so the result does not depend on
// timing; only a few registers per thread.
__device__ void block_reduce_rows(const float* __restrict__ rows, int kind, float& out_s, float& out_c) {
  static_assert(kThreads == 128, "four quarters of 32 rows");
  __shared__ float qs[4][32], qc[4][32];
  const int k = threadIdx.x & 31, quarter = threadIdx.x >> 5;
  const uchar4 ix = *reinterpret_cast<const uchar4*>(kTerm[kind][k]);
  float s = 0.f, c = 0.f;
  const float* r = rows + quarter * 32 * kRow;
  if (kind == kPointToPlane) {
    // no low parts (their slots hold zeros): the same sums without reading them
#pragma unroll 4
    for (int j = 0; j < 32; ++j, r += kRow) {
      const float x = r[ix.x], y = r[ix.y];
      const float hi = __fmul_rn(x, y);
      const float lo = fmaf(x, y, -hi);
      float e;
      two_sum(s, hi, s, e);
      c += lo + e;
    }
  } else {
#pragma unroll 4
    for (int j = 0; j < 32; ++j, r += kRow) {
      const float x = r[ix.x], y = r[ix.y], xl = r[ix.z], yl = r[ix.w];
      const float hi = __fmul_rn(x, y);
      const float lo = fmaf(x, y, -hi) + fmaf(x, yl, xl * y);
      float e;
      two_sum(s, hi, s, e);
      c += lo + e;
    }
  }
  qs[quarter][k] = s;
  qc[quarter][k] = c;
  __syncthreads();
  if (threadIdx.x < kPartial) {
    float ts = qs[0][k], tc = qc[0][k];
    for (int q = 1; q < 4; ++q) add_pair(ts, tc, qs[q][k], qc[q][k]);
    out_s = ts;
    out_c = tc;
  }
}

// The all-float64 form of the block partial: a butterfly reduce-scatter in each
// warp, then the warps in order, plain float64 adds.  Column t ends on thread t
// (t < kPartial) as `out`.
__device__ void block_reduce_f64(double (&v)[32], double& out) {
  __shared__ double ws[kThreads / 32][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int half = 16; half >= 1; half >>= 1) {
    const bool upper = (lane & half) != 0;
#pragma unroll
    for (int j = 0; j < half; ++j) {
      const double send = upper ? v[j] : v[j + half];
      const double keep = upper ? v[j + half] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, half);
    }
  }
  ws[warp][lane] = v[0];
  __syncthreads();
  const int t = threadIdx.x;
  if (t < kPartial) {
    double s = ws[0][t];
    for (int w = 1; w < kThreads / 32; ++w) s += ws[w][t];
    out = s;
  }
}

// On this GPU a float64 add, multiply, fma, compare or min/max keeps a warp
// busy for dozens of cycles however few of its lanes are active, while integer,
// float32, conversion and shuffle instructions are short.  The serial float64
// code below (the solve at the end of every iteration) is therefore written to
// issue few float64 instructions: independent entries sit on different lanes of
// one warp, and comparisons are made on integer bit patterns.

// A 64-bit integer ordered like the double it encodes (non-NaN values; -0 and
// +0 map to the same key).
__device__ __forceinline__ long long order_key(double v) {
  long long b = __double_as_longlong(v);
  if (b == static_cast<long long>(0x8000000000000000ULL)) b = 0;
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

// 1 / d.  For a positive d within 2^-100 .. 2^100: a float32 seed x (rounding
// plus rcp.approx, relative error below 2^-22), then 1/d = x / (1 - e) with
// e = 1 - d x, evaluated as x (1 + e + e^2): the omitted x e^3 / (1 - e) is
// below 2^-66 relative, so three float64 operations give the quotient to
// within rounding, against the dozens of a full division.  Otherwise (zero,
// negative, tiny, huge, not finite) the division.
__device__ __forceinline__ double recip(double d) {
  const int hi = __double2hiint(d);
  const int ex = (hi >> 20) & 0x7ff;  // biased exponent
  if (hi < 0 || ex < 1023 - 100 || ex > 1023 + 100) return 1.0 / d;
  float xs;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(xs) : "f"(__double2float_rn(d)));
  const double x = static_cast<double>(xs);
  const double e = fma(-d, x, 1.0);
  return fma(x, fma(e, e, e), x);
}

// The polynomial q(x^2) of sin x = x + x^3 q or cos x = 1 - x^2 q, truncated to
// its first N Taylor coefficients, by Horner's rule in x^2.
template <int N>
__device__ __forceinline__ double sincos_q(double x2, bool is_sin) {
  constexpr double kSinQ[7] = {-1.0 / 6.0,          1.0 / 120.0,          -1.0 / 5040.0,         1.0 / 362880.0,
                               -1.0 / 39916800.0,   1.0 / 6227020800.0,   -1.0 / 1307674368000.0};
  constexpr double kCosQ[7] = {1.0 / 2.0,           -1.0 / 24.0,          1.0 / 720.0,           -1.0 / 40320.0,
                               1.0 / 3628800.0,     -1.0 / 479001600.0,   1.0 / 87178291200.0};
  double q = is_sin ? kSinQ[N - 1] : kCosQ[N - 1];
#pragma unroll
  for (int k = N - 2; k >= 0; --k) q = fma(q, x2, is_sin ? kSinQ[k] : kCosQ[k]);
  return q;
}

__device__ __forceinline__ double shfl_d(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// Entry (i, j) of the symmetric 6x6 from the 21 upper-triangle sums (row-major order).
__device__ __forceinline__ double sym6(const double* sums, int i, int j) {
  const int a = i < j ? i : j, c = i < j ? j : i;
  return sums[a * 6 - (a * (a - 1)) / 2 + (c - a)];
}

// The Gauss-Newton update on one warp, in float64 (Eq. 2).  A x = -b is solved
// by sweeping the bordered symmetric matrix [A b; b^T 0] on pivots 0..5
// (Goodnight's symmetric sweep on pivot p = a_kk: a_kk <- -1/p, row and
// column k <- entry / p, every other a_ij <- a_ij - a_ik a_jk / p); after the
// last pivot the border holds A^-1 b, so x = -border.  The pivots are the
// Schur complements an LDL^T factorisation produces, so the frozen-pivot rule
// is the same: a pivot <= 1e-12 * max_j A_jj is not swept and its unknown is 0
// (the others then solve the system without it).  Lane l < 28 holds entry
// (i, j), i >= j, of the lower triangle, l = i (i + 1) / 2 + j, so a sweep step
// costs five float64 operations for the whole matrix.  Then sin and cos of the
// three angles on lanes 0..5 (as many Taylor terms as the largest angle needs
// for a truncation error below 2^-60; the library call from 0.25 rad), dR =
// Rz(gamma) Ry(beta) Rx(alpha) one entry per lane, and T <- [dR, t] T on lanes
// 4 r + c (Tpre: pose entry `lane` for lanes 0..11, and iters0 the iteration
// count, both fetched by the caller).
__device__ void solve_update(const double* sums, double Tpre, int iters0, IcpState* __restrict__ st, double eps,
                             float a, float mlim) {
  const int lane = threadIdx.x & 31;
  // this lane's entry; lanes 28..31 hold a copy of entry (0, 0) that nothing reads
  const int tl = lane < 28 ? lane : 0;
  const int i = (tl >= 1) + (tl >= 3) + (tl >= 6) + (tl >= 10) + (tl >= 15) + (tl >= 21);
  const int j = tl - (i * (i + 1)) / 2;
  double m = i < 6 ? sym6(sums, i, j) : (j < 6 ? sums[21 + j] : 0.0);
  long long kmax = order_key(sums[0]);
#pragma unroll
  for (int d = 1; d < 6; ++d) kmax = max(kmax, order_key(sym6(sums, d, d)));
  const double thr = 1e-12 * __longlong_as_double(kmax ^ ((kmax >> 63) & 0x7fffffffffffffffLL));
  const long long kthr = order_key(thr);
  unsigned frozen = 0u;
  // not unrolled: this runs once per launch on whichever SM finishes last, so its
  // instructions are fetched cold, and one loop body is fetched once, not six times
#pragma unroll 1
  for (int k = 0; k < 6; ++k) {
    const double p = shfl_d(m, (k * (k + 3)) / 2);
    if (!(order_key(p) > kthr)) {  // p <= thr
      frozen |= 1u << k;
      continue;
    }
    const double rp = recip(p);
    const double aik = shfl_d(m, i >= k ? (i * (i + 1)) / 2 + k : (k * (k + 1)) / 2 + i);
    const double ajk = shfl_d(m, j >= k ? (j * (j + 1)) / 2 + k : (k * (k + 1)) / 2 + j);
    const bool on_i = i == k, on_j = j == k;
    // pivot: -1/p;  row or column k: entry / p;  any other entry: entry - a_ik (a_jk / p)
    const double X = (on_i && on_j) ? -1.0 : ((on_i || on_j) ? m : ajk);
    const double Y = (on_i || on_j) ? 1.0 : -aik;
    const double Z = (on_i || on_j) ? 0.0 : m;
    m = fma(Y, X * rp, Z);
  }
  // x_k = -(border entry (6, k)) on lane 21 + k, 0 for a frozen pivot
  const int kx = lane - 21;
  const double xv = (kx >= 0 && kx < 6 && !((frozen >> kx) & 1u)) ? -m : 0.0;
  // sin (lanes 0..2) and cos (lanes 3..5) of alpha, beta, gamma
  const bool is_sin = lane < 3;
  const double xa = shfl_d(xv, 21 + lane % 3);
  const unsigned hx = is_sin ? (static_cast<unsigned>(__double2hiint(xa)) & 0x7fffffffu) : 0u;
  const unsigned hmax = __reduce_max_sync(0xffffffffu, hx);  // high word of the largest |angle|
  double f;
  if (hmax >= 0x3FD00000u) {  // some |angle| >= 2^-2
    double sn, cs;
    sincos(xa, &sn, &cs);
    f = is_sin ? sn : cs;
  } else {
    const double x2 = xa * xa;
    double q;
    if (hmax < 0x3EB00000u) q = sincos_q<1>(x2, is_sin);       // all |angle| < 2^-20
    else if (hmax < 0x3F300000u) q = sincos_q<2>(x2, is_sin);  // < 2^-12
    else if (hmax < 0x3F800000u) q = sincos_q<3>(x2, is_sin);  // < 2^-7
    else if (hmax < 0x3FB00000u) q = sincos_q<4>(x2, is_sin);  // < 2^-4
    else q = sincos_q<6>(x2, is_sin);                          // < 2^-2
    f = fma((is_sin ? xa : -1.0) * x2, q, is_sin ? xa : 1.0);
  }
  const double sa = shfl_d(f, 0), sb = shfl_d(f, 1), sg = shfl_d(f, 2);
  const double ca = shfl_d(f, 3), cb = shfl_d(f, 4), cg = shfl_d(f, 5);
  // entry e = 3 row + column of dR on lane e (lanes 9..31 repeat entry 8) as a1 a2 a3 + b1 b2:
  // row 0: cg cb, cg sb sa - sg ca, cg sb ca + sg sa;  row 1: sg cb, sg sb sa + cg ca,
  // sg sb ca - cg sa;  row 2: -sb, cb sa, cb ca
  const int e = lane < 9 ? lane : 8;
  const double a1 = e < 3 ? cg : (e < 6 ? sg : (e == 6 ? -1.0 : cb));
  const double a2 = (e == 0 || e == 3) ? cb : (e == 7 ? sa : (e == 8 ? ca : sb));
  const double a3 = (e == 1 || e == 4) ? sa : ((e == 2 || e == 5) ? ca : 1.0);
  const double b1 = e == 1 ? -sg : (e == 2 ? sg : (e == 4 ? cg : (e == 5 ? -cg : 0.0)));
  const double b2 = (e == 1 || e == 4) ? ca : ((e == 2 || e == 5) ? sa : 0.0);
  const double dR = fma(b1, b2, (a1 * a2) * a3);
  // row r of dR times column c of T (plus t_r in column 3) on lane 4 r + c
  const int r = (lane >> 2) < 3 ? (lane >> 2) : 0, c = lane & 3;
  const double d0 = shfl_d(dR, 3 * r), d1 = shfl_d(dR, 3 * r + 1), d2 = shfl_d(dR, 3 * r + 2);
  const double t0 = shfl_d(Tpre, c), t1 = shfl_d(Tpre, 4 + c), t2 = shfl_d(Tpre, 8 + c);
  const double xt = shfl_d(xv, 24 + r);
  const double tn = fma(d2, t2, fma(d1, t1, fma(d0, t0, c == 3 ? xt : 0.0)));
  if (lane < 12) {
    st->T[lane] = tn;
    if (c < 3) st->R[3 * r + c] = __double2float_rn(tn);
    else st->t[r] = __double2float_rn(tn);
  }
  // candidate lists pay once the updates are small: the update moves every
  // point p by at most |(alpha, beta, gamma)| |p| + |t| (to first order), with
  // |p| <= a; below mlim the pair keeps lists from the next launch on (float32:
  // only the speed depends on this)
  {
    const float xf = static_cast<float>(xv);
    const float q = xf * xf;
    const float w2 = (__shfl_sync(0xffffffffu, q, 21) + __shfl_sync(0xffffffffu, q, 22)) +
                     __shfl_sync(0xffffffffu, q, 23);
    const float t2 = (__shfl_sync(0xffffffffu, q, 24) + __shfl_sync(0xffffffffu, q, 25)) +
                     __shfl_sync(0xffffffffu, q, 26);
    if (lane == 0 && sqrtf(w2) * a + sqrtf(t2) < mlim) st->lists_on = 1;
  }
  // converged when |(alpha, beta, gamma)|^2 < eps^2 and |t|^2 < eps^2 (eps > 0)
  bool done = false;
  if (order_key(eps) > 0) {
    const double sq = xv * xv;
    const double s3 = (sq + __shfl_down_sync(0xffffffffu, sq, 1)) + __shfl_down_sync(0xffffffffu, sq, 2);
    const unsigned small = __ballot_sync(0xffffffffu, order_key(s3) < order_key(eps * eps));
    done = ((small >> 21) & 1u) && ((small >> 24) & 1u);
  }
  if (lane == 0) {
    if (frozen) st->degenerate = 1;
    st->iters = iters0 + 1;
    if (done) st->done = 1;
  }
}

// Helpers of the serial float64 code: 2^k (|k| < 1023), the biased exponent of
// a double, and a float32 reciprocal (rcp.approx) of a double.
__device__ __forceinline__ double pow2(int k) { return __longlong_as_double(static_cast<long long>(1023 + k) << 52); }
__device__ __forceinline__ int bexp(double v) { return (__double2hiint(v) >> 20) & 0x7ff; }
__device__ __forceinline__ float rcp_f(double d) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(__double2float_rn(d)));
  return r;
}


// Point-to-point update on one warp in float64 (TransformationEstimationPointToPoint,
// Sec. 3.3): the rigid motion minimising sum |R p + t - q|^2 over the matched
// pairs, by Horn's unit-quaternion closed form.  The block sums hold the
// moments of a = p - c and b = q - c for a fixed reference point c near the
// clouds (sums 0-2: a, 3-5: b, 6-14: a b^T row-major, 15: |a|^2, 16: |b|^2),
// from which the centred cross-covariance S and E0 = (sum|a - mean a|^2 +
// sum|b - mean b|^2) / 2 follow.  Horn's trace-free symmetric N (built from S,
// one entry per lane) is scaled by 2^-e with 2^e >= |N|_F, which puts every
// eigenvalue in [-1, 1] and is exact; its largest eigenvalue comes from the
// characteristic quartic x^4 + c2 x^2 + c1 x + c0 (c2 = -tr(N^2)/2,
// c1 = -tr(N^3)/3, c0 = det N) by Newton's method from x = 1, as in the QCP
// method of Theobald (Acta Cryst. A 61, 2005): to the right of its largest
// root the quartic is increasing and convex (the roots of its derivatives
// interlace its own), so the iterates fall monotonically onto the root; float32
// steps first, then float64 steps with a float32 reciprocal of the slope
// (each contracts the error by about 2^-22) until the step is below 2^-50 of the
// root.  The second largest eigenvalue comes from the deflated cubic the same
// way.  A gap below 1e-6 E0 (E0 bounds every eigenvalue's magnitude) leaves the
// rotation undetermined: R = I, the degenerate flag is set.  (Newton on a
// double root stops about 1e-8 from it, so a threshold near the float64
// rounding level would miss exact degeneracy; float32 inputs cannot fix a
// rotation with a smaller gap anyway.)  Otherwise the quaternion q is the
// column of adj(N - lambda I) whose diagonal entry has the largest magnitude
// (for a simple eigenvalue adj is a multiple of v v^T), and dR is the rotation
// of q / |q| formed directly from q and 1 / |q|^2 (the same for q and -q).
// t = mean q - dR mean p;  T <- [dR t; 0 1] T;  done when the rotation angle
// and |t| are below eps, the angle tested as |q_xyz|^2 < tan^2(eps/2) q_w^2.
// Few float64 instructions: comparisons on integer bit patterns, exact
// power-of-two scalings, no division or square root.
__device__ void solve_update_p2p(const double* sums, double Tpre, int iters0, IcpState* __restrict__ st,
                                 double eps, double eps_tan2, float cx, float cy, float cz) {
  __shared__ double sS[9], sN[16], sM[16];
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const double n = sums[29];
  const double inv_n = recip(n);
  // means of a (lanes 0..2) and b (lanes 3..5), and n times them
  const double mk = lane < 6 ? sums[lane] * inv_n : 0.0;
  const double nm = n * mk;
  {
    const int i = lane < 9 ? lane / 3 : 0, j = lane < 9 ? lane % 3 : 0;
    const double s = fma(-shfl_d(nm, i), shfl_d(mk, 3 + j), sums[6 + (lane < 9 ? lane : 0)]);
    if (lane < 9) sS[lane] = s;
  }
  // E0 = (sum |a - mean a|^2 + sum |b - mean b|^2) / 2
  double e0;
  {
    double q = lane < 6 ? nm * mk : 0.0;
    q += __shfl_xor_sync(full, q, 1);
    q += __shfl_xor_sync(full, q, 2);
    q += __shfl_xor_sync(full, q, 4);
    e0 = 0.5 * ((sums[15] + sums[16]) - shfl_d(q, 0));
  }
  __syncwarp();
  if (lane < 16) {
    // Horn's N, entry (i, j) on lane 4 i + j as (s1 S[k1] + s2 S[k2]) + s3 S[k3], S index 3 row + col
    const int k1 = static_cast<int>((0x0561501661051650ULL >> (4 * lane)) & 15);
    const int k2 = static_cast<int>((0x4723743223473274ULL >> (4 * lane)) & 15);
    const unsigned neg1 = 0x8400u, neg2 = 0x913Eu, neg3 = 0x0420u, has3 = 0x8421u;
    const int k3 = 8;
    double a = sS[k1], b = sS[k2], c = sS[k3];
    if ((neg1 >> lane) & 1u) a = -a;
    if ((neg2 >> lane) & 1u) b = -b;
    if ((neg3 >> lane) & 1u) c = -c;
    const double ab = a + b;
    const double v = ab + c;
    sN[lane] = ((has3 >> lane) & 1u) ? v : ab;
  }
  __syncwarp();
  // tr(N^2) on lanes 0..15 and tr(N^3) on lanes 16..31 of one register; det N (Laplace along rows 0, 1,
  // lane k < 6 takes column pair k) on another
  double r1, r2 = 0.0;
  {
    const int h = lane & 15, i = h >> 2, j = h & 3;
    double n2 = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) n2 = fma(sN[4 * i + k], sN[4 * k + j], n2);
    r1 = (lane < 16 ? sN[h] : n2) * sN[lane < 16 ? h : 4 * j + i];
    if (lane < 6) {
      const int a = lane < 3 ? 0 : (lane < 5 ? 1 : 2);
      const int b = lane < 3 ? lane + 1 : (lane < 5 ? lane - 1 : 3);
      const int c = (a != 0 && b != 0) ? 0 : ((a != 1 && b != 1) ? 1 : 2);
      const int d = 6 - a - b - c;
      const double top = sN[a] * sN[4 + b] - sN[b] * sN[4 + a];
      const double bot = sN[8 + c] * sN[12 + d] - sN[8 + d] * sN[12 + c];
      r2 = ((1 + a + b) & 1) ? -top * bot : top * bot;
    }
  }
#pragma unroll
  for (int off = 8; off >= 1; off >>= 1) r1 += __shfl_xor_sync(full, r1, off);
#pragma unroll
  for (int off = 4; off >= 1; off >>= 1) r2 += __shfl_xor_sync(full, r2, off);
  const double t2 = shfl_d(r1, 0), t3 = shfl_d(r1, 16), dt = shfl_d(r2, 0);
  double w = 1.0, x = 0.0, y = 0.0, z = 0.0;
  bool degenerate = true;
  const int et = bexp(t2);
  if (et > 0 && et < 0x7ff && order_key(e0) > 0) {
    // scale N by 2^-e with 2^e >= |N|_F: every eigenvalue in [-1, 1], and the scaling is exact
    const int e = (et - 1022 + 1) >> 1;
    const double c2 = t2 * -pow2(-2 * e - 1);
    const double c1 = (t3 * (-pow2(-2 * e) * (1.0 / 3.0))) * pow2(-e);  // = -t3 2^-3e / 3, no division
    const double c0 = (dt * pow2(-2 * e)) * pow2(-2 * e);
    // largest root of x^4 + c2 x^2 + c1 x + c0 by Newton from 1: float32 to convergence, then float64
    // steps with the float32 reciprocal of the slope (each contracts the error by 2^-22 or better)
    float xf = 1.0f;
    {
      const float f2 = static_cast<float>(c2), f1 = static_cast<float>(c1), f0 = static_cast<float>(c0);
      for (int k = 0; k < 64; ++k) {
        const float x2 = xf * xf;
        const float f = (x2 + f2) * x2 + (f1 * xf + f0);
        const float d = (4.0f * x2 + 2.0f * f2) * xf + f1;
        if (!(f > 0.0f) || !(d > 0.0f)) break;
        const float nx = xf - f / d;
        if (!(nx < xf)) break;
        xf = nx;
      }
    }
    double l1 = xf;
    const double two_c2 = c2 + c2;
    for (int k = 0; k < 8; ++k) {
      const double x2 = l1 * l1;
      const double f = fma(x2 + c2, x2, fma(c1, l1, c0));
      const double d = fma(fma(4.0, x2, two_c2), l1, c1);
      const float rd = rcp_f(d);
      if (!(rd > 0.0f && rd < 3.0e38f)) break;
      const double step = f * static_cast<double>(rd);
      l1 -= step;
      if (step == 0.0 || bexp(step) + 50 < max(bexp(l1), 1023 - 20)) break;
    }
    // second root from the deflated cubic x^3 + l1 x^2 + a1 x + a0: float32 Newton from l1, one float64 step
    const double a1 = fma(l1, l1, c2), a0 = fma(l1, a1, c1);
    float yf = static_cast<float>(l1);
    {
      const float g2 = yf, g1 = static_cast<float>(a1), g0 = static_cast<float>(a0);
      for (int k = 0; k < 64; ++k) {
        const float f = ((yf + g2) * yf + g1) * yf + g0;
        const float d = (3.0f * yf + 2.0f * g2) * yf + g1;
        if (!(f > 0.0f) || !(d > 0.0f)) break;
        const float ny = yf - f / d;
        if (!(ny < yf)) break;
        yf = ny;
      }
    }
    double l2 = yf;
    {
      const double f = fma(fma(l2 + l1, l2, a1), l2, a0);
      const double d = fma(fma(3.0, l2, l1 + l1), l2, a1);
      const float rd = rcp_f(d);
      if (rd > 0.0f && rd < 3.0e38f) l2 -= f * static_cast<double>(rd);
    }
    degenerate = !(order_key(l1 - l2) > order_key(1e-6 * e0 * pow2(-e)));
    if (!degenerate) {
      if (lane < 16) sM[lane] = fma(sN[lane], pow2(-e), (lane % 5 == 0) ? -l1 : 0.0);
      __syncwarp();
      // cofactor (i, j) of M = N / 2^e - l1 I on lane 4 i + j
      double cof = 0.0;
      if (lane < 16) {
        const int i = lane >> 2, j = lane & 3;
        const int r0 = i == 0 ? 1 : 0, r1i = i <= 1 ? 2 : 1, r2i = i <= 2 ? 3 : 2;
        const int q0 = j == 0 ? 1 : 0, q1 = j <= 1 ? 2 : 1, q2 = j <= 2 ? 3 : 2;
        const double m0 = fma(-sM[4 * r1i + q2], sM[4 * r2i + q1], sM[4 * r1i + q1] * sM[4 * r2i + q2]);
        const double m1 = fma(-sM[4 * r1i + q2], sM[4 * r2i + q0], sM[4 * r1i + q0] * sM[4 * r2i + q2]);
        const double m2 = fma(-sM[4 * r1i + q1], sM[4 * r2i + q0], sM[4 * r1i + q0] * sM[4 * r2i + q1]);
        const double d3 = fma(sM[4 * r0 + q2], m2, fma(-sM[4 * r0 + q1], m1, sM[4 * r0 + q0] * m0));
        cof = ((i + j) & 1) ? -d3 : d3;
      }
      // adj(M) is a multiple of v v^T: take the column whose diagonal entry is largest in magnitude
      const long long k0 = __double_as_longlong(shfl_d(cof, 0)) & 0x7fffffffffffffffLL;
      const long long k1 = __double_as_longlong(shfl_d(cof, 5)) & 0x7fffffffffffffffLL;
      const long long k2 = __double_as_longlong(shfl_d(cof, 10)) & 0x7fffffffffffffffLL;
      const long long k3 = __double_as_longlong(shfl_d(cof, 15)) & 0x7fffffffffffffffLL;
      int jb = 0;
      long long best = k0;
      if (k1 > best) { best = k1; jb = 1; }
      if (k2 > best) { best = k2; jb = 2; }
      if (k3 > best) { best = k3; jb = 3; }
      w = shfl_d(cof, jb);
      x = shfl_d(cof, 4 + jb);
      y = shfl_d(cof, 8 + jb);
      z = shfl_d(cof, 12 + jb);
      if (best == 0 || best >= 0x7ff0000000000000LL) degenerate = true;  // no usable column
    }
  }
  if (degenerate) w = 1.0, x = y = z = 0.0;
  // dR from q = (w, x, y, z) of any length: entry e = 3 row + col on lane e as (A B + C D) 2 / |q|^2 + K
  const double s2 = fma(z, z, fma(y, y, fma(x, x, w * w)));
  const double two_inv = 2.0 * recip(s2);
  const int e = lane < 9 ? lane : 8;
  double A, B, C, D, K = 0.0;
  // diagonal: 2 (w^2 + q_i^2) / |q|^2 - 1;  off-diagonal: 2 (q_a q_b +- w q_c) / |q|^2
  const int ri = e / 3, ci = e % 3;
  auto qsel = [&](int k) { return k == 0 ? x : (k == 1 ? y : z); };
  if (ri == ci) {
    A = w; B = w; C = qsel(ri); D = C; K = -1.0;
  } else {
    const int oth = 3 - ri - ci;
    A = qsel(ri < ci ? ri : ci); B = qsel(ri < ci ? ci : ri); D = qsel(oth);
    // sign of w q_c: + for (1,0), (0,2), (2,1); - for (0,1), (2,0), (1,2)
    const bool plus = (ri == 1 && ci == 0) || (ri == 0 && ci == 2) || (ri == 2 && ci == 1);
    C = plus ? w : -w;
  }
  const double dR = fma(fma(A, B, C * D), two_inv, K);
  // translation t_r = mean q_r - (dR mean p)_r, mean p = mean a + c, mean q = mean b + c, on lanes 4 r + c
  const double cc = lane < 6 ? static_cast<double>((lane % 3) == 0 ? cx : ((lane % 3) == 1 ? cy : cz)) : 0.0;
  const double mpq = lane < 6 ? fma(sums[lane], inv_n, cc) : 0.0;  // lanes 0..2: mean p, 3..5: mean q
  const int r = (lane >> 2) < 3 ? (lane >> 2) : 0, c = lane & 3;
  const double d0 = shfl_d(dR, 3 * r), d1 = shfl_d(dR, 3 * r + 1), d2 = shfl_d(dR, 3 * r + 2);
  const double tr = shfl_d(mpq, 3 + r) - fma(d2, shfl_d(mpq, 2), fma(d1, shfl_d(mpq, 1), d0 * shfl_d(mpq, 0)));
  const double t0 = shfl_d(Tpre, c), t1 = shfl_d(Tpre, 4 + c), tt2 = shfl_d(Tpre, 8 + c);
  const double tn = fma(d2, tt2, fma(d1, t1, fma(d0, t0, c == 3 ? tr : 0.0)));
  if (lane < 12) {
    st->T[lane] = tn;
    if (c < 3) st->R[3 * r + c] = __double2float_rn(tn);
    else st->t[r] = __double2float_rn(tn);
  }
  bool done = false;
  if (order_key(eps) > 0) {
    // angle < eps  <=>  |(x, y, z)|^2 < tan^2(eps / 2) w^2;  |t| < eps
    const double v2 = fma(z, z, fma(y, y, x * x));
    const bool rot_ok = degenerate || order_key(v2) < order_key((w * w) * eps_tan2);
    const double tx = shfl_d(tr, 0), ty = shfl_d(tr, 4), tz = shfl_d(tr, 8);
    const double tl2 = fma(tz, tz, fma(ty, ty, tx * tx));
    done = rot_ok && order_key(tl2) < order_key(eps * eps);
  }
  if (lane == 0) {
    if (degenerate) st->degenerate = 1;
    st->iters = iters0 + 1;
    if (done) st->done = 1;
  }
}

// The convergence threshold as the device reads it: eps if eps > 0, else 0
// (never; also for NaN), so that the device tests it on its bit pattern.
inline double stop_eps(double eps) { return eps > 0.0 ? eps : 0.0; }

// tan^2(eps / 2), the point-to-point rotation threshold (see solve_update_p2p).
inline double stop_tan2(double eps) {
  if (!(eps > 0.0)) return 0.0;
  if (eps >= 3.141592653589793) return 1e300;
  const double t = std::tan(0.5 * eps);
  return t * t;
}

// Everything one registration problem brings to an iteration launch.
struct PairDesc {
  GridView g;
  float cell, r;
  double eps;          // convergence threshold of this pair (0: never; see stop_eps)
  double eps_tan2;     // tan^2(eps / 2) (see stop_tan2)
  int kind;            // kPointToPlane or kPointToPoint
  float ctr[3];        // point-to-point: reference point subtracted before the moments
  const float4* src4;  // cell-sorted source, .w = original index bits
  int ns;
  int ntiles;          // ceil(ns / (kThreads ppt)), at least 1
  int tile0;           // first global tile of this pair
  IcpState* st;
  unsigned long long* acc;  // nacc x kPartial fixed-point sums (see add_fixed), zero between launches
  int nacc;                 // accumulator rows: min(kAccRows, ntiles)
  float bnd_a, bnd_b;       // per-correspondence bounds the sums are scaled by (see set_sums)
  int ppt;             // sub-tiles of kThreads points per tile (see icp_tile)
  ListRef lists;       // per source point last matches and candidate lists (see ListSink); pb null: none kept
  float list_motion;   // the pair keeps candidate lists once an update moves points by less (< 0: never)
  int32_t* corr_out;   // kCorrOnly / kEvaluate outputs (by original source index), or null
  float* d2_out;
};

// Fixed-point sums.  Every tile adds its partial of each sum column to one of
// its pair's kAccRows accumulator rows as a 64-bit integer count of units 2^E
// (E per column), by integer atomics.  Integer addition is exact and
// associative, so the totals do not depend on the order in which tiles add
// them, nor on which other pairs share the launch.  E rests on an a-priori
// bound: a column's total is at most ns times a bound on one correspondence's
// term, and E puts that bound below 2^62, so no accumulator overflows; a unit
// is then at most 2^-61 of the bound, and each partial rounds by at most one
// unit.

// Bound on one correspondence's value in row slot `slot` (kTerm numbering).
// Point-to-plane: |J_0..2| = |p x n| <= a L, |J_3..5| = |n| <= L, |r| <= R L,
// d2 <= R^2, flag 1, where a bounds |p|, L the normals' length, R the radius.
// Point-to-point: |a| <= a, |b| <= b (both parts of each), |a|^2, |b|^2,
// d2 <= R^2, flag 1.
__device__ __forceinline__ float slot_bound(int kind, int slot, float a, float b, float L, float R) {
  if (slot == kOne) return 1.f;
  if (slot == kZero) return 0.f;
  if (kind == kPointToPlane) {
    if (slot < 3) return a * L;
    if (slot < 6) return L;
    if (slot == 6) return R * L;
    if (slot == 7) return R * R;
    return 1.f;  // 8: the match flag
  }
  if (slot < 6) return a;   // a, high and low parts
  if (slot < 12) return b;  // b, high and low parts
  if (slot == 12) return a * a;
  if (slot == 13) return b * b;
  if (slot == 14) return R * R;
  return 1.f;  // 15: the match flag
}

// E of sum column k: floor(log2(bound)) + 1 - 62, the bound computed in float32
// with a 1% margin on every factor (nlen: the target normals' length bound).
__device__ __forceinline__ int sum_exponent(const PairDesc& P, int k, float nlen) {
  const uchar4 ix = *reinterpret_cast<const uchar4*>(kTerm[P.kind][k]);
  const float R = P.r * 1.01f, L = nlen * 1.01f, a = P.bnd_a * 1.01f, b = P.bnd_b * 1.01f;
  const float B = slot_bound(P.kind, ix.x, a, b, L, R) * slot_bound(P.kind, ix.y, a, b, L, R) *
                  (static_cast<float>(max(P.ns, 1)) * 1.01f);
  if (B != B) return -126;    // a NaN bound: report every nonzero term
  if (!(B > 0.f)) return 0;  // an empty column
  const int e = ((__float_as_int(B) >> 23) & 0xff) - 127;
  // a bound beyond float range (absurd coordinates): the smallest unit, so that
  // every nonzero term of the column is reported rather than rounded away
  if (e == 128) return -126;
  return min(max(e + 1 - 62, -126), 126);
}

// Adds this lane's column k of the block partial, the exact pair ts + tc, to
// accumulator row `acc` in units of 2^E.  A partial whose value is not below
// 2^62 units (outside its bound, or not finite) is left out and counted in
// column kBadCol, which the finish reports as non-finite sums.  Warp 0, lane k.
__device__ __forceinline__ void add_fixed(unsigned long long* acc, int k, float ts, float tc, int E) {
  const float sc = __int_as_float((127 - E) << 23);  // 2^-E
  const float hs = ts * sc, hc = tc * sc;             // exact (an underflow is below one unit)
  const bool ok = fabsf(hs) < 0x1p62f && fabsf(hc) < 0x1p62f;
  long long v = ok ? __float2ll_rn(hs) + __float2ll_rn(hc) : 0;
  const bool bad = __any_sync(0xffffffffu, !ok);
  if (k == kBadCol) v = bad ? 1 : 0;
  if (v != 0) atomicAdd(acc + k, static_cast<unsigned long long>(v));
}

// The same for a float64 partial.
__device__ __forceinline__ void add_fixed_f64(unsigned long long* acc, int k, double s, int E) {
  const double h = s * __longlong_as_double(static_cast<long long>(1023 - E) << 52);  // exact
  const bool ok = (__double_as_longlong(h) & 0x7fffffffffffffffLL) < 0x43D0000000000000LL;  // |h| < 2^62
  long long v = ok ? __double2ll_rn(h) : 0;
  const bool bad = __any_sync(0xffffffffu, !ok);
  if (k == kBadCol) v = bad ? 1 : 0;
  if (v != 0) atomicAdd(acc + k, static_cast<unsigned long long>(v));
}

// Run by the last tile of a pair to arrive: the totals of every sum column
// (integer adds, in any order) converted to float64 with one rounding, the
// accumulator rows cleared for the next launch; then per mode the update, the
// stored normal equations, or fitness / rmse.
__device__ void finish(const PairDesc& P, int mode, float nlen) {
  static_assert(kThreads == 128 && kPartial == 32 && kAccRows % 4 == 0, "4 x 32 threads over the rows");
  __shared__ long long sub[4][kPartial];
  __shared__ double sums[kPartial];
  __shared__ bool bad;
  const int col = threadIdx.x & 31, q = threadIdx.x >> 5;
  IcpState* const st = P.st;
  // the pose rows the update multiplies and the iteration count, fetched with the accumulators
  const double Tpre = threadIdx.x < 12 ? st->T[threadIdx.x] : 0.0;
  const int iters0 = st->iters;
  unsigned long long v[kAccRows / 4];
#pragma unroll
  for (int j = 0; j < kAccRows / 4; ++j) {
    const int row = q + 4 * j;
    v[j] = row < P.nacc ? __ldcg(P.acc + static_cast<size_t>(row) * kPartial + col) : 0ull;
  }
  unsigned long long t = 0ull;
#pragma unroll
  for (int j = 0; j < kAccRows / 4; ++j) {
    t += v[j];
    const int row = q + 4 * j;
    if (row < P.nacc) P.acc[static_cast<size_t>(row) * kPartial + col] = 0ull;
  }
  sub[q][col] = static_cast<long long>(t);
  __syncthreads();
  if (threadIdx.x < kPartial) {
    const long long tot = sub[0][col] + sub[1][col] + sub[2][col] + sub[3][col];
    const int E = sum_exponent(P, col, nlen);
    sums[col] = __ll2double_rn(tot) * __longlong_as_double(static_cast<long long>(1023 + E) << 52);
    if (col == kBadCol) bad = tot != 0;
  }
  __syncthreads();
  const double count = sums[29];
  if (mode == kEvaluate) {
    if (threadIdx.x == 0) {
      if (bad) st->nonfinite = 1;
      st->fitness = P.ns > 0 ? count / static_cast<double>(P.ns) : 0.0;
      st->rmse = count > 0.0 ? sqrt(sums[28] / count) : 0.0;
    }
    return;
  }
  if (mode == kEquations) {
    const int t2 = threadIdx.x;
    if (t2 < 36) st->A[t2] = sym6(sums, t2 / 6, t2 % 6);
    else if (t2 < 42) st->b[t2 - 36] = sums[21 + (t2 - 36)];
    else if (t2 < 45) st->stats[t2 - 42] = sums[27 + (t2 - 42)];
    else if (t2 == 45 && bad) st->nonfinite = 1;
    return;
  }
  if (threadIdx.x >= 32) return;
  if (bad || order_key(count) < order_key(P.kind == kPointToPoint ? 3.0 : 6.0)) {
    if (threadIdx.x == 0) {
      if (bad) st->nonfinite = 1;
      else st->few_corr = 1;
      st->done = 1;
    }
    return;
  }
  if (P.kind == kPointToPoint)
    solve_update_p2p(sums, Tpre, iters0, st, P.eps, P.eps_tan2, P.ctr[0], P.ctr[1], P.ctr[2]);
  else solve_update(sums, Tpre, iters0, st, P.eps, P.bnd_a, P.list_motion);
}


// Point-to-point terms of one correspondence about the reference point c =
// P.ctr (near the clouds, so the moments do not cancel): a = p - c, b = q - c,
// a b^T (row-major), |a|^2, |b|^2, d2 and 1, in the slots solve_update_p2p
// reads.  All float64: a and b are exact, the products round once.
__device__ __forceinline__ void p2p_terms(const PairDesc& P, float3 p, float4 q, float d2, double (&v)[32]) {
  const double a[3] = {static_cast<double>(p.x) - P.ctr[0], static_cast<double>(p.y) - P.ctr[1],
                       static_cast<double>(p.z) - P.ctr[2]};
  const double b[3] = {static_cast<double>(q.x) - P.ctr[0], static_cast<double>(q.y) - P.ctr[1],
                       static_cast<double>(q.z) - P.ctr[2]};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    v[k] = a[k];
    v[3 + k] = b[k];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) v[6 + 3 * i + j] = a[i] * b[j];
  v[15] = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
  v[16] = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  v[28] = d2;
  v[29] = 1.0;
}

// The all-float64 terms of one correspondence (p, target bp at d2 = bd2) in the
// sum columns: point-to-plane every term from the float32 p, q, n, each product
// and sum rounded once in the oracle's order (no fused multiply-add);
// point-to-point the moments of p2p_terms.  Zero when bp < 0.
__device__ __forceinline__ void f64_terms(const PairDesc& P, float3 p, int bp, float bd2, double (&v)[32]) {
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = 0.0;
  if (bp >= 0 && P.kind == kPointToPoint) {
    p2p_terms(P, p, P.g.pts[bp], bd2, v);
  } else if (bp >= 0) {
    const float4 q = P.g.pts[bp];
    const float4 n = P.g.nrm[bp];
    const double px = p.x, py = p.y, pz = p.z, nx = n.x, ny = n.y, nz = n.z;
    const double dx = __dsub_rn(px, static_cast<double>(q.x));
    const double dy = __dsub_rn(py, static_cast<double>(q.y));
    const double dz = __dsub_rn(pz, static_cast<double>(q.z));
    const double res = __dadd_rn(__dadd_rn(__dmul_rn(dx, nx), __dmul_rn(dy, ny)), __dmul_rn(dz, nz));
    double J[6];
    J[0] = __dsub_rn(__dmul_rn(py, nz), __dmul_rn(pz, ny));
    J[1] = __dsub_rn(__dmul_rn(pz, nx), __dmul_rn(px, nz));
    J[2] = __dsub_rn(__dmul_rn(px, ny), __dmul_rn(py, nx));
    J[3] = nx;
    J[4] = ny;
    J[5] = nz;
    int k = 0;
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int b = a; b < 6; ++b) v[k++] = __dmul_rn(J[a], J[b]);
#pragma unroll
    for (int a = 0; a < 6; ++a) v[21 + a] = __dmul_rn(J[a], res);
    v[27] = __dmul_rn(res, res);
    v[28] = static_cast<double>(bd2);
    v[29] = 1.0;
  }
}

// The float32 factors of one correspondence in a row of kRow slots (see kTerm):
// point-to-plane J0..J5, r, d2, 1; point-to-point a = p - c and b = q - c as
// exact (high, low) pairs, |a|^2, |b|^2, d2, 1.  Slot kOne holds 1, every other
// slot 0 when bp < 0.
template <class Row>
__device__ __forceinline__ void row_factors(const PairDesc& P, float3 p, int bp, float bd2, Row&& row) {
#pragma unroll
  for (int k = 0; k < kRow; ++k) row(k) = 0.f;
  row(kOne) = 1.f;
  if (bp < 0) return;
  const float4 q = P.g.pts[bp];
  if (P.kind == kPointToPoint) {
    // a = p - c and b = q - c as exact pairs (c = P.ctr, near the clouds)
    const float pv[3] = {p.x, p.y, p.z}, qv[3] = {q.x, q.y, q.z};
    float aa = 0.f, bb = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float ah, al, bh, bl;
      two_sum(pv[k], -P.ctr[k], ah, al);
      two_sum(qv[k], -P.ctr[k], bh, bl);
      row(k) = ah;
      row(3 + k) = al;
      row(6 + k) = bh;
      row(9 + k) = bl;
      aa += ah * ah;
      bb += bh * bh;
    }
    row(12) = aa;
    row(13) = bb;
    row(14) = bd2;
    row(15) = 1.f;
  } else {
    const float4 n = P.g.nrm[bp];
    const float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
    row(0) = p.y * n.z - p.z * n.y;
    row(1) = p.z * n.x - p.x * n.z;
    row(2) = p.x * n.y - p.y * n.x;
    row(3) = n.x;
    row(4) = n.y;
    row(5) = n.z;
    row(6) = dx * n.x + dy * n.y + dz * n.z;
    row(7) = bd2;
    row(8) = 1.f;
  }
}

// One tile of one ICP step: P.ppt sub-tiles of kThreads consecutive
// cell-sorted source points each (tile j of pair P).  mode kIterate: skipped
// once the pair is done; the other modes always run.  kCorrOnly writes
// corr/d2 and no sums.  Each sub-tile's partial of every sum column is the
// transposed compensated reduction of its rows; the tile's partial is the
// compensated sum of its sub-tiles' partials in order, added once to the
// pair's fixed-point accumulators; the last tile of the pair to arrive
// performs the pair's solve and update (see finish).  Block-uniform control
// flow.
template <bool F64, class St>
__device__ void icp_tile(const PairDesc& P, int j, int mode, St& stage) {
  // the state the tile starts with (the stop flag, the list mode, the pose) is
  // loaded together with the first sub-tile's points: one memory round trip
  const int done = P.st->done;
  const int lists_on = P.st->lists_on;
  const int phase = P.st->phase;
  float R[9], t[3];
#pragma unroll
  for (int k = 0; k < 9; ++k) R[k] = P.st->R[k];
#pragma unroll
  for (int k = 0; k < 3; ++k) t[k] = P.st->t[k];
  const int mode_in = mode;
  if (mode == kServe) {
    if (phase >= 2) return;
    mode = phase == 0 ? kIterate : kEvaluate;
  }
  const bool keep = P.lists.pb != nullptr;  // matches (and lists) are kept across launches
  // (a launch form without list support searches every point: the same
  // correspondences and the same sums, only slower)
  const bool lists = St::kLists && keep && lists_on && P.kind == kPointToPlane;
  const float r2 = __fmul_rn(P.r, P.r);
  const float sigma = __fmul_rn(P.r, kSkin), Rl = __fadd_rn(P.r, sigma);
  // the lists being rebuilt (see ListSink) in the stage's last kListPts points
  float(*const s_ld)[kThreads] = reinterpret_cast<float(*)[kThreads]>(&stage.pts[St::kStagePts - kListPts]);
  int(*const s_lp)[kThreads] = reinterpret_cast<int(*)[kThreads]>(&s_ld[kList][0]);
  float tile_s = 0.f, tile_c = 0.f;  // the tile's partial (threads < kPartial)
  double tile_f64 = 0.0;
  for (int sub = 0; sub < P.ppt; ++sub) {
    const int i = (j * P.ppt + sub) * kThreads + threadIdx.x;
    const bool live = i < P.ns;
    // (the source, hints and lists are read once per launch: loaded with the
    // streaming hint, so that the targets and normals the gathers reuse stay in L2)
    const float4 s = live ? __ldcs(&P.src4[i]) : make_float4(3.0e38f, 3.0e38f, 3.0e38f, 0.f);
    // the last match seeds the search (before lists, of every point; with lists,
    // of the points their lists no longer cover); loaded with the point, not
    // after the state, so that the tile starts with one memory round trip
    int hint = (keep && live) ? __ldcs(&P.lists.hint[i]) : -1;
    float4 pb = make_float4(0.f, 0.f, 0.f, -1.f);
    int4 l[kListVec];
#pragma unroll
    for (int k = 0; k < kListVec; ++k) l[k] = make_int4(-1, -1, -1, -1);
    uint2 gap = make_uint2(0u, 0u);
    if (lists && live) {
      pb = __ldcs(&P.lists.pb[i]);
#pragma unroll
      for (int k = 0; k < kListVec; ++k) l[k] = __ldcs(&P.lists.idx[kListVec * i + k]);
      gap = __ldcs(&P.lists.gap[i]);
    }
    if (mode == kIterate && done) return;
    const float3 p = live ? xform_rn(R, t, s.x, s.y, s.z) : make_float3(3.0e38f, 3.0e38f, 3.0e38f);
    // Once the pair keeps lists, a point whose list still covers it is decided
    // by the list alone; the others search the grid from their last match (and
    // rebuild their lists).  Before that, every point searches from the last
    // matches of itself and its warp neighbours.  In the latency form the
    // searches of a sub-tile run block-staged in shared memory (each from
    // global memory when the staged set does not fit); in the throughput form
    // each runs from global memory.
    Nearest nb{r2, 0x7fffffff, -1};
    bool need = live;
    if (lists) {
      const bool covered = list_scan(P.g, pb, l, gap, sigma, p.x, p.y, p.z, nb);  // every lane
      need = live && !covered;
      if (need && hint >= 0) consider(nb, P.g.pts[hint], hint, p.x, p.y, p.z);
    } else {
      first_bound(P.g, p.x, p.y, p.z, hint, nb);
    }
    // (before lists every live point searches: no vote needed)
    if (!lists || __syncthreads_or(need)) {
      if (lists) {
        ListSink ls{nb, s_ld, s_lp, list_lim(nb.d2, sigma), 0, 0.f, 0};
        if (!(St::kStaged && staged_search(P.g, P.cell, p.x, p.y, p.z, Rl, need, ls, stage, St::kStagePts - kListPts)) &&
            need)
          box_search_global(P.g, P.cell, p.x, p.y, p.z, Rl, ls);
        if (need) list_store(P.lists, i, ls, p.x, p.y, p.z, sigma);
        nb = ls.nb;
      } else {
        NnSink ns{nb};
        if (!(St::kStaged && staged_search(P.g, P.cell, p.x, p.y, p.z, P.r, need, ns, stage)) && need)
          box_search_global(P.g, P.cell, p.x, p.y, p.z, P.r, ns);
        nb = ns.nb;
      }
    }
    const float bd2 = nb.d2;
    const int bp = live ? nb.pos : -1;
    if (keep && live && (!lists || need)) P.lists.hint[i] = bp;
    if (live && P.corr_out) {  // kCorrOnly, or a final evaluation that reports its correspondence set
      const int o = __float_as_int(s.w);
      P.corr_out[o] = bp >= 0 ? __float_as_int(P.g.pts[bp].w) : -1;
      P.d2_out[o] = bp >= 0 ? bd2 : 0.f;
    }
    if (mode == kCorrOnly) continue;
    if constexpr (F64) {
      double v[32];
      f64_terms(P, p, bp, bd2, v);
      double col = 0.0;
      block_reduce_f64(v, col);
      if (threadIdx.x < kPartial) tile_f64 += col;
      __syncthreads();  // the reduction's shared words are free again
    } else {
      // per-correspondence factors as one row per thread in shared memory (the
      // staged points are no longer needed), then the transposed reduction
      __syncthreads();  // every thread has finished reading the staged points
      static_assert(St::kStagePts * 4 >= kThreads * kRow, "the stage holds one row per thread");
      float* rows = reinterpret_cast<float*>(stage.pts);
      float* row = rows + threadIdx.x * kRow;
      row_factors(P, p, bp, bd2, [&](int k) -> float& { return row[k]; });
      __syncthreads();
      float ts = 0.f, tc = 0.f;
      block_reduce_rows(rows, P.kind, ts, tc);
      if (threadIdx.x < kPartial) add_pair(tile_s, tile_c, ts, tc);
    }
  }
  if (mode == kCorrOnly) return;
  // this tile's partial of every sum goes to accumulator row j % nacc, scaled by
  // the bounds (nlen: the target normals' length bound)
  unsigned long long* const acc = P.acc + static_cast<size_t>(j % P.nacc) * kPartial;
  const float nlen = (P.kind == kPointToPlane && P.g.nrm) ? P.g.nrm[P.g.n].x : 0.f;
  if (threadIdx.x < kPartial) {
    const int E = sum_exponent(P, threadIdx.x, nlen);
    if constexpr (F64) add_fixed_f64(acc, threadIdx.x, tile_f64, E);
    else add_fixed(acc, threadIdx.x, tile_s, tile_c, E);
  }
  // the last tile of the pair to arrive finishes the launch for the pair
  __shared__ bool last;
  if (threadIdx.x < kPartial) __threadfence();  // the lanes that added the partial publish it
  __syncthreads();
  if (threadIdx.x == 0) {
    last = atomicAdd(&P.st->arrived, 1u) == static_cast<unsigned>(P.ntiles - 1);
    if (last) P.st->arrived = 0u;  // ready for the next launch
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  finish(P, mode, nlen);
  if (mode_in == kServe && threadIdx.x == 0) {  // the thread that wrote the state in finish
    IcpState* const st = P.st;
    st->phase = mode == kEvaluate ? 2 : ((st->done || st->iters >= st->cap) ? 1 : 0);
  }
}

// One ICP step of every pair: a persistent kernel whose blocks walk the global
// tiles (tile, tile + gridDim.x, ...).  pairs == nullptr means the single pair
// `one` owns every tile.  The pair of a tile comes from tile_pair.  Tiles of
// different pairs are independent, and a pair's sums are exact integer sums of
// its tiles' partials, so every pair's result is the same alone and in any batch.
// F64 selects the all-float64 per-correspondence arithmetic (precision study);
// Cfg the stage size and the blocks per SM the registers are budgeted for.
template <bool F64, class Cfg>
__global__ void __launch_bounds__(kThreads, Cfg::kMinBlocks) k_icp_iter(PairDesc one, const PairDesc* __restrict__ pairs,
                                                                     const int* __restrict__ tile_pair,
                                                                     const int* __restrict__ ntiles_total, int mode,
                                                                     unsigned* __restrict__ queue, int parity) {
  __shared__ Stage<Cfg> stage;
  __shared__ PairDesc P;
  __shared__ int s_next;
  // Launched as a programmatic dependent of the previous iteration, this grid
  // may be placed on the GPU before that one ends; everything it reads (the
  // pose, the hints, the counters) is the previous grid's output, so wait for
  // its completion here.  Then let the next iteration start placing its blocks.
  // Both are no-ops for an ordinary launch.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int n = pairs ? *ntiles_total : one.ntiles;
  // Tiles [0, gridDim.x) go to the blocks in order; the rest are claimed one
  // at a time from queue[parity], so blocks that drew cheap tiles take more
  // (results do not depend on which block runs a tile, nor on when it adds its
  // partial).  queue[parity ^ 1] is the counter of the next launch on
  // this queue; the previous launch, which used it, has finished here.
  if (queue && blockIdx.x == 0 && threadIdx.x == 0) queue[parity ^ 1] = 0u;
  __shared__ int s_pair;
  int tile = blockIdx.x;
  while (tile < n) {
    if (threadIdx.x == 0) {
      s_pair = pairs ? tile_pair[tile] : 0;
      P = pairs ? pairs[s_pair] : one;
    }
    __syncthreads();
    icp_tile<F64>(P, tile - P.tile0, mode, stage);
    if (threadIdx.x == 0)
      s_next = queue ? static_cast<int>(gridDim.x + atomicAdd(&queue[parity], 1u)) : tile + static_cast<int>(gridDim.x);
    __syncthreads();
    tile = s_next;
  }
}

// Blocks of one configuration of the persistent iteration kernel that are
// resident on the GPU together.
// (computed once, thread-safely, on first use)
template <bool F64, class Cfg>
int resident_blocks() {
  static const int resident = [] {
    int dev = 0, sms = kNumSMs, per_sm = 1;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_icp_iter<F64, Cfg>, kThreads, 0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    (void)cudaGetLastError();
    return sms * per_sm;
  }();
  return resident;
}

// Grid of a persistent launch: every tile at once when they fit on the GPU
// together, else as many blocks as are resident (they loop over tiles).
inline int grid_for(int ntiles, int resident) { return ntiles < resident ? (ntiles < 1 ? 1 : ntiles) : resident; }

// Launch configuration per size class, class = floor(log2(tiles of the
// launch)): 0 automatic (the latency form while every tile of the launch is
// resident at once in it, else the throughput form), 1 latency, 2 throughput.
std::atomic<int> g_tile_cfg[32];

inline int size_class(int ntiles) {
  int c = 0;
  while (c < 31 && (2LL << c) <= ntiles) ++c;
  return c;
}

bool throughput_form(int ntiles) {
  const int pin = g_tile_cfg[size_class(ntiles)].load(std::memory_order_relaxed);
  if (pin == 1) return false;
  if (pin == 2) return true;
  return ntiles > resident_blocks<false, CfgLatency>();
}

// The dynamic tile queue of a sequence of launches: two counters, zero
// before the first launch; launch k of the sequence passes parity k & 1.
struct TileQueue {
  unsigned* counters = nullptr;  // may be null: blocks then stride over tiles statically
  int parity = 0;
};

template <bool F64, class Cfg>
void launch_form(int ntiles, const PairDesc& one, const PairDesc* pairs, const int* tile_pair, const int* d_ntiles,
                 int mode, cudaStream_t s, bool dependent, TileQueue q) {
  const int grid = grid_for(ntiles, resident_blocks<F64, Cfg>());
  if (!dependent) {
    k_icp_iter<F64, Cfg><<<grid, kThreads, 0, s>>>(one, pairs, tile_pair, d_ntiles, mode, q.counters, q.parity);
    return;
  }
  // programmatic dependent launch: the grid is placed while the previous
  // iteration's tail (group sums, solve) still runs, and waits in the kernel
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_icp_iter<F64, Cfg>, one, pairs, tile_pair, d_ntiles, mode, q.counters, q.parity) !=
      cudaSuccess) {
    (void)cudaGetLastError();
    k_icp_iter<F64, Cfg><<<grid, kThreads, 0, s>>>(one, pairs, tile_pair, d_ntiles, mode, q.counters, q.parity);
  }
}

// One launch of the iteration kernel over `ntiles` work items on stream s;
// `dependent`: as a programmatic dependent of the preceding kernel of s.
void launch_iter(bool f64, int ntiles, const PairDesc& one, const PairDesc* pairs, const int* tile_pair,
                 const int* d_ntiles, int mode, cudaStream_t s, bool dependent = false, TileQueue q = TileQueue{}) {
  if (f64) launch_form<true, CfgLatency>(ntiles, one, pairs, tile_pair, d_ntiles, mode, s, dependent, q);
  else if (throughput_form(ntiles))
    launch_form<false, CfgThroughput>(ntiles, one, pairs, tile_pair, d_ntiles, mode, s, dependent, q);
  else launch_form<false, CfgLatency>(ntiles, one, pairs, tile_pair, d_ntiles, mode, s, dependent, q);
}

// Sub-tiles per tile (points per thread) of a pair of ns source points, per
// size class of the pair (floor(log2(ns))): 0 automatic (kAutoPpt), else 1, 2
// or 4.  A property of the pair, so that it tiles the same way alone, in a
// batch and in the server.
std::atomic<int> g_ppt[32];
int pair_ppt(int64_t ns) {
  int c = 0;
  while (c < 31 && (2LL << c) <= ns) ++c;
  const int pin = g_ppt[c].load(std::memory_order_relaxed);
  if (pin == 1 || pin == 2 || pin == 4) return pin;
  // automatic: measured on a 94,829-point pair (one wave of tiles: 1 best) and
  // a 2,000,000-point pair (4 best, 2 between)
  return ns >= (1 << 20) ? 4 : (ns >= (1 << 18) ? 2 : 1);
}

// Tiles of a pair of ns points with ppt sub-tiles of kThreads points each.
inline int pair_tiles(int64_t ns, int ppt) {
  const int64_t per = static_cast<int64_t>(kThreads) * ppt;
  const int64_t b = (ns + per - 1) / per;
  return static_cast<int>(b < 1 ? 1 : b);
}

// Tiles of kThreads points (one point per thread): the allocation-free call's
// tiles, pose evaluation's, and an upper bound on any pair's tiles.
inline int tiles_of(int64_t ns) { return pair_tiles(ns, 1); }

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
  if (ns < 0 || ns > 0x7fffffffLL - kThreads || (ns > 0 && !d_src) || stride < 3) {
    set_error("%s: invalid source cloud (n=%lld stride=%d)", fn, static_cast<long long>(ns), stride);
    return O3G_ERR_ARG;
  }
  return O3G_OK;
}

inline int accum_rows(int ntiles) { return ntiles < kAccRows ? (ntiles < 1 ? 1 : ntiles) : kAccRows; }

// Points a pair's descriptor at its accumulator rows (accum_rows(P.ntiles) x
// kPartial, zero) and sets the bounds its sums are scaled by, from the
// target's coordinate box: point-to-plane, bnd_a >= |p| for every transformed
// source point p within r of a target point (the box corner farthest from the
// origin, plus r); point-to-point, bnd_a >= |p - c| and bnd_b >= |q - c| for
// the reference point c = P.ctr.  Needs P.kind, P.ctr, P.r and P.ntiles.
void set_sums(PairDesc& P, const o3g_grid* g, unsigned long long* acc) {
  P.acc = acc;
  P.nacc = accum_rows(P.ntiles);
  const bool p2p = P.kind == kPointToPoint;
  double far = 0.0;
  for (int corner = 0; corner < 8; ++corner) {
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
      const double x = ((corner >> a) & 1) ? g->box_hi[a] : g->box_lo[a];
      const double d = x - (p2p ? static_cast<double>(P.ctr[a]) : 0.0);
      d2 += d * d;
    }
    far = std::max(far, std::sqrt(d2));
  }
  // rounded up (the device adds a further 1% per factor)
  P.bnd_a = static_cast<float>((far + static_cast<double>(P.r)) * 1.001 + 1e-30);
  P.bnd_b = static_cast<float>(far * 1.001 + 1e-30);
}

// Everything one ICP-style call needs on the device: the cell-sorted source,
// the iteration state and the fixed-point accumulators.
struct Work {
  SortedCloud src;         // the cell-sorted source when this Work sorts it
  const float4* pts = nullptr;  // the sorted source in use (own, or sorted by the caller)
  const int* aux = nullptr;     // its flags (aux[6]: a non-finite coordinate)
  DevBuf state;
  DevBuf acc;    // accum_rows(nblk) x kPartial fixed-point sums
  DevBuf lists;  // per source point candidate lists (see ListSink): ns float4, then 2 ns int4
  DevBuf queue;  // the dynamic tile queue (2 counters)
  int nblk = 1;
  int ppt = 1;
  int launches = 0;  // launches so far (the queue parity)
  explicit Work(cudaStream_t s) : src(s), state(s), acc(s), lists(s), queue(s) {}
  int32_t prepare(const float* d_src, int64_t ns, int32_t stride, float cell, const double* T, cudaStream_t s,
                  const SortedCloud* pre = nullptr) {
    if (pre) {
      pts = pre->pts;
      aux = pre->aux.as<int>();
    } else {
      O3G_TRY_STATUS(sort_cloud(d_src, ns, stride, s, &src));
      pts = src.pts;
      aux = src.aux.as<int>();
    }
    ppt = pair_ppt(ns);
    nblk = pair_tiles(ns, ppt);
    O3G_TRY(state.alloc(sizeof(IcpState)));
    const size_t acc_bytes = sizeof(unsigned long long) * kPartial * accum_rows(nblk);
    O3G_TRY(acc.alloc(acc_bytes));
    O3G_TRY(cudaMemsetAsync(acc.p, 0, acc_bytes, s));
    O3G_TRY(queue.alloc(sizeof(unsigned) * 2));
    O3G_TRY(cudaMemsetAsync(queue.p, 0, sizeof(unsigned) * 2, s));
    O3G_TRY(lists.alloc(kListBytes * (ns > 0 ? ns : 1)));
    O3G_TRY(cudaMemsetAsync(lists.p, 0xff, kListBytes * (ns > 0 ? ns : 1), s));  // no lists yet
    k_init_state<<<1, 32, 0, s>>>(state.as<IcpState>(), to_pose(T));
    count_launch();
    return O3G_OK;
  }
  int32_t launch(const o3g_grid* g, int ns, float r, double eps, int mode, int32_t* corr, float* d2,
                 cudaStream_t s, bool f64 = false, int kind = kPointToPlane, bool dependent = false) {
    PairDesc P;
    P.g = g->view();
    P.cell = g->cell;
    P.r = r;
    P.eps = stop_eps(eps);
    P.eps_tan2 = stop_tan2(eps);
    P.kind = kind;
    // the centre of the grid's box: near every point that can find a partner
    for (int k = 0; k < 3; ++k)
      P.ctr[k] = kind == kPointToPoint ? (static_cast<float>(g->lo[k]) + 0.5f * static_cast<float>(g->span[k])) * g->cell
                                       : 0.f;
    P.src4 = pts;
    P.ns = ns;
    P.ntiles = nblk;
    P.ppt = ppt;
    P.tile0 = 0;
    P.st = state.as<IcpState>();
    set_sums(P, g, acc.as<unsigned long long>());
    P.lists = (mode == kIterate || mode == kEvaluate) ? list_ref(lists.p, ns) : ListRef{nullptr, nullptr, nullptr, nullptr};
    P.list_motion = list_motion(ns, r);
    P.corr_out = corr;
    P.d2_out = d2;
    launch_iter(f64, nblk, P, nullptr, nullptr, nullptr, mode, s, dependent,
                TileQueue{queue.as<unsigned>(), launches & 1});
    ++launches;
    count_launch();
    return O3G_OK;
  }
};

}  // namespace

int32_t icp_run(const o3g_grid* g, const float* d_src, int64_t ns, int32_t stride, const double* init_T,
                double max_corr_dist, int32_t max_iter, double eps, double* out_T, double* out_fitness,
                double* out_rmse, int32_t* out_iters, cudaStream_t s, int32_t precision, bool point_to_point,
                const SortedCloud* pre, int32_t* d_corr, float* d_d2) {
  const char* fn = point_to_point ? "o3g_icp_point_to_point_grid" : "o3g_icp_point_to_plane_grid";
  const int kind = point_to_point ? kPointToPoint : kPointToPlane;
  if (precision != O3G_PREC_F32_COMPENSATED && precision != O3G_PREC_F64) {
    set_error("%s: unknown precision %d", fn, precision);
    return O3G_ERR_ARG;
  }
  const bool f64 = precision == O3G_PREC_F64;
  if (!g || !out_T || !out_fitness || !out_rmse || max_iter < 0 || !(max_corr_dist >= 0.0) ||
      !std::isfinite(max_corr_dist)) {
    set_error("%s: invalid argument", fn);
    return O3G_ERR_ARG;
  }
  O3G_TRY_STATUS(check_src(fn, d_src, ns, stride));
  if (!point_to_point && !g->has_normals) {
    set_error("%s: the target grid carries no normals (attach or estimate them first)", fn);
    return O3G_ERR_ARG;
  }
  if (!pose_ok(init_T)) {
    set_error("%s: init_T is null or not finite", fn);
    return O3G_ERR_NONFINITE;
  }
  const float r = static_cast<float>(max_corr_dist);
  Work w(s);
  O3G_TRY_STATUS(w.prepare(d_src, ns, stride, g->cell, init_T, s, pre));
  const int n = static_cast<int>(ns);
  for (int it = 0; it < max_iter; ++it) {
    TimedRegion tr(O3G_KERNEL_ICP_CORR, s);
    w.launch(g, n, r, eps, kIterate, nullptr, nullptr, s, f64, kind, it > 0);
  }
  w.launch(g, n, r, eps, kEvaluate, d_corr, d_d2, s, f64, kind, max_iter > 0);
  O3G_TRY(cudaGetLastError());
  IcpState h;
  int aux[8];
  O3G_TRY(cudaMemcpyAsync(&h, w.state.p, sizeof(IcpState), cudaMemcpyDeviceToHost, s));
  O3G_TRY(cudaMemcpyAsync(aux, w.aux, sizeof(aux), cudaMemcpyDeviceToHost, s));
  O3G_TRY(cudaStreamSynchronize(s));
  if (aux[6]) {
    set_error("%s: non-finite source coordinate", fn);
    return O3G_ERR_NONFINITE;
  }
  if (h.nonfinite) {
    set_error("%s: the update sums became non-finite", fn);
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

extern "C" int32_t o3g_normal_equations_ex(const o3g_grid* g, const float* d_src, int64_t ns, int32_t stride,
                                           const double* T, float max_corr_dist, int32_t precision, double* out_A,
                                           double* out_b, double* out_stats, void* stream) {
  const char* fn = "o3g_normal_equations";
  if (!g || !out_A || !out_b || !out_stats || !(max_corr_dist >= 0.f) || !std::isfinite(max_corr_dist) ||
      (precision != O3G_PREC_F32_COMPENSATED && precision != O3G_PREC_F64)) {
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
  w.launch(g, static_cast<int>(ns), max_corr_dist, 0.0, kEquations, nullptr, nullptr, s,
           precision == O3G_PREC_F64);
  O3G_TRY(cudaGetLastError());
  IcpState h;
  int aux[8];
  O3G_TRY(cudaMemcpyAsync(&h, w.state.p, sizeof(IcpState), cudaMemcpyDeviceToHost, s));
  O3G_TRY(cudaMemcpyAsync(aux, w.aux, sizeof(aux), cudaMemcpyDeviceToHost, s));
  O3G_TRY(cudaStreamSynchronize(s));
  if (aux[6]) {
    set_error("%s: non-finite source coordinate", fn);
    return O3G_ERR_NONFINITE;
  }
  if (h.nonfinite) {
    set_error("%s: a sum left its bound or was not finite (check the target normals)", fn);
    return O3G_ERR_NONFINITE;
  }
  for (int k = 0; k < 36; ++k) out_A[k] = h.A[k];
  for (int k = 0; k < 6; ++k) out_b[k] = h.b[k];
  for (int k = 0; k < 3; ++k) out_stats[k] = h.stats[k];
  return O3G_OK;
}

extern "C" int32_t o3g_normal_equations(const o3g_grid* g, const float* d_src, int64_t ns, int32_t stride,
                                        const double* T, float max_corr_dist, double* out_A, double* out_b,
                                        double* out_stats, void* stream) {
  return o3g_normal_equations_ex(g, d_src, ns, stride, T, max_corr_dist, O3G_PREC_F32_COMPENSATED, out_A, out_b,
                                 out_stats, stream);
}

extern "C" int32_t o3g_icp_point_to_plane_grid(const o3g_grid* g, const float* d_src, int64_t ns, int32_t stride,
                                               const double* init_T, double max_corr_dist, int32_t max_iter,
                                               double eps, double* out_T, double* out_fitness, double* out_rmse,
                                               int32_t* out_iters, void* stream) {
  return icp_run(g, d_src, ns, stride, init_T, max_corr_dist, max_iter, eps, out_T, out_fitness, out_rmse, out_iters,
                 static_cast<cudaStream_t>(stream), O3G_PREC_F32_COMPENSATED);
}

extern "C" int32_t o3g_icp_point_to_point_grid(const o3g_grid* g, const float* d_src, int64_t ns, int32_t stride,
                                               const double* init_T, double max_corr_dist, int32_t max_iter,
                                               double eps, double* out_T, double* out_fitness, double* out_rmse,
                                               int32_t* out_iters, void* stream) {
  return icp_run(g, d_src, ns, stride, init_T, max_corr_dist, max_iter, eps, out_T, out_fitness, out_rmse, out_iters,
                 static_cast<cudaStream_t>(stream), O3G_PREC_F32_COMPENSATED, true);
}

extern "C" int32_t o3g_icp_point_to_plane_grid_ex(const o3g_grid* g, const float* d_src, int64_t ns, int32_t stride,
                                                  const double* init_T, double max_corr_dist, int32_t max_iter,
                                                  double eps, int32_t precision, double* out_T, double* out_fitness,
                                                  double* out_rmse, int32_t* out_iters, void* stream) {
  return icp_run(g, d_src, ns, stride, init_T, max_corr_dist, max_iter, eps, out_T, out_fitness, out_rmse, out_iters,
                 static_cast<cudaStream_t>(stream), precision);
}

extern "C" int32_t o3g_icp_point_to_plane_grid_corr(const o3g_grid* g, const float* d_src, int64_t ns,
                                                    int32_t stride, const double* init_T, double max_corr_dist,
                                                    int32_t max_iter, double eps, int32_t precision, double* out_T,
                                                    double* out_fitness, double* out_rmse, int32_t* out_iters,
                                                    int32_t* d_corr, float* d_d2, void* stream) {
  if (ns > 0 && (!d_corr || !d_d2)) {
    set_error("o3g_icp_point_to_plane_grid_corr: the correspondence outputs are null");
    return O3G_ERR_ARG;
  }
  return icp_run(g, d_src, ns, stride, init_T, max_corr_dist, max_iter, eps, out_T, out_fitness, out_rmse, out_iters,
                 static_cast<cudaStream_t>(stream), precision, false, nullptr, d_corr, d_d2);
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
  O3G_TRY_STATUS(o3g_build_grid(d_tgt, nt, tgt_stride, static_cast<float>(max_corr_dist * 1.002), nullptr, &g));
  int32_t st = o3g_grid_set_normals(g, d_tgt_nrm, n_nrm, nrm_stride, nullptr);
  if (st >= 0)
    st = icp_run(g, d_src, ns, src_stride, init_T, max_corr_dist, max_iter, 0.0, out_T, out_fitness, out_rmse, nullptr,
                 nullptr, O3G_PREC_F32_COMPENSATED);
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
constexpr size_t kNaOffSrc = 0;
constexpr size_t kNaOffState = align256(kNaOffSrc + sizeof(float4) * static_cast<size_t>(O3G_NOALLOC_MAX_POINTS));
constexpr size_t kNaOffAcc = align256(kNaOffState + sizeof(IcpState));
constexpr size_t kNaOffFlag = align256(kNaOffAcc + sizeof(unsigned long long) * kPartial * kAccRows);
constexpr size_t kNaBytes = align256(kNaOffFlag + sizeof(int));
static_assert(kNaBytes == 4203520, "update the size stated in o3g.h");

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
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(base + kNaOffAcc);
  int* bad = reinterpret_cast<int*>(base + kNaOffFlag);
  const int n = static_cast<int>(ns);
  const int nblk = tiles_of(ns);
  // the accumulators and the input flag must start at zero; the state is rewritten by k_init_state
  O3G_TRY(cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * kPartial * accum_rows(nblk), s));
  O3G_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
  if (n > 0) {
    k_pack_src<<<(n + kThreads - 1) / kThreads, kThreads, 0, s>>>(d_src, n, stride, src4, bad);
    count_launch();
  }
  k_init_state<<<1, 32, 0, s>>>(st, to_pose(init_T));
  count_launch();
  const float r = static_cast<float>(max_corr_dist);
  const GridView gv = g->view();
  for (int it = 0; it <= max_iter; ++it) {
    const int mode = it < max_iter ? kIterate : kEvaluate;
    PairDesc P;
    P.g = gv;
    P.cell = g->cell;
    P.r = r;
    P.eps = stop_eps(eps);
    P.eps_tan2 = stop_tan2(eps);
    P.kind = kPointToPlane;
    P.ctr[0] = P.ctr[1] = P.ctr[2] = 0.f;
    P.src4 = src4;
    P.ns = n;
    P.ntiles = nblk;
    P.ppt = 1;
    P.tile0 = 0;
    P.st = st;
    set_sums(P, g, acc);
    P.lists = ListRef{nullptr, nullptr, nullptr, nullptr};
    P.list_motion = -1.f;
    P.corr_out = nullptr;
    P.d2_out = nullptr;
    launch_iter(false, nblk, P, nullptr, nullptr, nullptr, mode, s);
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

// ---------------------------------------------------------------------------
// Batched point-to-plane ICP: many independent registrations advance together,
// one persistent launch per iteration over the (pair, tile) work items of all
// pairs; the iteration sequence is captured once as a CUDA graph and launched.

namespace o3g {
namespace {

std::mutex g_graph_mutex;
cudaStream_t g_graph_stream[kNaMaxDevices] = {};
cudaStream_t g_side_stream[kNaMaxDevices] = {};

// A non-blocking stream of the library per device, used to capture graphs
// (the legacy default stream cannot be captured).
cudaError_t graph_stream(cudaStream_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_graph_mutex);
  if (!g_graph_stream[dev]) {
    e = cudaStreamCreateWithFlags(&g_graph_stream[dev], cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
  }
  *out = g_graph_stream[dev];
  return cudaSuccess;
}

// Launches `iters` iteration steps and one evaluation step of the batch on s,
// through a captured CUDA graph when capture works, else directly.
int32_t run_iterations(const PairDesc* descs, const int* tile_pair, const int* d_ntiles, int ntiles, int max_iter,
                       double eps, unsigned* queue, cudaStream_t s) {
  PairDesc dummy{};
  auto enqueue = [&](cudaStream_t q) {
    for (int it = 0; it <= max_iter; ++it)
      launch_iter(false, ntiles, dummy, descs, tile_pair, d_ntiles, it < max_iter ? kIterate : kEvaluate, q, false,
                  TileQueue{queue, it & 1});
  };
  cudaStream_t cs = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool ok = graph_stream(&cs) == cudaSuccess && cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming) == cudaSuccess;
  if (ok) {
    ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      enqueue(cs);
      ok = cudaStreamEndCapture(cs, &graph) == cudaSuccess && graph != nullptr;
    }
    ok = ok && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    ok = ok && cudaEventRecord(ev_in, s) == cudaSuccess && cudaStreamWaitEvent(cs, ev_in, 0) == cudaSuccess &&
         cudaGraphLaunch(exec, cs) == cudaSuccess && cudaEventRecord(ev_out, cs) == cudaSuccess &&
         cudaStreamWaitEvent(s, ev_out, 0) == cudaSuccess;
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (ev_in) cudaEventDestroy(ev_in);
  if (ev_out) cudaEventDestroy(ev_out);
  if (!ok) {
    (void)cudaGetLastError();
    enqueue(s);  // capture unavailable: plain launches, same work
  }
  count_launch(max_iter + 1);
  O3G_TRY(cudaGetLastError());
  return O3G_OK;
}

}  // namespace

// A library-owned non-blocking stream per device for work that runs beside the
// caller's stream (the source sort of the combined registration entry points).
cudaError_t side_stream(cudaStream_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_graph_mutex);
  if (!g_side_stream[dev]) {
    e = cudaStreamCreateWithFlags(&g_side_stream[dev], cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
  }
  *out = g_side_stream[dev];
  return cudaSuccess;
}
}  // namespace o3g

extern "C" int32_t o3g_icp_point_to_plane_batch(int32_t n_pairs, const o3g_grid* const* tgts, const float* const* d_src,
                                                const int64_t* ns, const int32_t* strides, const double* init_T,
                                                const double* max_corr_dist, int32_t max_iter, double eps,
                                                double* out_T, double* out_fitness, double* out_rmse,
                                                int32_t* out_iters, int32_t* out_status, void* stream) {
  using namespace o3g;
  const char* fn = "o3g_icp_point_to_plane_batch";
  if (n_pairs < 0 || max_iter < 0 || (n_pairs > 0 && (!tgts || !d_src || !ns || !strides || !init_T ||
                                                       !max_corr_dist || !out_T || !out_fitness || !out_rmse ||
                                                       !out_iters || !out_status))) {
    set_error("%s: invalid argument", fn);
    return O3G_ERR_ARG;
  }
  if (n_pairs == 0) return O3G_OK;
  std::vector<int64_t> off(n_pairs + 1, 0);
  std::vector<int> ntiles(n_pairs), ppts(n_pairs);
  int64_t tiles_total = 0, rows_total = 0;
  for (int p = 0; p < n_pairs; ++p) {
    if (!tgts[p] || !tgts[p]->has_normals || !(max_corr_dist[p] >= 0.0) || !std::isfinite(max_corr_dist[p])) {
      set_error("%s: pair %d: missing target grid, target normals or a valid max_corr_dist", fn, p);
      return O3G_ERR_ARG;
    }
    O3G_TRY_STATUS(check_src(fn, d_src[p], ns[p], strides[p]));
    if (!pose_ok(init_T + 16 * p)) {
      set_error("%s: pair %d: init_T is not finite", fn, p);
      return O3G_ERR_NONFINITE;
    }
    off[p + 1] = off[p] + ns[p];
    ppts[p] = pair_ppt(ns[p]);
    ntiles[p] = pair_tiles(ns[p], ppts[p]);
    tiles_total += ntiles[p];
    rows_total += accum_rows(ntiles[p]);
  }
  if (off[n_pairs] > 0x7fffffffLL - kThreads || tiles_total > 0x7fffffffLL) {
    set_error("%s: %lld source points in total exceed the supported size", fn, static_cast<long long>(off[n_pairs]));
    return O3G_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t total = off[n_pairs];
  DevBuf d_ptrs(s), d_strides(s), d_off(s), d_src4(s), d_aux(s), d_states(s), d_acc(s), d_cnt(s), d_lists(s),
      d_descs(s), d_tiles(s), d_poses(s);
  O3G_TRY(d_ptrs.alloc(sizeof(float*) * n_pairs));
  O3G_TRY(d_strides.alloc(sizeof(int32_t) * n_pairs));
  O3G_TRY(d_off.alloc(sizeof(int64_t) * (n_pairs + 1)));
  O3G_TRY(d_src4.alloc(sizeof(float4) * (total > 0 ? total : 1)));
  O3G_TRY(d_aux.alloc(sizeof(int) * 8 * n_pairs));
  O3G_TRY(d_states.alloc(sizeof(IcpState) * n_pairs));
  O3G_TRY(d_acc.alloc(sizeof(unsigned long long) * kPartial * rows_total));
  O3G_TRY(d_cnt.alloc(sizeof(unsigned) * 2));  // the tile queue
  O3G_TRY(d_lists.alloc(kListBytes * (total > 0 ? total : 1)));
  O3G_TRY(d_descs.alloc(sizeof(PairDesc) * n_pairs));
  O3G_TRY(d_tiles.alloc(sizeof(int) * (tiles_total + 1)));
  O3G_TRY(d_poses.alloc(sizeof(double) * 16 * n_pairs));
  // host-side tables
  std::vector<PairDesc> descs(n_pairs);
  std::vector<int> tile_pair(tiles_total + 1);
  IcpState* states = d_states.as<IcpState>();
  unsigned long long* acc = d_acc.as<unsigned long long>();
  int64_t t0 = 0, a0 = 0;
  for (int p = 0; p < n_pairs; ++p) {
    PairDesc& P = descs[p];
    P.g = tgts[p]->view();
    P.cell = tgts[p]->cell;
    P.r = static_cast<float>(max_corr_dist[p]);
    P.eps = stop_eps(eps);
    P.eps_tan2 = stop_tan2(eps);
    P.kind = kPointToPlane;
    P.ctr[0] = P.ctr[1] = P.ctr[2] = 0.f;
    P.src4 = d_src4.as<float4>() + off[p];
    P.ns = static_cast<int>(ns[p]);
    P.ntiles = ntiles[p];
    P.ppt = ppts[p];
    P.tile0 = static_cast<int>(t0);
    P.st = states + p;
    set_sums(P, tgts[p], acc + static_cast<size_t>(kPartial) * a0);
    P.lists = list_ref(static_cast<unsigned char*>(d_lists.p) + kListBytes * off[p], ns[p]);
    P.list_motion = list_motion(ns[p], P.r);
    P.corr_out = nullptr;
    P.d2_out = nullptr;
    for (int k = 0; k < ntiles[p]; ++k) tile_pair[t0 + k] = p;
    t0 += ntiles[p];
    a0 += P.nacc;
  }
  tile_pair[tiles_total] = static_cast<int>(tiles_total);  // read by the kernel as the tile count
  std::vector<int32_t> h_strides(strides, strides + n_pairs);
  O3G_TRY(cudaMemcpyAsync(d_ptrs.p, d_src, sizeof(float*) * n_pairs, cudaMemcpyHostToDevice, s));
  O3G_TRY(cudaMemcpyAsync(d_strides.p, h_strides.data(), sizeof(int32_t) * n_pairs, cudaMemcpyHostToDevice, s));
  O3G_TRY(cudaMemcpyAsync(d_off.p, off.data(), sizeof(int64_t) * (n_pairs + 1), cudaMemcpyHostToDevice, s));
  O3G_TRY(cudaMemcpyAsync(d_descs.p, descs.data(), sizeof(PairDesc) * n_pairs, cudaMemcpyHostToDevice, s));
  O3G_TRY(cudaMemcpyAsync(d_tiles.p, tile_pair.data(), sizeof(int) * (tiles_total + 1), cudaMemcpyHostToDevice, s));
  O3G_TRY(cudaMemcpyAsync(d_poses.p, init_T, sizeof(double) * 16 * n_pairs, cudaMemcpyHostToDevice, s));
  O3G_TRY(cudaMemsetAsync(d_cnt.p, 0, sizeof(unsigned) * 2, s));
  O3G_TRY(cudaMemsetAsync(d_acc.p, 0, sizeof(unsigned long long) * kPartial * rows_total, s));
  O3G_TRY(cudaMemsetAsync(d_lists.p, 0xff, kListBytes * (total > 0 ? total : 1), s));
  O3G_TRY_STATUS(sort_clouds_batch(reinterpret_cast<const float* const*>(d_ptrs.p), d_strides.as<int32_t>(),
                                   d_off.as<int64_t>(), n_pairs, total, s, d_src4.as<float4>(), d_aux.as<int>()));
  k_init_states<<<(n_pairs + 127) / 128, 128, 0, s>>>(states, d_poses.as<double>(), n_pairs);
  count_launch();
  {
    TimedRegion tr(O3G_KERNEL_ICP_BATCH, s);
    O3G_TRY_STATUS(run_iterations(d_descs.as<PairDesc>(), d_tiles.as<int>(), d_tiles.as<int>() + tiles_total,
                                  static_cast<int>(tiles_total), max_iter, eps, d_cnt.as<unsigned>(), s));
  }
  std::vector<IcpState> h(n_pairs);
  std::vector<int> aux(8 * n_pairs);
  O3G_TRY(cudaMemcpyAsync(h.data(), states, sizeof(IcpState) * n_pairs, cudaMemcpyDeviceToHost, s));
  O3G_TRY(cudaMemcpyAsync(aux.data(), d_aux.p, sizeof(int) * 8 * n_pairs, cudaMemcpyDeviceToHost, s));
  O3G_TRY(cudaStreamSynchronize(s));
  for (int p = 0; p < n_pairs; ++p) {
    for (int k = 0; k < 16; ++k) out_T[16 * p + k] = h[p].T[k];
    out_fitness[p] = h[p].fitness;
    out_rmse[p] = h[p].rmse;
    out_iters[p] = h[p].iters;
    out_status[p] = aux[8 * p + 6] || h[p].nonfinite ? O3G_ERR_NONFINITE
                    : h[p].few_corr                  ? O3G_WARN_FEW_CORR
                    : h[p].degenerate                ? O3G_WARN_DEGENERATE
                                                     : O3G_OK;
  }
  return O3G_OK;
}

// ---------------------------------------------------------------------------
// Serving: a request loop with continuous batching.  Requests wait in a queue
// until a slot and the device-memory budget allow their admission (host copy to
// device, target grid, normals, source layout, state); every step advances all
// admitted requests by one iteration in a single persistent launch and retires
// the ones that have finished (evaluation launch, results kept for polling).
// A request's arithmetic, order and tiling are those of the single-pair entry
// points, so its result does not depend on what else is being served.

struct o3g_server {
  struct Request {
    int64_t id;
    std::vector<float> src, tgt, nrm;
    float normal_radius;
    int normal_max_nn;
    double T0[16];
    double r;
    int max_iter;
    double eps;
  };
  struct Slot {
    bool used = false;
    int64_t id = -1;
    o3g_grid* grid = nullptr;
    float4* src4 = nullptr;
    int* src_aux = nullptr;
    void* lists = nullptr;  // candidate lists (kListBytes per source point)
    unsigned long long* acc = nullptr;  // accum_rows(ntiles) x kPartial fixed-point sums
    int ns = 0, ntiles = 1, ppt = 1;
    int max_iter = 0;
    double eps = 0.0;
    float r = 0.f;
    int64_t bytes = 0;
    int iters = 0;
    bool done = false;
    bool fresh = false;  // admitted in the current step (its first launches come in the next)
  };
  struct Result {
    int32_t status;
    double T[16];
    double fitness, rmse;
    int32_t iters;
  };
  cudaStream_t s = nullptr;   // the stream the iterations run on (the caller's)
  cudaStream_t as = nullptr;  // the library's admission stream
  cudaEvent_t admitted = nullptr;  // recorded on `as` after admissions; `s` waits for it
  int max_active = 0;
  int64_t budget = 0, used = 0;
  int64_t next_id = 0;
  std::deque<Request> waiting;
  std::vector<Slot> slots;
  void* states = nullptr;   // max_active IcpState, slot-indexed
  void* descs = nullptr;    // max_active PairDesc
  int* tiles = nullptr;     // tile table (+1 count), grows
  int64_t tiles_cap = 0;
  unsigned* queue = nullptr;  // the dynamic tile queue of the server's launches (2 counters)
  int64_t launches = 0;
  std::map<int64_t, Result> finished;
};

namespace o3g {
namespace {

// Device memory a request will hold while admitted (upper bound before its grid exists).
int64_t request_bytes(int64_t ns, int64_t nt) {
  const int64_t rows = accum_rows(tiles_of(ns));
  return ns * (16 + static_cast<int64_t>(kListBytes) + 12) + rows * kPartial * 8 + nt * (16 + 16 + 4 + 12 + 12) +
         4 * (32 * nt + (1 << 20)) + sizeof(IcpState);
}

void release_slot(o3g_server* sv, o3g_server::Slot& sl) {
  if (sl.grid) o3g_free_grid(sl.grid);
  dfree(sl.src4, sv->s);
  dfree(sl.src_aux, sv->s);
  dfree(sl.lists, sv->s);
  dfree(sl.acc, sv->s);
  sv->used -= sl.bytes;
  sl = o3g_server::Slot();
}

// Admission of one request into free slot k (device copies, grid, normals, layout, state).
int32_t admit(o3g_server* sv, int k, o3g_server::Request& rq) {
  cudaStream_t s = sv->as;  // the admission stream: copies, grid, normals and sort overlap the iterations
  o3g_server::Slot& sl = sv->slots[k];
  const int64_t ns = static_cast<int64_t>(rq.src.size() / 3), nt = static_cast<int64_t>(rq.tgt.size() / 3);
  sl.used = true;
  sl.id = rq.id;
  sl.ns = static_cast<int>(ns);
  sl.ppt = pair_ppt(ns);
  sl.ntiles = pair_tiles(ns, sl.ppt);
  sl.max_iter = rq.max_iter;
  sl.eps = rq.eps;
  sl.r = static_cast<float>(rq.r);
  sl.bytes = request_bytes(ns, nt);
  sv->used += sl.bytes;
  DevBuf d_src(s), d_tgt(s), d_nrm(s);
  O3G_TRY(d_src.alloc(sizeof(float) * 3 * (ns > 0 ? ns : 1)));
  O3G_TRY(d_tgt.alloc(sizeof(float) * 3 * (nt > 0 ? nt : 1)));
  if (ns > 0) O3G_TRY(cudaMemcpyAsync(d_src.p, rq.src.data(), sizeof(float) * 3 * ns, cudaMemcpyHostToDevice, s));
  if (nt > 0) O3G_TRY(cudaMemcpyAsync(d_tgt.p, rq.tgt.data(), sizeof(float) * 3 * nt, cudaMemcpyHostToDevice, s));
  O3G_TRY_STATUS(o3g_build_grid(d_tgt.as<float>(), nt, 3, static_cast<float>(rq.r * 1.002), s, &sl.grid));
  if (!rq.nrm.empty()) {
    O3G_TRY(d_nrm.alloc(sizeof(float) * 3 * (nt > 0 ? nt : 1)));
    if (nt > 0) O3G_TRY(cudaMemcpyAsync(d_nrm.p, rq.nrm.data(), sizeof(float) * 3 * nt, cudaMemcpyHostToDevice, s));
    O3G_TRY_STATUS(o3g_grid_set_normals(sl.grid, d_nrm.as<float>(), nt, 3, s));
  } else {
    O3G_TRY_STATUS(estimate_normals_impl(sl.grid, rq.normal_radius, rq.normal_max_nn, nullptr, nullptr, 3, s));
  }
  SortedCloud sc(s);
  O3G_TRY_STATUS(sort_cloud(d_src.as<float>(), ns, 3, s, &sc));
  sl.src4 = sc.pts;
  sl.src_aux = sc.aux.as<int>();
  sc.buf.p = nullptr;  // now owned by the slot
  sc.aux.p = nullptr;
  O3G_TRY(dmalloc(&sl.lists, kListBytes * (ns > 0 ? ns : 1), s));
  O3G_TRY(cudaMemsetAsync(sl.lists, 0xff, kListBytes * (ns > 0 ? ns : 1), s));
  const size_t acc_bytes = sizeof(unsigned long long) * kPartial * accum_rows(sl.ntiles);
  O3G_TRY(dmalloc(reinterpret_cast<void**>(&sl.acc), acc_bytes, s));
  O3G_TRY(cudaMemsetAsync(sl.acc, 0, acc_bytes, s));
  k_init_state<<<1, 32, 0, s>>>(static_cast<IcpState*>(sv->states) + k, to_pose(rq.T0), rq.max_iter);
  count_launch();
  O3G_TRY(cudaGetLastError());
  sl.iters = 0;
  sl.done = false;
  return O3G_OK;
}

PairDesc slot_desc(o3g_server* sv, int k, int tile0) {
  o3g_server::Slot& sl = sv->slots[k];
  PairDesc P;
  P.g = sl.grid->view();
  P.cell = sl.grid->cell;
  P.r = sl.r;
  P.eps = stop_eps(sl.eps);
  P.eps_tan2 = stop_tan2(sl.eps);
  P.kind = kPointToPlane;
  P.ctr[0] = P.ctr[1] = P.ctr[2] = 0.f;
  P.src4 = sl.src4;
  P.ns = sl.ns;
  P.ntiles = sl.ntiles;
  P.ppt = sl.ppt;
  P.tile0 = tile0;
  P.st = static_cast<IcpState*>(sv->states) + k;
  set_sums(P, sl.grid, sl.acc);
  P.lists = list_ref(sl.lists, sl.ns);
  P.list_motion = list_motion(sl.ns, sl.r);
  P.corr_out = nullptr;
  P.d2_out = nullptr;
  return P;
}

// Launches per o3g_server_step (stages every admitted request advances by).
constexpr int kServeStages = 8;

// `launches` launches of `mode` over the given slots (after the first, each as a
// programmatic dependent of the one before).
int32_t launch_slots(o3g_server* sv, const std::vector<int>& ks, int mode, int launches = 1) {
  cudaStream_t s = sv->s;
  std::vector<PairDesc> d;
  std::vector<int> tiles;
  int64_t t0 = 0;
  for (int k : ks) {
    d.push_back(slot_desc(sv, k, static_cast<int>(t0)));
    for (int j = 0; j < sv->slots[k].ntiles; ++j) tiles.push_back(static_cast<int>(d.size() - 1));
    t0 += sv->slots[k].ntiles;
  }
  tiles.push_back(static_cast<int>(t0));
  if (static_cast<int64_t>(tiles.size()) > sv->tiles_cap) {
    dfree(sv->tiles, s);
    sv->tiles = nullptr;
    sv->tiles_cap = static_cast<int64_t>(tiles.size()) * 2;
    O3G_TRY(dmalloc(reinterpret_cast<void**>(&sv->tiles), sizeof(int) * sv->tiles_cap, s));
  }
  O3G_TRY(cudaMemcpyAsync(sv->descs, d.data(), sizeof(PairDesc) * d.size(), cudaMemcpyHostToDevice, s));
  O3G_TRY(cudaMemcpyAsync(sv->tiles, tiles.data(), sizeof(int) * tiles.size(), cudaMemcpyHostToDevice, s));
  PairDesc dummy{};
  for (int l = 0; l < launches; ++l) {
    launch_iter(false, static_cast<int>(t0), dummy, static_cast<const PairDesc*>(sv->descs), sv->tiles,
                sv->tiles + t0, mode, s, l > 0, TileQueue{sv->queue, static_cast<int>(sv->launches & 1)});
    ++sv->launches;
    count_launch();
  }
  O3G_TRY(cudaGetLastError());
  return O3G_OK;
}

}  // namespace
}  // namespace o3g

extern "C" int64_t o3g_server_request_bytes(int64_t ns, int64_t nt) {
  if (ns < 0 || nt < 0 || ns > 0x7fffffffLL || nt > 0x7fffffffLL) return -1;
  return o3g::request_bytes(ns, nt);
}

extern "C" int32_t o3g_server_create(int32_t max_active, int64_t hbm_budget_bytes, void* stream, o3g_server** out) {
  using namespace o3g;
  if (!out || max_active < 1 || max_active > 65536 || hbm_budget_bytes <= 0) {
    set_error("o3g_server_create: invalid argument");
    return O3G_ERR_ARG;
  }
  *out = nullptr;
  o3g_server* sv = new (std::nothrow) o3g_server();
  if (!sv) {
    set_error("o3g_server_create: host allocation failed");
    return O3G_ERR_OOM;
  }
  sv->s = static_cast<cudaStream_t>(stream);
  if (cudaStreamCreateWithFlags(&sv->as, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&sv->admitted, cudaEventDisableTiming) != cudaSuccess) {
    if (sv->as) cudaStreamDestroy(sv->as);
    delete sv;
    return cuda_fail(cudaGetLastError(), "o3g_server_create");
  }
  sv->max_active = max_active;
  sv->budget = hbm_budget_bytes;
  sv->slots.resize(max_active);
  cudaError_t e = dmalloc(&sv->states, sizeof(IcpState) * max_active, sv->s);
  if (e == cudaSuccess) e = dmalloc(&sv->descs, sizeof(PairDesc) * max_active, sv->s);
  if (e == cudaSuccess) e = dmalloc(reinterpret_cast<void**>(&sv->queue), sizeof(unsigned) * 2, sv->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(sv->queue, 0, sizeof(unsigned) * 2, sv->s);
  if (e != cudaSuccess) {
    dfree(sv->states, sv->s);
    dfree(sv->descs, sv->s);
    dfree(sv->queue, sv->s);
    (void)cudaStreamSynchronize(sv->s);
    cudaEventDestroy(sv->admitted);
    cudaStreamDestroy(sv->as);
    delete sv;
    return cuda_fail(e, "o3g_server_create");
  }
  *out = sv;
  return O3G_OK;
}

extern "C" int32_t o3g_server_destroy(o3g_server* sv) {
  using namespace o3g;
  if (!sv) return O3G_OK;
  for (auto& sl : sv->slots)
    if (sl.used) release_slot(sv, sl);
  dfree(sv->states, sv->s);
  dfree(sv->descs, sv->s);
  dfree(sv->tiles, sv->s);
  dfree(sv->queue, sv->s);
  (void)cudaStreamSynchronize(sv->as);
  (void)cudaStreamSynchronize(sv->s);
  cudaEventDestroy(sv->admitted);
  cudaStreamDestroy(sv->as);
  delete sv;
  return O3G_OK;
}

extern "C" int32_t o3g_server_submit(o3g_server* sv, const float* h_src, int64_t ns, const float* h_tgt, int64_t nt,
                                     const float* h_tgt_nrm, float normal_radius, int32_t normal_max_nn,
                                     const double* init_T, double max_corr_dist, int32_t max_iter, double eps,
                                     int64_t* out_id) {
  using namespace o3g;
  const char* fn = "o3g_server_submit";
  if (!sv || !out_id || ns < 0 || nt < 0 || ns > 0x7fffffffLL - kThreads || nt > 0x7fffffffLL - 4096 ||
      (ns > 0 && !h_src) || (nt > 0 && !h_tgt) || max_iter < 0 || !(max_corr_dist > 0.0) ||
      !std::isfinite(max_corr_dist) ||
      (!h_tgt_nrm && (normal_max_nn < 1 || normal_max_nn > O3G_MAX_NN || !(normal_radius >= 0.f)))) {
    set_error("%s: invalid argument", fn);
    return O3G_ERR_ARG;
  }
  if (!pose_ok(init_T)) {
    set_error("%s: init_T is null or not finite", fn);
    return O3G_ERR_NONFINITE;
  }
  if (request_bytes(ns, nt) > sv->budget) {
    set_error("%s: the request needs more device memory (%lld bytes) than the whole budget", fn,
              static_cast<long long>(request_bytes(ns, nt)));
    return O3G_ERR_OOM;
  }
  o3g_server::Request rq;
  rq.id = sv->next_id++;
  rq.src.assign(h_src, h_src + 3 * ns);
  rq.tgt.assign(h_tgt, h_tgt + 3 * nt);
  if (h_tgt_nrm) rq.nrm.assign(h_tgt_nrm, h_tgt_nrm + 3 * nt);
  rq.normal_radius = normal_radius;
  rq.normal_max_nn = normal_max_nn;
  for (int k = 0; k < 16; ++k) rq.T0[k] = init_T[k];
  rq.r = max_corr_dist;
  rq.max_iter = max_iter;
  rq.eps = eps;
  sv->waiting.push_back(std::move(rq));
  *out_id = sv->waiting.back().id;
  return O3G_OK;
}

extern "C" int32_t o3g_server_step(o3g_server* sv, int32_t* out_active, int32_t* out_waiting, int32_t* out_completed) {
  using namespace o3g;
  if (!sv) {
    set_error("o3g_server_step: server is null");
    return O3G_ERR_ARG;
  }
  cudaStream_t s = sv->s;
  // kServeStages launches over the requests admitted in earlier steps, each
  // launch advancing every one by one stage of its own (an iteration, or the
  // evaluation after the last one); the admissions of this step run on the
  // admission stream while they execute, and join in the next step
  std::vector<int> active_slots;
  for (int k = 0; k < sv->max_active; ++k)
    if (sv->slots[k].used && !sv->slots[k].fresh) active_slots.push_back(k);
  if (!active_slots.empty()) O3G_TRY_STATUS(launch_slots(sv, active_slots, kServe, kServeStages));
  bool admitted = false;
  // admit while a slot is free and the budget allows (first come, first served)
  while (!sv->waiting.empty()) {
    int k = -1;
    for (int j = 0; j < sv->max_active; ++j)
      if (!sv->slots[j].used) {
        k = j;
        break;
      }
    o3g_server::Request& rq = sv->waiting.front();
    const int64_t need = request_bytes(static_cast<int64_t>(rq.src.size() / 3), static_cast<int64_t>(rq.tgt.size() / 3));
    if (k < 0 || sv->used + need > sv->budget) break;
    const int32_t st = admit(sv, k, rq);
    admitted = true;
    if (st < 0) {
      release_slot(sv, sv->slots[k]);
      o3g_server::Result res{};
      res.status = st;
      sv->finished[rq.id] = res;
      sv->waiting.pop_front();
      continue;
    }
    sv->slots[k].fresh = true;
    sv->waiting.pop_front();
  }
  // later launches see the requests admitted so far
  if (admitted) {
    O3G_TRY(cudaEventRecord(sv->admitted, sv->as));
    O3G_TRY(cudaStreamWaitEvent(s, sv->admitted, 0));
  }
  if (active_slots.empty()) {  // nothing was running: the new requests start at once
    for (int k = 0; k < sv->max_active; ++k)
      if (sv->slots[k].used && sv->slots[k].fresh) {
        sv->slots[k].fresh = false;
        active_slots.push_back(k);
      }
    if (!active_slots.empty()) O3G_TRY_STATUS(launch_slots(sv, active_slots, kServe, kServeStages));
  }
  for (auto& sl : sv->slots) sl.fresh = false;
  int completed = 0;
  if (!active_slots.empty()) {
    std::vector<IcpState> h(sv->max_active);
    O3G_TRY(cudaMemcpyAsync(h.data(), sv->states, sizeof(IcpState) * sv->max_active, cudaMemcpyDeviceToHost, s));
    O3G_TRY(cudaStreamSynchronize(s));
    std::vector<int> finishing;
    for (int k : active_slots) {
      auto& sl = sv->slots[k];
      sl.iters = h[k].iters;
      sl.done = h[k].done != 0;
      if (h[k].phase >= 2) finishing.push_back(k);
    }
    if (!finishing.empty()) {
      std::vector<int> aux(8 * sv->max_active, 0);
      for (int k : finishing)
        O3G_TRY(cudaMemcpyAsync(aux.data() + 8 * k, sv->slots[k].src_aux, sizeof(int) * 8, cudaMemcpyDeviceToHost, s));
      O3G_TRY(cudaStreamSynchronize(s));
      for (int k : finishing) {
        auto& sl = sv->slots[k];
        o3g_server::Result res;
        for (int q = 0; q < 16; ++q) res.T[q] = h[k].T[q];
        res.fitness = h[k].fitness;
        res.rmse = h[k].rmse;
        res.iters = h[k].iters;
        res.status = aux[8 * k + 6] || h[k].nonfinite ? O3G_ERR_NONFINITE
                     : h[k].few_corr                  ? O3G_WARN_FEW_CORR
                     : h[k].degenerate                ? O3G_WARN_DEGENERATE
                                                      : O3G_OK;
        sv->finished[sl.id] = res;
        release_slot(sv, sl);
        ++completed;
      }
    }
  }
  int active = 0;
  for (const auto& sl : sv->slots) active += sl.used;
  if (out_active) *out_active = active;
  if (out_waiting) *out_waiting = static_cast<int32_t>(sv->waiting.size());
  if (out_completed) *out_completed = completed;
  return O3G_OK;
}

extern "C" int32_t o3g_server_poll(o3g_server* sv, int64_t id, int32_t* out_done, double* out_T, double* out_fitness,
                                   double* out_rmse, int32_t* out_iters, int32_t* out_status) {
  using namespace o3g;
  if (!sv || !out_done) {
    set_error("o3g_server_poll: invalid argument");
    return O3G_ERR_ARG;
  }
  auto it = sv->finished.find(id);
  if (it == sv->finished.end()) {
    if (id < 0 || id >= sv->next_id) {
      set_error("o3g_server_poll: unknown request %lld", static_cast<long long>(id));
      return O3G_ERR_ARG;
    }
    *out_done = 0;
    return O3G_OK;
  }
  const auto& r = it->second;
  *out_done = 1;
  if (out_T)
    for (int k = 0; k < 16; ++k) out_T[k] = r.T[k];
  if (out_fitness) *out_fitness = r.fitness;
  if (out_rmse) *out_rmse = r.rmse;
  if (out_iters) *out_iters = r.iters;
  if (out_status) *out_status = r.status;
  sv->finished.erase(it);
  return O3G_OK;
}

extern "C" int32_t o3g_server_completed(o3g_server* sv, int64_t* ids, int32_t cap, int32_t* out_n) {
  using namespace o3g;
  if (!sv || !out_n || cap < 0 || (cap > 0 && !ids)) {
    set_error("o3g_server_completed: invalid argument");
    return O3G_ERR_ARG;
  }
  int32_t n = 0;
  for (const auto& kv : sv->finished) {
    if (n >= cap) break;
    ids[n++] = kv.first;
  }
  *out_n = n;
  return O3G_OK;
}

// ---------------------------------------------------------------------------
// Hypothesis validation: fitness and inlier rmse of the whole source at many
// candidate poses against one target grid (the check RANSAC spends its time
// in, Sec. 3.3).  One persistent launch walks the (pose, tile) work items; each
// block runs the exact correspondence search of the ICP kernel for its tile at
// its pose and stores (|C|, sum d2) for the tile; a second launch sums each
// pose's tiles in fixed order on one warp.

namespace o3g {
namespace {

struct PoseF {
  float R[9], t[3];
};

__global__ void k_pose_round(const double* __restrict__ poses, int n, PoseF* __restrict__ out) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= n) return;
  const double* T = poses + 16 * static_cast<size_t>(h);
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) out[h].R[3 * r + c] = __double2float_rn(T[4 * r + c]);
    out[h].t[r] = __double2float_rn(T[4 * r + 3]);
  }
}

template <class Cfg>
__global__ void __launch_bounds__(kThreads, Cfg::kMinBlocks) k_eval_poses(GridView g, float cell, float r,
                                                             const float4* __restrict__ src4, int ns, int ntiles,
                                                             const PoseF* __restrict__ poses, int n_poses,
                                                             double* __restrict__ partials) {
  __shared__ Stage<Cfg> stage;
  __shared__ double ws[kThreads / 32][2];
  const int64_t items = static_cast<int64_t>(ntiles) * n_poses;
  const float r2 = __fmul_rn(r, r);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
    const int h = static_cast<int>(item / ntiles), j = static_cast<int>(item % ntiles);
    float R[9], t[3];
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = poses[h].R[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) t[k] = poses[h].t[k];
    const int i = j * kThreads + threadIdx.x;
    const bool live = i < ns;
    const float4 s = live ? src4[i] : make_float4(3.0e38f, 3.0e38f, 3.0e38f, 0.f);
    const float3 p = live ? xform_rn(R, t, s.x, s.y, s.z) : make_float3(3.0e38f, 3.0e38f, 3.0e38f);
    NnSink ns{Nearest{r2, 0x7fffffff, -1}};
    if (!staged_search(g, cell, p.x, p.y, p.z, r, live, ns, stage) && live)
      box_search_global(g, cell, p.x, p.y, p.z, r, ns);
    const Nearest nb = ns.nb;
    double cnt = (live && nb.pos >= 0) ? 1.0 : 0.0;
    double d2 = (live && nb.pos >= 0) ? static_cast<double>(nb.d2) : 0.0;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
      d2 += __shfl_xor_sync(0xffffffffu, d2, off);
    }
    if (lane == 0) {
      ws[warp][0] = cnt;
      ws[warp][1] = d2;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
      double v = ws[0][threadIdx.x];
      for (int w = 1; w < kThreads / 32; ++w) v += ws[w][threadIdx.x];
      partials[2 * static_cast<size_t>(item) + threadIdx.x] = v;
    }
    __syncthreads();
  }
}

// One warp per pose: the pose's tiles summed in fixed order (lane l takes tiles
// l, l + 32, ... in order, then a butterfly over lanes).
__global__ void k_eval_sum(const double* __restrict__ partials, int ntiles, int n_poses, int ns,
                           double* __restrict__ out) {
  const int h = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (h >= n_poses) return;
  double cnt = 0.0, d2 = 0.0;
  for (int j = lane; j < ntiles; j += 32) {
    const size_t k = 2 * (static_cast<size_t>(h) * ntiles + j);
    cnt += partials[k];
    d2 += partials[k + 1];
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
    d2 += __shfl_xor_sync(0xffffffffu, d2, off);
  }
  if (lane == 0) {
    out[3 * static_cast<size_t>(h) + 0] = ns > 0 ? cnt / static_cast<double>(ns) : 0.0;
    out[3 * static_cast<size_t>(h) + 1] = cnt > 0.0 ? sqrt(d2 / cnt) : 0.0;
    out[3 * static_cast<size_t>(h) + 2] = cnt;
  }
}

template <class Cfg>
int eval_resident() {
  static const int resident = [] {
    int dev = 0, sms = kNumSMs, per_sm = 1;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_eval_poses<Cfg>, kThreads, 0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    (void)cudaGetLastError();
    return sms * per_sm;
  }();
  return resident;
}

}  // namespace
}  // namespace o3g

extern "C" int32_t o3g_evaluate_poses(const o3g_grid* g, const float* d_src, int64_t ns, int32_t stride,
                                      int32_t n_poses, const double* poses, double max_corr_dist,
                                      double* out_fitness, double* out_rmse, int64_t* out_inliers, void* stream) {
  const char* fn = "o3g_evaluate_poses";
  if (!g || n_poses < 0 || (n_poses > 0 && (!poses || !out_fitness || !out_rmse)) || !(max_corr_dist >= 0.0) ||
      !std::isfinite(max_corr_dist)) {
    set_error("%s: invalid argument", fn);
    return O3G_ERR_ARG;
  }
  O3G_TRY_STATUS(check_src(fn, d_src, ns, stride));
  for (int64_t k = 0; k < 16 * static_cast<int64_t>(n_poses); ++k)
    if (!std::isfinite(poses[k])) {
      set_error("%s: pose %lld is not finite", fn, static_cast<long long>(k / 16));
      return O3G_ERR_NONFINITE;
    }
  if (n_poses == 0) return O3G_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int ntiles = tiles_of(ns);
  const int64_t items = static_cast<int64_t>(ntiles) * n_poses;
  SortedCloud src(s);
  DevBuf d_poses(s), d_posef(s), part(s), out(s);
  O3G_TRY_STATUS(sort_cloud(d_src, ns, stride, s, &src));
  O3G_TRY(d_poses.alloc(sizeof(double) * 16 * static_cast<size_t>(n_poses)));
  O3G_TRY(d_posef.alloc(sizeof(PoseF) * static_cast<size_t>(n_poses)));
  O3G_TRY(part.alloc(sizeof(double) * 2 * static_cast<size_t>(items)));
  O3G_TRY(out.alloc(sizeof(double) * 3 * static_cast<size_t>(n_poses)));
  O3G_TRY(cudaMemcpyAsync(d_poses.p, poses, sizeof(double) * 16 * static_cast<size_t>(n_poses),
                          cudaMemcpyHostToDevice, s));
  {
    TimedRegion tr(O3G_KERNEL_EVAL, s);
    k_pose_round<<<(n_poses + 127) / 128, 128, 0, s>>>(d_poses.as<double>(), n_poses, d_posef.as<PoseF>());
    const int it = static_cast<int>(std::min<int64_t>(items, 0x7fffffff));
    if (throughput_form(it))
      k_eval_poses<CfgEval><<<grid_for(it, eval_resident<CfgEval>()), kThreads, 0, s>>>(
          g->view(), g->cell, static_cast<float>(max_corr_dist), src.pts, static_cast<int>(ns), ntiles,
          d_posef.as<PoseF>(), n_poses, part.as<double>());
    else
      k_eval_poses<CfgLatency><<<grid_for(it, eval_resident<CfgLatency>()), kThreads, 0, s>>>(
          g->view(), g->cell, static_cast<float>(max_corr_dist), src.pts, static_cast<int>(ns), ntiles,
          d_posef.as<PoseF>(), n_poses, part.as<double>());
    k_eval_sum<<<(n_poses + 3) / 4, 128, 0, s>>>(part.as<double>(), ntiles, n_poses, static_cast<int>(ns),
                                                 out.as<double>());
    count_launch(3);
  }
  O3G_TRY(cudaGetLastError());
  std::vector<double> h(3 * static_cast<size_t>(n_poses));
  int aux[8];
  O3G_TRY(cudaMemcpyAsync(h.data(), out.p, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
  O3G_TRY(cudaMemcpyAsync(aux, src.aux.p, sizeof(aux), cudaMemcpyDeviceToHost, s));
  O3G_TRY(cudaStreamSynchronize(s));
  if (aux[6]) {
    set_error("%s: non-finite source coordinate", fn);
    return O3G_ERR_NONFINITE;
  }
  for (int k = 0; k < n_poses; ++k) {
    out_fitness[k] = h[3 * k];
    out_rmse[k] = h[3 * k + 1];
    if (out_inliers) out_inliers[k] = static_cast<int64_t>(h[3 * k + 2]);
  }
  return O3G_OK;
}

extern "C" int32_t o3g_set_tile_config(int32_t size_class, int32_t cfg) {
  if (size_class < 0 || size_class > 31 || cfg < 0 || cfg > 2) {
    o3g::set_error("o3g_set_tile_config: size class %d or configuration %d out of range", size_class, cfg);
    return O3G_ERR_ARG;
  }
  o3g::g_tile_cfg[size_class].store(cfg, std::memory_order_relaxed);
  return O3G_OK;
}

extern "C" int32_t o3g_get_tile_config(int32_t size_class) {
  if (size_class < 0 || size_class > 31) return O3G_ERR_ARG;
  return o3g::g_tile_cfg[size_class].load(std::memory_order_relaxed);
}

extern "C" int32_t o3g_set_points_per_thread(int32_t size_class, int32_t ppt) {
  if (size_class < 0 || size_class > 31 || !(ppt == 0 || ppt == 1 || ppt == 2 || ppt == 4)) {
    o3g::set_error("o3g_set_points_per_thread: size class %d or points per thread %d out of range", size_class, ppt);
    return O3G_ERR_ARG;
  }
  o3g::g_ppt[size_class].store(ppt, std::memory_order_relaxed);
  return O3G_OK;
}

extern "C" int32_t o3g_get_points_per_thread(int32_t size_class) {
  if (size_class < 0 || size_class > 31) return O3G_ERR_ARG;
  return o3g::g_ppt[size_class].load(std::memory_order_relaxed);
}
