// Error reporting and device-memory pool of libo3g.so.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <vector>

#include "o3g_internal.cuh"

namespace o3g {

namespace {
thread_local char g_last_error[512] = "";
std::mutex g_pool_mutex;
constexpr int kMaxDevices = 64;
cudaMemPool_t g_pools[kMaxDevices] = {};
}  // namespace

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
}

int32_t cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
  (void)cudaGetLastError();  // clear a non-sticky error so later calls can proceed
  return e == cudaErrorMemoryAllocation ? O3G_ERR_OOM : O3G_ERR_CUDA;
}

// One private pool per device, created on first use.  Freed blocks stay in the
// pool (release threshold = max) so that repeated calls do not return memory to
// the driver and allocate it again.
static cudaError_t pool_for_current_device(cudaMemPool_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_pool_mutex);
  if (!g_pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool;
    e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t thr = UINT64_MAX;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    if (e != cudaSuccess) return e;
    g_pools[dev] = pool;
  }
  *out = g_pools[dev];
  return cudaSuccess;
}

cudaError_t dmalloc(void** p, size_t bytes, cudaStream_t s) {
  cudaMemPool_t pool;
  cudaError_t e = pool_for_current_device(&pool);
  if (e != cudaSuccess) return e;
  return cudaMallocFromPoolAsync(p, bytes ? bytes : 16, pool, s);
}

void dfree(void* p, cudaStream_t s) {
  if (p) (void)cudaFreeAsync(p, s);
}

// ------------------------------------------------------ instrumentation

namespace {
std::atomic<int64_t> g_launches{0};
std::atomic<int> g_timing{0};
constexpr int kKinds = 7;
struct EventPair {
  cudaEvent_t a, b;
};
std::mutex g_ev_mutex;
std::vector<EventPair> g_events[kKinds];
std::vector<cudaEvent_t> g_free_events;

cudaEvent_t take_event() {
  std::lock_guard<std::mutex> lock(g_ev_mutex);
  if (!g_free_events.empty()) {
    cudaEvent_t e = g_free_events.back();
    g_free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return e;
}
}  // namespace

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

TimedRegion::TimedRegion(int k, cudaStream_t st) : kind(k), s(st) {
  if (!g_timing.load(std::memory_order_relaxed) || k < 0 || k >= kKinds) return;
  cudaEvent_t e = take_event();
  if (e && cudaEventRecord(e, s) == cudaSuccess) ev0 = e;
}

TimedRegion::~TimedRegion() {
  if (!ev0) return;
  cudaEvent_t e1 = take_event();
  if (!e1 || cudaEventRecord(e1, s) != cudaSuccess) return;
  std::lock_guard<std::mutex> lock(g_ev_mutex);
  g_events[kind].push_back({static_cast<cudaEvent_t>(ev0), e1});
}

}  // namespace o3g

extern "C" int64_t o3g_launch_count(void) { return o3g::g_launches.load(); }

extern "C" int32_t o3g_timing_enable(int32_t on) {
  o3g::g_timing.store(on ? 1 : 0);
  return O3G_OK;
}

extern "C" int32_t o3g_timing_read(int32_t kind, double* total_ms, int64_t* launches, int32_t reset) {
  using namespace o3g;
  if (kind < 0 || kind >= kKinds || !total_ms || !launches) {
    set_error("o3g_timing_read: invalid argument");
    return O3G_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_ev_mutex);
  double ms = 0.0;
  for (const EventPair& p : g_events[kind]) {
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(p.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, p.a, p.b);
    if (e != cudaSuccess) return cuda_fail(e, "o3g_timing_read");
    ms += t;
  }
  *total_ms = ms;
  *launches = static_cast<int64_t>(g_events[kind].size());
  if (reset) {
    for (const EventPair& p : g_events[kind]) {
      g_free_events.push_back(p.a);
      g_free_events.push_back(p.b);
    }
    g_events[kind].clear();
  }
  return O3G_OK;
}

extern "C" const char* o3g_last_error(void) { return o3g::g_last_error; }

extern "C" int32_t o3g_abi_version(void) { return 1; }
