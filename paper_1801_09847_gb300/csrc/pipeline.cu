// The whole pairwise refinement as one call (Sec. 3.3: estimate_normals on the
// target, then registration_icp with TransformationEstimationPointToPlane()):
// from device buffers (o3g_register_point_to_plane) or from host buffers
// (o3g_register_point_to_plane_host).  The source's spatial sort needs only the
// source, so it runs on a library stream beside the caller's, while the target
// grid is built and its normals are estimated; the iterations wait for both.
#include <cmath>

#include "o3g_internal.cuh"

using namespace o3g;

namespace {

// Owns the events of one fork/join and destroys them on every exit path.
struct Events {
  cudaEvent_t fork = nullptr, ready = nullptr, done = nullptr;
  cudaError_t create() {
    cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
    return e;
  }
  ~Events() {
    if (fork) cudaEventDestroy(fork);
    if (ready) cudaEventDestroy(ready);
    if (done) cudaEventDestroy(done);
  }
};

int32_t register_run(const char* fn, const float* d_src, int64_t ns, int32_t src_stride, const float* d_tgt,
                     int64_t nt, int32_t tgt_stride, const float* d_nrm, int32_t nrm_stride, float normal_radius,
                     int32_t normal_max_nn, const double* init_T, double max_corr_dist, int32_t max_iter, double eps,
                     double* out_T, double* out_fitness, double* out_rmse, int32_t* out_iters, cudaStream_t s) {
  if (ns < 0 || nt < 0 || (ns > 0 && !d_src) || (nt > 0 && !d_tgt) || src_stride < 3 || tgt_stride < 3 ||
      (d_nrm && nrm_stride < 3) || !(max_corr_dist > 0.0) || !std::isfinite(max_corr_dist) ||
      (!d_nrm && (normal_max_nn < 1 || normal_max_nn > O3G_MAX_NN || !(normal_radius >= 0.f)))) {
    set_error("%s: invalid argument", fn);
    return O3G_ERR_ARG;
  }
  if (ns > 0x7fffffffLL - 128) {
    set_error("%s: invalid source cloud (n=%lld)", fn, static_cast<long long>(ns));
    return O3G_ERR_ARG;
  }
  cudaStream_t side = nullptr;
  O3G_TRY(side_stream(&side));
  Events ev;
  O3G_TRY(ev.create());
  // fork: the source sort on the side stream, after everything already on s
  O3G_TRY(cudaEventRecord(ev.fork, s));
  O3G_TRY(cudaStreamWaitEvent(side, ev.fork, 0));
  SortedCloud sc(side);  // its buffers are allocated and freed on the side stream
  const int32_t st_sort = sort_cloud(d_src, ns, src_stride, side, &sc);
  if (st_sort < 0) return st_sort;
  O3G_TRY(cudaEventRecord(ev.ready, side));
  // meanwhile on s: the target grid and its normals
  o3g_grid* g = nullptr;
  int32_t st = o3g_build_grid(d_tgt, nt, tgt_stride, static_cast<float>(max_corr_dist * 1.002), s, &g);
  if (st >= 0) {
    if (d_nrm) st = o3g_grid_set_normals(g, d_nrm, nt, nrm_stride, s);
    else st = estimate_normals_impl(g, normal_radius, normal_max_nn, nullptr, nullptr, 3, s);
  }
  // join: the iterations read the sorted source
  cudaError_t e = cudaStreamWaitEvent(s, ev.ready, 0);
  if (st >= 0 && e != cudaSuccess) st = cuda_fail(e, "join");
  if (st >= 0)
    st = icp_run(g, d_src, ns, src_stride, init_T, max_corr_dist, max_iter, eps, out_T, out_fitness, out_rmse,
                 out_iters, s, O3G_PREC_F32_COMPENSATED, false, &sc);
  // the sorted source is freed on the side stream once s is done with it
  e = cudaEventRecord(ev.done, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ev.done, 0);
  if (e != cudaSuccess) {
    (void)cudaStreamSynchronize(s);
    if (st >= 0) st = cuda_fail(e, "release");
  }
  if (g) o3g_free_grid(g);
  return st;
}

}  // namespace

extern "C" int32_t o3g_register_point_to_plane(const float* d_src, int64_t ns, int32_t src_stride, const float* d_tgt,
                                               int64_t nt, int32_t tgt_stride, const float* d_tgt_nrm,
                                               int32_t nrm_stride, float normal_radius, int32_t normal_max_nn,
                                               const double* init_T, double max_corr_dist, int32_t max_iter,
                                               double eps, double* out_T, double* out_fitness, double* out_rmse,
                                               int32_t* out_iters, void* stream) {
  return register_run("o3g_register_point_to_plane", d_src, ns, src_stride, d_tgt, nt, tgt_stride, d_tgt_nrm,
                      nrm_stride, normal_radius, normal_max_nn, init_T, max_corr_dist, max_iter, eps, out_T,
                      out_fitness, out_rmse, out_iters, static_cast<cudaStream_t>(stream));
}

extern "C" int32_t o3g_register_point_to_plane_host(const float* h_src, int64_t ns, const float* h_tgt, int64_t nt,
                                                    const float* h_tgt_nrm, float normal_radius,
                                                    int32_t normal_max_nn, const double* init_T,
                                                    double max_corr_dist, int32_t max_iter, double eps,
                                                    double* out_T, double* out_fitness, double* out_rmse,
                                                    int32_t* out_iters, void* stream) {
  const char* fn = "o3g_register_point_to_plane_host";
  if (ns < 0 || nt < 0 || (ns > 0 && !h_src) || (nt > 0 && !h_tgt) || !(max_corr_dist > 0.0) ||
      !std::isfinite(max_corr_dist) ||
      (!h_tgt_nrm && (normal_max_nn < 1 || normal_max_nn > O3G_MAX_NN || !(normal_radius >= 0.f)))) {
    set_error("%s: invalid argument", fn);
    return O3G_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DevBuf src(s), tgt(s), nrm(s);
  O3G_TRY(src.alloc(sizeof(float) * 3 * (ns > 0 ? ns : 1)));
  O3G_TRY(tgt.alloc(sizeof(float) * 3 * (nt > 0 ? nt : 1)));
  if (h_tgt_nrm) O3G_TRY(nrm.alloc(sizeof(float) * 3 * (nt > 0 ? nt : 1)));
  if (ns > 0) O3G_TRY(cudaMemcpyAsync(src.p, h_src, sizeof(float) * 3 * ns, cudaMemcpyHostToDevice, s));
  if (nt > 0) O3G_TRY(cudaMemcpyAsync(tgt.p, h_tgt, sizeof(float) * 3 * nt, cudaMemcpyHostToDevice, s));
  if (h_tgt_nrm && nt > 0)
    O3G_TRY(cudaMemcpyAsync(nrm.p, h_tgt_nrm, sizeof(float) * 3 * nt, cudaMemcpyHostToDevice, s));
  return register_run(fn, src.as<float>(), ns, 3, tgt.as<float>(), nt, 3, h_tgt_nrm ? nrm.as<float>() : nullptr, 3,
                      normal_radius, normal_max_nn, init_T, max_corr_dist, max_iter, eps, out_T, out_fitness,
                      out_rmse, out_iters, s);
}
