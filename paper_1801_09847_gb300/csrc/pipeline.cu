// The whole pairwise refinement from host buffers: the call a user with clouds
// in host memory makes (Sec. 3.3: estimate_normals on the target, then
// registration_icp with TransformationEstimationPointToPlane()).
#include <cmath>

#include "o3g_internal.cuh"

using namespace o3g;

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
  if (ns > 0) O3G_TRY(cudaMemcpyAsync(src.p, h_src, sizeof(float) * 3 * ns, cudaMemcpyHostToDevice, s));
  if (nt > 0) O3G_TRY(cudaMemcpyAsync(tgt.p, h_tgt, sizeof(float) * 3 * nt, cudaMemcpyHostToDevice, s));
  o3g_grid* g = nullptr;
  O3G_TRY_STATUS(o3g_build_grid(tgt.as<float>(), nt, 3, static_cast<float>(max_corr_dist * 1.002), stream, &g));
  int32_t st;
  if (h_tgt_nrm) {
    cudaError_t e = nrm.alloc(sizeof(float) * 3 * (nt > 0 ? nt : 1));
    if (e == cudaSuccess && nt > 0)
      e = cudaMemcpyAsync(nrm.p, h_tgt_nrm, sizeof(float) * 3 * nt, cudaMemcpyHostToDevice, s);
    st = e == cudaSuccess ? o3g_grid_set_normals(g, nrm.as<float>(), nt, 3, stream) : cuda_fail(e, "normals upload");
  } else {
    st = estimate_normals_impl(g, normal_radius, normal_max_nn, nullptr, nullptr, 3, s);
  }
  if (st >= 0)
    st = icp_run(g, src.as<float>(), ns, 3, init_T, max_corr_dist, max_iter, eps, out_T, out_fitness, out_rmse,
                 out_iters, s);
  o3g_free_grid(g);
  return st;
}
