// C ABI of the 3-D SHOITV path: the stand-alone 3-D regulariser gradient and
// APPGA on a volume whose slices share one system matrix (the batched solver
// in volume mode; the 3-D stencil is kernels_vol.cu).
#include <cuda_runtime.h>

#include <cmath>
#include <limits>
#include <string>
#include <vector>

#include "appga.h"
#include "appga_internal.h"
#include "batched_internal.h"
#include "handles.h"

using namespace appga;

namespace {

#define CK(call) APPGA_CK(call)

// Phi of the result volume f (slice-major): the slices' data terms, which the
// solve left in the workspace's host mirror (entries 2z, double-float
// projections), plus the 3-D regulariser of f, summed in FP64 on the host in
// slice order.
appga_status volume_objective(appga_ctx* ctx, appga_matrix* M, int nz, const float* f,
                              const appga_params* p, double* phi) {
  BatchWorkspace& b = *M->bw;
  cudaStream_t s = ctx->stream;
  std::vector<double> data((size_t)nz);
  for (int z = 0; z < nz; ++z) data[(size_t)z] = b.vscal_host[2 * z];
  Vol3Args va{};
  va.n = M->n;
  va.nz = nz;
  va.f[0] = f;
  va.lam1 = (float)p->lambda1;
  va.lam2 = (float)p->lambda2;
  va.eps = (float)p->eps;
  va.want_reg = 1;
  va.pstride = nz;
  va.gR = b.gR;           // scratch: the batched workspace holds d * Kp >= d * nz floats
  va.partial = b.fpartial;
  CK(launch_stencil3d(va, s));
  double* reg = b.vscal + 2 * nz;
  CK(launch_sum_pairs(b.fpartial, stencil3d_grid(M->n, nz), nz, nz, reg, s));
  CK(cudaMemcpyAsync(b.vscal_host + 2 * nz, reg, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double tot = 0.0;
  for (int z = 0; z < nz; ++z) tot += data[(size_t)z];
  *phi = tot + b.vscal_host[2 * nz];
  return APPGA_OK;
}

}  // namespace

extern "C" appga_status appga_shoitv3d_grad(appga_ctx* ctx, int32_t n_side, int32_t nz,
                                            const float* f, double lambda1, double lambda2,
                                            double eps, float* out, double* reg_out,
                                            void* stream) {
  if (!ctx || !f || !out) return fail(APPGA_EINVAL, "null argument");
  if (n_side < 1 || n_side > 46340) return fail(APPGA_EINVAL, "n_side must be in [1, 46340]");
  if (nz < 1 || nz > stencil3d_max_slices())
    return fail(APPGA_EINVAL, "nz must be in [1, " + std::to_string(stencil3d_max_slices()) + "]");
  if (!(lambda1 >= 0.0) || !(lambda2 >= 0.0) || !(eps > 0.0) || !std::isfinite(lambda1) ||
      !std::isfinite(lambda2) || !std::isfinite(eps))
    return fail(APPGA_EINVAL, "lambda1, lambda2 must be finite and >= 0, eps finite and > 0");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const int rows = stencil3d_grid(n_side, nz);
  float2* partial = nullptr;
  if (reg_out) CK(cudaMallocAsync((void**)&partial, (size_t)rows * nz * sizeof(float2), s));
  Vol3Args va{};
  va.n = n_side;
  va.nz = nz;
  va.f[0] = f;
  va.lam1 = (float)lambda1;
  va.lam2 = (float)lambda2;
  va.eps = (float)eps;
  va.want_reg = reg_out ? 1 : 0;
  va.pstride = nz;
  va.gR = out;
  va.partial = partial;
  cudaError_t e = launch_stencil3d(va, s);
  if (e == cudaSuccess && reg_out) e = launch_sum_pairs(partial, rows, nz, nz, reg_out, s);
  if (partial) {
    const cudaError_t e2 = cudaFreeAsync(partial, s);
    if (e == cudaSuccess) e = e2;
  }
  if (e != cudaSuccess) return cuda_fail(e, "appga_shoitv3d_grad");
  return APPGA_OK;
}

extern "C" appga_status appga_reconstruct_volume(appga_ctx* ctx, const appga_matrix* mat,
                                                 int32_t nz, const float* g, const float* gamma,
                                                 const float* f_init, const appga_params* params,
                                                 float* f_out, appga_stats* stats_host,
                                                 void* stream) {
  if (!ctx || !mat || !g || !gamma || !params || !f_out) return fail(APPGA_EINVAL, "null argument");
  if (mat->ctx != ctx) return fail(APPGA_EINVAL, "matrix belongs to another context");
  if (nz < 1 || nz > stencil3d_max_slices())
    return fail(APPGA_EINVAL, "nz must be in [1, " + std::to_string(stencil3d_max_slices()) + "]");
  appga_status rc = appga_params_validate(params);
  if (rc != APPGA_OK) return rc;
  auto* M = const_cast<appga_matrix*>(mat);
  rc = volume_solve(ctx, M, nz, g, gamma, f_init, params, f_out, stream);
  if (rc != APPGA_OK) return rc;
  if (!stats_host) return APPGA_OK;
  const BatchWorkspace& b = *M->bw;
  const SlotState& s0 = b.slots_host[0];
  appga_stats st{};
  st.iters = s0.result_k - s0.k0;
  st.result_k = s0.result_k;
  st.stopped_early = s0.stopped_early;
  st.flags = b.bst_host->flags;
  int64_t hits = 0;
  for (int z = 0; z < nz; ++z) hits += (int64_t)b.slots_host[z].guard_hits;
  st.guard_hits = hits;
  st.phi = std::numeric_limits<double>::quiet_NaN();
  st.phi_prev = std::numeric_limits<double>::quiet_NaN();
  const bool track = params->track_objective != 0 || params->rel_obj_tol > 0.0;
  if (track) {
    st.phi_prev = s0.stopped_early ? b.bst_host->phi_tot_prev : b.bst_host->phi_tot_cur;
    if ((rc = enter_stream(ctx, stream)) != APPGA_OK) return rc;
    double phi = 0.0;
    rc = volume_objective(ctx, M, nz, f_out, params, &phi);
    if (rc != APPGA_OK) return rc;
    st.phi = phi;
    if ((rc = leave_stream(ctx, stream)) != APPGA_OK) return rc;
  }
  *stats_host = st;
  return APPGA_OK;
}
