// AFPPA solver (appga_afppa_reconstruct): the APPGA forward and pixel phases
// plus the dual-update kernel, captured as a CUDA graph of S steps and
// replayed; every step is (pixel phase, dual update, forward phase).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "afppa_internal.h"
#include "appga.h"
#include "appga_internal.h"
#include "handles.h"

namespace appga {

void free_afppa_workspace(AfppaWorkspace* aw) {
  if (!aw) return;
  for (auto& p : aw->b) cudaFree(p);
  for (auto& p : aw->c) cudaFree(p);
  cudaFree(aw->norms);
  cudaFreeHost(aw->norms_host);
  *aw = AfppaWorkspace();
}

namespace {

#define CK(call) APPGA_CK(call)
constexpr int kAfppaGraphSteps = 16;

appga_status ensure_afppa_workspace(appga_matrix* M) {
  if (M->aw) return APPGA_OK;
  auto* aw = new AfppaWorkspace();
  const size_t d = (size_t)M->d;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = dalloc(&aw->b[i], 2 * d, &M->bytes);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = dalloc(&aw->c[i], 4 * d, &M->bytes);
  if (e == cudaSuccess) e = dalloc(&aw->norms, 2);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&aw->norms_host, 2 * sizeof(double));
  if (e != cudaSuccess) {
    free_afppa_workspace(aw);
    delete aw;
    return cuda_fail(e, "AFPPA workspace");
  }
  M->aw = aw;
  return APPGA_OK;
}

}  // namespace
}  // namespace appga

using namespace appga;

extern "C" appga_status appga_afppa_reconstruct(appga_ctx* ctx, const appga_matrix* mat,
                                                const float* g, const float* gamma,
                                                const float* f_init, const appga_params* p,
                                                float* f_out, float* b_out, float* c_out,
                                                appga_afppa_stats* stats, void* stream) {
  auto* M = const_cast<appga_matrix*>(mat);
  appga_status rc = check_params_and_mat(ctx, M, p);
  if (rc != APPGA_OK) return rc;
  if (!g || !gamma || !f_out) return fail(APPGA_EINVAL, "g, gamma and f_out must be non-NULL");
  if (p->rel_obj_tol != 0.0)
    return fail(APPGA_EINVAL, "AFPPA makes max_iters maps: rel_obj_tol must be 0");
  if ((rc = ensure_workspace(M)) != APPGA_OK) return rc;
  if ((rc = ensure_afppa_workspace(M)) != APPGA_OK) return rc;
  if ((rc = enter_stream(ctx, stream)) != APPGA_OK) return rc;
  cudaStream_t s = ctx->stream;
  Workspace& ws = M->ws;
  AfppaWorkspace& aw = *M->aw;
  if ((rc = validate_inputs(M, g, gamma, f_init, s)) != APPGA_OK) return rc;
  const bool bf16 = bf16_requested(M, p);
  const int d = M->d;
  const size_t fb = (size_t)d * sizeof(float);

  // f^0 = f^1 = f_init (or TMC * 1_disk); zero duals; B^T [b~; c~] = 0
  const int k0 = 1;
  float* cur = ws.f[k0 % 3];
  if (f_init) {
    CK(cudaMemcpyAsync(cur, f_init, fb, cudaMemcpyDeviceToDevice, s));
  } else {
    CK(launch_initial_image(g, gamma, M->m, M->n, M->na, M->npfov, ws.partial_aux, ws.gtick,
                            ws.st_scratch, cur, s));
  }
  CK(cudaMemcpyAsync(ws.f[(k0 + 2) % 3], cur, fb, cudaMemcpyDeviceToDevice, s));
  for (int i = 0; i < 3; ++i) {
    CK(cudaMemsetAsync(aw.b[i], 0, 2 * fb, s));
    CK(cudaMemsetAsync(aw.c[i], 0, 4 * fb, s));
  }
  CK(cudaMemsetAsync(ws.gR, 0, fb, s));

  SolverState h{};
  h.k = k0;
  h.k0 = k0;
  h.k_last = k0 + p->max_iters - 1;
  h.done = p->max_iters == 0 ? 1 : 0;
  h.k_next = k0;
  h.done_next = h.done;
  h.result_k = k0;
  CK(cudaMemcpyAsync(ws.st, &h, sizeof h, cudaMemcpyHostToDevice, s));
  if ((rc = momentum_table(M, ws.st, k0, p, s)) != APPGA_OK) return rc;

  // y^{k0-1} = A f^{k0-1}, then the first forward phase (y^{k0}, w^{k0})
  FwdArgs init{};
  init.A = M->A;
  init.use_bf16 = bf16 ? 1 : 0;
  init.f[0] = ws.f[(k0 + 2) % 3];
  init.y[0] = ws.y[(k0 + 1) & 1];
  init.g = g;
  init.gamma = gamma;
  init.st = ws.st_scratch;
  init.partial = ws.partial_aux;
  init.gtick = ws.gtick;
  init.solver_acc = 1;
  init.n = M->n;
  CK(launch_forward(init, s));
  FwdArgs fa{};
  fa.A = M->A;
  fa.use_bf16 = bf16 ? 1 : 0;
  for (int i = 0; i < 3; ++i) fa.f[i] = ws.f[i];
  fa.y[0] = ws.y[0];
  fa.y[1] = ws.y[1];
  fa.w = ws.w;
  fa.g = g;
  fa.gamma = gamma;
  fa.st = ws.st;
  fa.partial = ws.partial_r;
  fa.gtick = ws.gtick;
  fa.loop = 1;
  fa.no_stencil = 1;
  fa.want_data = 0;
  fa.n = M->n;
  fa.ip = iter_params(p, false);
  fa.theta_tab = ws.theta_tab;
  // the APPGA loop's projection layout (tiled gathers, sliced or folded)
  PixArgs pa{};
  loop_layout(M, &fa, &pa);
  CK(loop_gather_copy(M, ws.f[k0 % 3], s));
  CK(launch_forward(fa, s));

  pa.At = M->At;
  pa.n = M->n;
  for (int i = 0; i < 3; ++i) pa.f[i] = ws.f[i];
  pa.w = ws.w;
  pa.gR = ws.gR;
  pa.inv_lambda = bf16 ? M->inv_lambda_bf16 : M->inv_lambda;
  pa.pfreeze = ws.pfreeze;
  pa.st = ws.st;
  pa.partial = ws.partial_p;
  pa.gtick = ws.gtick;
  pa.ip = iter_params(p, false);
  pa.use_bf16 = bf16 ? 1 : 0;
  pa.want_pmax = 1;
  pa.theta_tab = ws.theta_tab;
  DualArgs da{};
  da.n = M->n;
  da.lambda1 = (float)p->lambda1;
  da.lambda2 = (float)p->lambda2;
  for (int i = 0; i < 3; ++i) {
    da.f[i] = ws.f[i];
    da.b[i] = aw.b[i];
    da.c[i] = aw.c[i];
  }
  da.gR = ws.gR;
  da.st = ws.st;

  if (p->max_iters > 0) {
    const int S = p->graph_iters > 0 ? p->graph_iters : kAfppaGraphSteps;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < S && e == cudaSuccess; ++i) {
      e = launch_pixel(pa, s);
      if (e == cudaSuccess) e = launch_afppa_dual(da, s);
      if (e == cudaSuccess) e = launch_forward(fa, s);
    }
    const cudaError_t e2 = cudaStreamEndCapture(s, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    const int reps = (p->max_iters + S - 1) / S;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = cudaGraphLaunch(exec, s);
    if (exec) cudaGraphExecDestroy(exec);
    if (e != cudaSuccess) return cuda_fail(e, "AFPPA graph");
  }
  CK(cudaMemcpyAsync(ws.st_host, ws.st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const SolverState fin = *ws.st_host;
  const int rk = fin.result_k;
  CK(cudaMemcpyAsync(f_out, ws.f[rk % 3], fb, cudaMemcpyDeviceToDevice, s));
  // the duals of the last map: the dual update of step K wrote b^{K+1}, c^{K+1}
  if (b_out) CK(cudaMemcpyAsync(b_out, aw.b[rk % 3], 2 * fb, cudaMemcpyDeviceToDevice, s));
  if (c_out) CK(cudaMemcpyAsync(c_out, aw.c[rk % 3], 4 * fb, cudaMemcpyDeviceToDevice, s));
  CK(launch_norms2(d, ws.f[rk % 3], ws.f[(rk + 2) % 3], aw.norms, s));
  CK(cudaMemcpyAsync(aw.norms_host, aw.norms, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (stats) {
    std::memset(stats, 0, sizeof *stats);
    stats->iters = rk - k0;
    stats->flags = fin.flags;
    stats->guard_hits = (int64_t)fin.guard_hits;
    stats->re = aw.norms_host[1] > 0.0 ? std::sqrt(aw.norms_host[0] / aw.norms_host[1]) : 0.0;
    stats->rho1 = fin.rho1;
    stats->rho2 = fin.rho2;
  }
  appga_status r3 = leave_stream(ctx, stream);
  if (r3 != APPGA_OK) return r3;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  if (fin.flags & APPGA_FLAG_NONFINITE)
    return fail(APPGA_ENUMERIC, "a non-finite value appeared in the iteration");
  return APPGA_OK;
}
