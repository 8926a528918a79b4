// Batched C ABI: K slices sharing one matrix, iterated together by the
// slot-minor SpMM kernels under captured CUDA graphs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "appga.h"
#include "appga_internal.h"
#include "batched_internal.h"
#include "handles.h"

namespace appga {

void free_batch_workspace(BatchWorkspace* bw) {
  if (!bw) return;
  if (bw->gexec) cudaGraphExecDestroy(bw->gexec);
  for (auto& p : bw->f) cudaFree(p);
  for (auto& p : bw->y) cudaFree(p);
  cudaFree(bw->w);
  cudaFree(bw->gR);
  cudaFree(bw->pfreeze);
  cudaFree(bw->g);
  cudaFree(bw->gamma);
  cudaFree(bw->slots);
  cudaFree(bw->bst);
  cudaFree(bw->partial);
  cudaFree(bw->fpartial);
  cudaFree(bw->gtick);
  cudaFree(bw->flag);
  for (auto& p : bw->fsm) cudaFree(p);
  cudaFree(bw->gsm);
  cudaFree(bw->vscal);
  cudaFreeHost(bw->vscal_host);
  cudaFreeHost(bw->slots_host);
  cudaFreeHost(bw->bst_host);
  cudaFreeHost(bw->flag_host);
  if (bw->side) cudaStreamDestroy(bw->side);
  if (bw->ev_fork) cudaEventDestroy(bw->ev_fork);
  if (bw->ev_join) cudaEventDestroy(bw->ev_join);
  *bw = BatchWorkspace();
}

int64_t batch_workspace_bytes(int m, int d, int Kp) {
  const int64_t ngroups = batch_max_blocks() / 64 + 2;
  int64_t b = 0;
  b += (int64_t)5 * d * Kp * sizeof(float);  // f ring, gR, pfreeze
  b += (int64_t)5 * m * Kp * sizeof(float);  // y ring, w, g, gamma
  b += (int64_t)Kp * sizeof(SlotState) + sizeof(BatchState);
  b += (2 * batch_max_blocks() + ngroups + 2) * Kp * (int64_t)sizeof(float2);
  b += ngroups * (int64_t)sizeof(unsigned int) + (int64_t)sizeof(int);
  b += (int64_t)(Kp + 2) * sizeof(double);
  return b;
}

cudaError_t alloc_batch_workspace(BatchWorkspace& b, int m, int d, int Kp) {
  b = BatchWorkspace();
  const size_t dd = (size_t)d * Kp, mm = (size_t)m * Kp;
  const int maxb = batch_max_blocks();
  const int ngroups = maxb / 64 + 2;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = dalloc(&b.f[i], dd);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = dalloc(&b.y[i], mm);
  if (e == cudaSuccess) e = dalloc(&b.w, mm);
  if (e == cudaSuccess) e = dalloc(&b.gR, dd);
  if (e == cudaSuccess) e = dalloc(&b.pfreeze, dd);
  if (e == cudaSuccess) e = dalloc(&b.g, mm);
  if (e == cudaSuccess) e = dalloc(&b.gamma, mm);
  if (e == cudaSuccess) e = dalloc(&b.slots, (size_t)Kp);
  if (e == cudaSuccess) e = dalloc(&b.bst, 1);
  if (e == cudaSuccess) e = dalloc(&b.partial, (size_t)(maxb + ngroups + 2) * Kp);
  if (e == cudaSuccess) e = dalloc(&b.fpartial, (size_t)maxb * Kp);
  if (e == cudaSuccess) e = dalloc(&b.gtick, (size_t)ngroups);
  if (e == cudaSuccess) e = dalloc(&b.flag, 1);
  if (e == cudaSuccess) e = dalloc(&b.vscal, (size_t)2 * Kp + 2);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b.vscal_host, (2 * Kp + 2) * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(b.gtick, 0, (size_t)ngroups * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(b.bst, 0, sizeof(BatchState));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b.slots_host, Kp * sizeof(SlotState));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b.bst_host, sizeof(BatchState));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b.flag_host, sizeof(int));
  if (e != cudaSuccess) {
    free_batch_workspace(&b);
    return e;
  }
  b.Kp = Kp;
  b.m = m;
  b.d = d;
  return cudaSuccess;
}

BatchSchedule tuned_schedule(const appga_matrix* M, int Kp, bool bf16) {
  auto it = M->tuned.find(Kp * 2 + (bf16 ? 1 : 0));
  return it == M->tuned.end() ? BatchSchedule() : it->second;
}

void make_batch_args(const DevCSR& A, const DevCSR& At, const float* inv_lambda, int n,
                     BatchWorkspace& b, bool bf16, bool track, const BatchSchedule& sch,
                     BFwdArgs* fa, BPixArgs* pa) {
  *fa = BFwdArgs{};
  fa->spmv_per_sm = sch.spmv_per_sm;
  fa->stencil_per_sm = sch.stencil_per_sm;
  fa->gather_rows = sch.gather_rows_fw;
  fa->A = A;
  fa->n = n;
  fa->Kp = b.Kp;
  fa->track = track ? 1 : 0;
  fa->use_bf16 = bf16 ? 1 : 0;
  for (int i = 0; i < 3; ++i) fa->f[i] = b.f[i];
  fa->y[0] = b.y[0];
  fa->y[1] = b.y[1];
  fa->w = b.w;
  fa->g = b.g;
  fa->gamma = b.gamma;
  fa->gR = b.gR;
  fa->slots = b.slots;
  fa->bst = b.bst;
  fa->fpartial = b.fpartial;
  *pa = BPixArgs{};
  pa->blocks_per_sm = sch.pixel_per_sm;
  pa->gather_rows = sch.gather_rows_px;
  pa->At = At;
  pa->n = n;
  pa->Kp = b.Kp;
  pa->use_bf16 = bf16 ? 1 : 0;
  for (int i = 0; i < 3; ++i) pa->f[i] = b.f[i];
  pa->w = b.w;
  pa->gR = b.gR;
  pa->inv_lambda = inv_lambda;
  pa->pfreeze = b.pfreeze;
  pa->slots = b.slots;
  pa->bst = b.bst;
  pa->partial = b.partial;
  pa->gtick = b.gtick;
  pa->fpartial = b.fpartial;
  pa->n_fpartial = bforward_grid(*fa);
  pa->track = track ? 1 : 0;
}

cudaError_t capture_batch_graph(const BFwdArgs& fa, const BPixArgs& pa, int S, cudaStream_t s,
                                cudaGraphExec_t* out, const VolumeSteps* vb) {
  *out = nullptr;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < S && e == cudaSuccess; ++i) {
    e = launch_bpixel(pa, s);
    if (e == cudaSuccess && vb)
      e = launch_slots_to_slices(vb->slot_ring, vb->slice_ring, vb->d, vb->Kp, vb->nz,
                                 vb->va.bst, 0, s);
    if (vb) {
      // the 3-D stencil needs only the iterate: its branch runs beside the
      // forward phase (which reads the same iterate and writes w, y and the
      // objective rows before the stencil's) and joins before the update
      if (e == cudaSuccess) e = cudaEventRecord(vb->ev_fork, s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(vb->side, vb->ev_fork, 0);
      if (e == cudaSuccess) e = launch_stencil3d(vb->va, vb->side);
      if (e == cudaSuccess)
        e = launch_slices_to_slots(vb->va.gR, fa.gR, vb->d, vb->Kp, vb->nz, vb->va.bst,
                                   vb->side);
      if (e == cudaSuccess) e = cudaEventRecord(vb->ev_join, vb->side);
    }
    if (e == cudaSuccess) e = launch_bforward(fa, s);
    if (e == cudaSuccess && vb) e = cudaStreamWaitEvent(s, vb->ev_join, 0);
  }
  const cudaError_t e2 = cudaStreamEndCapture(s, &graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  return e;
}

SlotState slot_from_params(const appga_params* p, int k0, bool active) {
  SlotState s{};
  s.active = active ? 1 : 0;
  s.k = k0;
  s.k0 = k0;
  s.k_last = k0 + p->max_iters - 1;
  s.done = (active && p->max_iters > 0) ? 0 : 1;
  s.result_k = k0;
  s.freeze_iter = p->precond_freeze_iter;
  s.momentum = p->momentum;
  s.lambda1 = (float)p->lambda1;
  s.lambda2 = (float)p->lambda2;
  s.eps = (float)p->eps;
  s.beta = (float)p->beta;
  s.omega = p->omega;
  s.a = p->a;
  s.b = p->b;
  s.rel_tol = p->rel_obj_tol;
  s.phi_cur = std::numeric_limits<double>::quiet_NaN();
  s.phi_prev = s.phi_cur;
  s.phi_k = -1;
  return s;
}

namespace {

constexpr int kBatchGraphIters = 8;
// forward-phase blocks per SM in volume mode: 5 (one resident wave at 48
// registers per thread) measured fastest with the 3-D stencil's branch
// beside it (680.6 us per 64 x 256^2 volume iteration; 4: 725.9, 3: 842.7,
// the batched default of 8: 727.3); 0 keeps the batched default
#ifndef APPGA_VOL_SPMV_PER_SM
#define APPGA_VOL_SPMV_PER_SM 5
#endif
// pixel-phase blocks per SM in volume mode (0: the batched default): 5, the
// 2-D autotuner's choice for 64 slices of 256^2, measured fastest here too
// (650.7 us per 64 x 256^2 volume iteration; 4: 682.6, 6: 736.4, default:
// 679.3)
#ifndef APPGA_VOL_PIXEL_PER_SM
#define APPGA_VOL_PIXEL_PER_SM 5
#endif

int padded_width(int K) { return K <= 32 ? 32 : (K <= 64 ? 64 : 128); }

appga_status ensure_batch_workspace(appga_matrix* M, int Kp) {
  if (M->bw && M->bw->Kp == Kp) return APPGA_OK;
  if (M->bw) {
    free_batch_workspace(M->bw);
  } else {
    M->bw = new BatchWorkspace();
  }
  const cudaError_t e = alloc_batch_workspace(*M->bw, M->m, M->d, Kp);
  if (e != cudaSuccess) {
    delete M->bw;
    M->bw = nullptr;
    return cuda_fail(e, "batched workspace allocation");
  }
  return APPGA_OK;
}

#define CK(call) APPGA_CK(call)

}  // namespace
}  // namespace appga

using namespace appga;

namespace appga {
namespace {

// One batched run of K <= 128 slices with launch schedule `sch` (its chunk
// field is ignored here) in a workspace at least min_width slots wide.
// Inputs are validated by the caller.
appga_status batched_solve(appga_ctx* ctx, appga_matrix* M, int32_t K, const float* g,
                           const float* gamma, const float* f_init, const appga_params* params,
                           float* f_out, appga_stats* stats_host, const BatchSchedule& sch,
                           void* stream, int min_width = 0, bool volume = false) {
  appga_status rc = APPGA_OK;
  const int Kp = std::max(padded_width(K), min_width);
  if ((rc = ensure_batch_workspace(M, Kp)) != APPGA_OK) return rc;
  if ((rc = enter_stream(ctx, stream)) != APPGA_OK) return rc;
  BatchWorkspace& b = *M->bw;
  cudaStream_t s = ctx->stream;
  const int m = M->m, d = M->d, n = M->n;
  const bool track = params->track_objective != 0 || params->rel_obj_tol > 0.0;
  const bool bf16 = params->a_precision == APPGA_PREC_BF16 && M->has_bf16;

  // input checks (g >= 0, gamma > 0, f_init >= 0, all finite) over every slice
  CK(cudaMemsetAsync(b.flag, 0, sizeof(int), s));
  CK(launch_validate_inputs(g, gamma, K * m, f_init, K * d, b.flag, s));
  CK(cudaMemcpyAsync(b.flag_host, b.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (*b.flag_host)
    return fail(APPGA_EDOMAIN,
                "inputs must satisfy: g finite and >= 0, gamma finite and > 0, f finite and >= 0");

  // slot-minor copies of the sinograms; padding slots hold harmless data
  CK(launch_to_slot_minor(g, K, m, b.g, Kp, 0, nullptr, s));
  CK(launch_to_slot_minor(gamma, K, m, b.gamma, Kp, 0, nullptr, s));
  CK(launch_fill_slots(b.g, m, Kp, K, Kp, 0.f, s));
  CK(launch_fill_slots(b.gamma, m, Kp, K, Kp, 1.f, s));

  // f^0 = f^1 = f_init (or the per-slice initial image) in the ring slots of step G0
  const int G0 = 1;
  float* cur = b.f[G0 % 3];
  if (f_init) {
    CK(launch_to_slot_minor(f_init, K, d, cur, Kp, 0, nullptr, s));
  } else {
    CK(launch_binit_image(g, gamma, m, n, M->na, M->npfov, K, Kp, 0, nullptr, cur, s));
  }
  CK(launch_fill_slots(cur, d, Kp, K, Kp, 0.f, s));
  CK(cudaMemcpyAsync(b.f[(G0 + 2) % 3], cur, (size_t)d * Kp * sizeof(float),
                     cudaMemcpyDeviceToDevice, s));

  for (int i = 0; i < Kp; ++i) b.slots_host[i] = slot_from_params(params, 1, i < K);
  CK(cudaMemcpyAsync(b.slots, b.slots_host, Kp * sizeof(SlotState), cudaMemcpyHostToDevice, s));
  CK(launch_binit_momentum(b.slots, Kp, false, s));
  BatchState hb{};
  hb.gstep = G0;
  hb.remaining = params->max_iters > 0 ? K : 0;
  hb.phi_tot_k = -1;
  *b.bst_host = hb;
  CK(cudaMemcpyAsync(b.bst, b.bst_host, sizeof(BatchState), cudaMemcpyHostToDevice, s));

  BFwdArgs fa;
  BPixArgs pa;
  make_batch_args(M->A, M->At, bf16 ? M->inv_lambda_bf16 : M->inv_lambda, n, b, bf16, track, sch,
                  &fa, &pa);
  // volume: the K slots are the slices of one volume.  The 3-D stencil runs
  // on slice-major copies of the iterates after the forward phase, leaves
  // its per-slice regulariser sums after the forward phase's rows, and its
  // gradient is moved back to the slot-minor gR; one stopping test
  VolumeSteps vb{};
  if (volume) {
    for (int i = 0; i < 3; ++i)
      if (!b.fsm[i]) CK(cudaMalloc((void**)&b.fsm[i], (size_t)d * Kp * sizeof(float)));
    if (!b.gsm) CK(cudaMalloc((void**)&b.gsm, (size_t)d * Kp * sizeof(float)));
    if (!b.side) CK(cudaStreamCreateWithFlags(&b.side, cudaStreamNonBlocking));
    if (!b.ev_fork) CK(cudaEventCreateWithFlags(&b.ev_fork, cudaEventDisableTiming));
    if (!b.ev_join) CK(cudaEventCreateWithFlags(&b.ev_join, cudaEventDisableTiming));
    vb.side = b.side;
    vb.ev_fork = b.ev_fork;
    vb.ev_join = b.ev_join;
    fa.no_stencil = 1;
    // leave room on each SM for a stencil block beside the forward phase's
    if (sch.spmv_per_sm == 0) fa.spmv_per_sm = APPGA_VOL_SPMV_PER_SM;
    if (sch.pixel_per_sm == 0 && APPGA_VOL_PIXEL_PER_SM > 0) pa.blocks_per_sm = APPGA_VOL_PIXEL_PER_SM;
    pa.joint = 1;
    const int nfw = bforward_grid(fa);
    Vol3Args& va = vb.va;
    va.n = n;
    va.nz = K;
    for (int i = 0; i < 3; ++i) {
      va.f[i] = b.fsm[i];
      vb.slot_ring[i] = b.f[i];
      vb.slice_ring[i] = b.fsm[i];
    }
    va.slots = b.slots;
    va.bst = b.bst;
    va.want_reg = track ? 1 : 0;
    va.pstride = Kp;
    va.gR = b.gsm;
    va.partial = b.fpartial + (size_t)nfw * Kp;
    vb.d = d;
    vb.Kp = Kp;
    vb.nz = K;
    pa.n_fpartial = nfw + (track ? stencil3d_grid(n, K) : 0);
  }

  // y^{k0-1}, then the first forward phase (w, y, stencil, Phi of f^{k0})
  BFwdArgs init = fa;
  init.mode = 1;
  CK(launch_bforward(init, s));
  CK(launch_bforward(fa, s));
  if (volume) {
    CK(launch_slots_to_slices(vb.slot_ring, vb.slice_ring, d, Kp, K, b.bst, 1, s));
    CK(launch_stencil3d(vb.va, s));
    CK(launch_slices_to_slots(vb.va.gR, b.gR, d, Kp, K, b.bst, s));
  }

  if (params->max_iters > 0) {
    const int S = params->graph_iters > 0 ? params->graph_iters : kBatchGraphIters;
    char key[256];
    // the graph's kernels see only the workspace, never K or the caller's buffers
    std::snprintf(key, sizeof key, "%d|%d|%d|%d|%d|%d|%d|%d|%d", Kp, (int)track, (int)bf16, S,
                  sch.spmv_per_sm, sch.stencil_per_sm, sch.pixel_per_sm, (int)volume,
                  volume ? K : 0);
    if (b.gexec == nullptr || b.gkey != key) {
      if (b.gexec) {
        cudaGraphExecDestroy(b.gexec);
        b.gexec = nullptr;
      }
      const cudaError_t e = capture_batch_graph(fa, pa, S, s, &b.gexec, volume ? &vb : nullptr);
      if (e != cudaSuccess) return cuda_fail(e, "batched graph capture");
      b.gkey = key;
    }
    const int reps = (params->max_iters + S - 1) / S;
    if (params->rel_obj_tol > 0.0) {
      cudaEvent_t ev[2];
      CK(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
      appga_status prc = APPGA_OK;
      for (int r = 0; r < reps; ++r) {
        cudaError_t e = cudaGraphLaunch(b.gexec, s);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(&b.bst_host->remaining, &b.bst->remaining, sizeof(int),
                              cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaEventRecord(ev[r & 1], s);
        if (e != cudaSuccess) {
          prc = cuda_fail(e, "batched graph replay");
          break;
        }
        if (r >= 1) {
          e = cudaEventSynchronize(ev[(r - 1) & 1]);
          if (e != cudaSuccess) {
            prc = cuda_fail(e, "cudaEventSynchronize");
            break;
          }
          if (b.bst_host->remaining == 0) break;
        }
      }
      cudaEventDestroy(ev[0]);
      cudaEventDestroy(ev[1]);
      if (prc != APPGA_OK) return prc;
    } else {
      for (int r = 0; r < reps; ++r) CK(cudaGraphLaunch(b.gexec, s));
    }
  }
  // a slot stopped by the test in the last pixel phase has its result one
  // ring entry back: move it into the current entry first
  CK(launch_resolve_rollback(fa, s));
  CK(cudaMemcpyAsync(b.bst_host, b.bst, sizeof(BatchState), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(b.slots_host, b.slots, Kp * sizeof(SlotState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const int Gf = b.bst_host->gstep;
  CK(launch_from_slot_minor(b.f[Gf % 3], K, d, Kp, 0, nullptr, f_out, s));
  if (track) {
    // the objective terms of every result image, in the arithmetic of
    // appga_objective, with one host round trip for all of them (2-D: data
    // term and regulariser per slice; volume: the data terms, the 3-D
    // regulariser follows with the statistics)
    if ((rc = objective_terms(M, K, f_out, g, gamma, params, !volume, b.vscal, s)) != APPGA_OK)
      return rc;
    CK(cudaMemcpyAsync(b.vscal_host, b.vscal, (size_t)2 * K * sizeof(double),
                       cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  rc = APPGA_OK;
  if (b.bst_host->flags & APPGA_FLAG_NONFINITE) rc = fail(APPGA_ENUMERIC, "a non-finite value appeared");
  if (stats_host) {
    for (int i = 0; i < K; ++i) {
      const SlotState& sl = b.slots_host[i];
      appga_stats& st = stats_host[i];
      st.iters = sl.result_k - sl.k0;
      st.result_k = sl.result_k;
      st.stopped_early = sl.stopped_early;
      st.flags = b.bst_host->flags;
      st.guard_hits = (int64_t)sl.guard_hits;
      st.phi = std::numeric_limits<double>::quiet_NaN();
      st.phi_prev = std::numeric_limits<double>::quiet_NaN();
      if (track) st.phi_prev = sl.stopped_early ? sl.phi_prev : sl.phi_cur;
    }
    if (track && !volume)
      for (int i = 0; i < K; ++i) stats_host[i].phi = b.vscal_host[2 * i] + b.vscal_host[2 * i + 1];
  }
  appga_status r3 = leave_stream(ctx, stream);
  if (r3 != APPGA_OK) return r3;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return rc;
}

appga_status check_batched_args(appga_ctx* ctx, const appga_matrix* mat, int32_t K,
                                const float* g, const float* gamma, const appga_params* params) {
  if (!ctx || !mat || !g || !gamma || !params) return fail(APPGA_EINVAL, "null argument");
  if (mat->ctx != ctx) return fail(APPGA_EINVAL, "matrix belongs to another context");
  if (K < 1 || K > 128) return fail(APPGA_EINVAL, "K must be in [1, 128]");
  appga_status rc = check_slot_width(mat, padded_width(K));
  if (rc != APPGA_OK) return rc;
  return appga_params_validate(params);
}

// K slices with schedule `sch`: as one batch, or as sub-batches of sch.chunk
// slices run one after another (each with the schedule tuned for its width).
appga_status batched_run(appga_ctx* ctx, appga_matrix* M, int32_t K, const float* g,
                         const float* gamma, const float* f_init, const appga_params* params,
                         float* f_out, appga_stats* stats_host, const BatchSchedule& sch,
                         void* stream) {
  if (sch.chunk <= 0 || sch.chunk >= K)
    return batched_solve(ctx, M, K, g, gamma, f_init, params, f_out, stats_host, sch, stream);
  // every sub-batch (the last one too) runs at the chunk's width, so the
  // workspace and its captured graph are reused
  for (int c0 = 0; c0 < K; c0 += sch.chunk) {
    const int kc = std::min(sch.chunk, K - c0);
    appga_status rc = batched_solve(
        ctx, M, kc, g + (size_t)c0 * M->m, gamma + (size_t)c0 * M->m,
        f_init ? f_init + (size_t)c0 * M->d : nullptr, params, f_out + (size_t)c0 * M->d,
        stats_host ? stats_host + c0 : nullptr, sch, stream, sch.chunk);
    if (rc != APPGA_OK) return rc;
  }
  return APPGA_OK;
}

}  // namespace

appga_status check_slot_width(const appga_matrix* M, int Kp) {
  if ((int64_t)std::max(M->m, M->d) * Kp > (int64_t)INT32_MAX)
    return fail(APPGA_EINVAL, "matrix too large for this batch width: max(m, d) * " +
                                  std::to_string(Kp) + " must stay below 2^31");
  return APPGA_OK;
}

appga_status volume_solve(appga_ctx* ctx, appga_matrix* M, int32_t K, const float* g,
                          const float* gamma, const float* f_init, const appga_params* params,
                          float* f_out, void* stream) {
  const bool bf16 = params->a_precision == APPGA_PREC_BF16 && M->has_bf16;
  const int Kp = padded_width(K);
  const appga_status rc = check_slot_width(M, Kp);
  if (rc != APPGA_OK) return rc;
  return batched_solve(ctx, M, K, g, gamma, f_init, params, f_out, nullptr,
                       tuned_schedule(M, Kp, bf16), stream, 0, true);
}

}  // namespace appga

extern "C" appga_status appga_reconstruct_batched(appga_ctx* ctx, const appga_matrix* mat,
                                                  int32_t K, const float* g, const float* gamma,
                                                  const float* f_init, const appga_params* params,
                                                  float* f_out, appga_stats* stats_host,
                                                  void* stream) {
  if (!f_out) return fail(APPGA_EINVAL, "null argument");
  appga_status rc = check_batched_args(ctx, mat, K, g, gamma, params);
  if (rc != APPGA_OK) return rc;
  auto* M = const_cast<appga_matrix*>(mat);
  const bool bf16 = params->a_precision == APPGA_PREC_BF16 && M->has_bf16;
  return batched_run(ctx, M, K, g, gamma, f_init, params, f_out, stats_host,
                     tuned_schedule(M, padded_width(K), bf16), stream);
}

namespace appga {
namespace {
// best gathered GB/s over launch shapes for the column stream `col` (nnz
// entries) into the slot-minor block x of `width` floats per row
appga_status probe_best(const DevCSR& M, bool forward, const float* x, int width, float* sink,
                        int launches, cudaStream_t s, double* best) {
  const long long nnz = M.nnz_padded;
  *best = 0.0;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  CK(cudaEventCreate(&ev[0]));
  cudaError_t e = cudaEventCreate(&ev[1]);
  for (const int per_sm : {3, 4, 5, 6, 8}) {
    for (int i = 0; i < 2 && e == cudaSuccess; ++i)
      e = launch_gather_probe(M, forward, x, width, sink, per_sm, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
    for (int i = 0; i < launches && e == cudaSuccess; ++i)
      e = launch_gather_probe(M, forward, x, width, sink, per_sm, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    if (e != cudaSuccess) break;
    const double gbs = (double)launches * (double)nnz * width * sizeof(float) / (ms * 1e-3) / 1e9;
    if (gbs > *best) *best = gbs;
  }
  cudaEventDestroy(ev[0]);
  if (ev[1]) cudaEventDestroy(ev[1]);
  if (e != cudaSuccess) return cuda_fail(e, "appga_gather_probe");
  return APPGA_OK;
}
}  // namespace
}  // namespace appga

extern "C" appga_status appga_gather_probe(appga_ctx* ctx, const appga_matrix* mat,
                                           int32_t width, int32_t launches, double* gbs_fwd,
                                           double* gbs_bwd) {
  if (!ctx || !mat || !gbs_fwd || !gbs_bwd) return fail(APPGA_EINVAL, "null argument");
  if (mat->ctx != ctx) return fail(APPGA_EINVAL, "matrix belongs to another context");
  if (width != 32 && width != 64 && width != 128)
    return fail(APPGA_EINVAL, "width must be 32, 64 or 128");
  if (launches < 1) return fail(APPGA_EINVAL, "launches must be >= 1");
  appga_status rc = check_slot_width(mat, width);
  if (rc != APPGA_OK) return rc;
  auto* M = const_cast<appga_matrix*>(mat);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(APPGA_ENODEV, "cudaSetDevice failed");
  rc = ensure_batch_workspace(M, width);
  if (rc != APPGA_OK) return rc;
  BatchWorkspace& b = *M->bw;
  cudaStream_t s = ctx->stream;
  float* sink = reinterpret_cast<float*>(b.partial);
  // forward projection: A's columns into the image block [d][width];
  // back-projection: A^T's columns into the weight block [m][width]
  CK(cudaMemsetAsync(b.f[0], 0, (size_t)M->d * width * sizeof(float), s));
  CK(cudaMemsetAsync(b.w, 0, (size_t)M->m * width * sizeof(float), s));
  rc = probe_best(M->A, true, b.f[0], width, sink, launches, s, gbs_fwd);
  if (rc == APPGA_OK) rc = probe_best(M->At, false, b.w, width, sink, launches, s, gbs_bwd);
  return rc;
}

extern "C" appga_status appga_autotune_batched(appga_ctx* ctx, const appga_matrix* mat,
                                               int32_t K, const float* g, const float* gamma,
                                               const appga_params* params,
                                               appga_batch_tuning* out_host) {
  float* f_scratch = nullptr;
  appga_status rc = check_batched_args(ctx, mat, K, g, gamma, params);
  if (rc != APPGA_OK) return rc;
  auto* M = const_cast<appga_matrix*>(mat);
  const bool bf16 = params->a_precision == APPGA_PREC_BF16 && M->has_bf16;
  const int Kp = padded_width(K);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(APPGA_ENODEV, "cudaSetDevice failed");
  CK(cudaMalloc((void**)&f_scratch, (size_t)K * M->d * sizeof(float)));
  cudaEvent_t ev[3];
  for (auto& e : ev) e = nullptr;
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaFree(f_scratch);
      return fail(APPGA_ECUDA, "cudaEventCreate failed");
    }
  cudaStream_t s = ctx->stream;
  // Trials run the solver itself on the caller's slices: kWarm maps (graph
  // capture, caches), then kWarm and kWarm + kTimed maps timed with events;
  // the difference is the cost of kTimed maps.
  constexpr int kWarm = 4, kTimed = 16;
  appga_params p = *params;
  p.rel_obj_tol = 0.0;
  auto trial = [&](const BatchSchedule& sch, double* us) -> appga_status {
    float ms[2] = {0.f, 0.f};
    for (int r = 0; r < 3; ++r) {
      p.max_iters = r == 2 ? kWarm + kTimed : kWarm;
      if (r > 0 && cudaEventRecord(ev[0], s) != cudaSuccess) return fail(APPGA_ECUDA, "event");
      appga_status st = batched_run(ctx, M, K, g, gamma, nullptr, &p, f_scratch, nullptr, sch, s);
      if (st != APPGA_OK) return st;
      if (r > 0) {
        if (cudaEventRecord(ev[1], s) != cudaSuccess || cudaEventSynchronize(ev[1]) != cudaSuccess)
          return fail(APPGA_ECUDA, "event");
        cudaEventElapsedTime(&ms[r - 1], ev[0], ev[1]);
      }
    }
    *us = 1e3 * (double)(ms[1] - ms[0]) / ((double)kTimed * K);
    return APPGA_OK;
  };
  BatchSchedule best;  // kernel defaults, whole batch
  double best_us = 0.0, default_us = 0.0;
  rc = trial(best, &best_us);
  default_us = best_us;
  // coordinate descent: sub-batch width, then SpMV, back-projection and stencil grids
  auto consider = [&](BatchSchedule cand) -> appga_status {
    if (cand == best) return APPGA_OK;
    double us = 0.0;
    appga_status st = trial(cand, &us);
    if (st != APPGA_OK) return st;
    if (us < best_us) {
      best = cand;
      best_us = us;
    }
    return APPGA_OK;
  };
  for (int c : {32, 64}) {
    if (rc != APPGA_OK || c >= Kp) break;
    BatchSchedule cand = best;
    cand.chunk = c;
    rc = consider(cand);
  }
  for (int v : {1, 2, 3, 4, 5, 6, 8, 12}) {
    if (rc != APPGA_OK) break;
    BatchSchedule cand = best;
    cand.spmv_per_sm = v;
    rc = consider(cand);
  }
  for (int v : {2, 3, 4, 5, 6, 8, 12}) {
    if (rc != APPGA_OK) break;
    BatchSchedule cand = best;
    cand.pixel_per_sm = v;
    rc = consider(cand);
  }
  for (int v : {1, 2, 3, 4, 8}) {
    if (rc != APPGA_OK) break;
    BatchSchedule cand = best;
    cand.stencil_per_sm = v;
    rc = consider(cand);
  }
  // rows gathered per step by each projection (kernel instances)
  if (rc == APPGA_OK) {
    BatchSchedule cand = best;
    cand.gather_rows_fw = 4;
    rc = consider(cand);
  }
  if (rc == APPGA_OK) {
    BatchSchedule cand = best;
    cand.gather_rows_px = 4;
    rc = consider(cand);
  }
  for (auto& e : ev) cudaEventDestroy(e);
  cudaFree(f_scratch);
  if (rc != APPGA_OK) return rc;
  M->tuned[Kp * 2 + (bf16 ? 1 : 0)] = best;
  if (out_host) {
    std::memset(out_host, 0, sizeof *out_host);
    out_host->K = K;
    out_host->a_precision = bf16 ? APPGA_PREC_BF16 : APPGA_PREC_FP32;
    out_host->spmv_per_sm = best.spmv_per_sm;
    out_host->stencil_per_sm = best.stencil_per_sm;
    out_host->pixel_per_sm = best.pixel_per_sm;
    out_host->chunk = best.chunk;
    out_host->gather_rows_fw = best.gather_rows_fw == 0 ? 8 : best.gather_rows_fw;
    out_host->gather_rows_px = best.gather_rows_px == 0 ? 8 : best.gather_rows_px;
    out_host->us_per_slice_iter = best_us;
    out_host->us_per_slice_iter_default = default_us;
  }
  return APPGA_OK;
}

extern "C" appga_status appga_batch_schedule_get(const appga_matrix* mat,
                                                 appga_batch_tuning* t) {
  if (!mat || !t) return fail(APPGA_EINVAL, "null argument");
  if (t->K < 1 || t->K > 128) return fail(APPGA_EINVAL, "K must be in [1, 128]");
  const BatchSchedule sch =
      tuned_schedule(mat, padded_width(t->K), t->a_precision == APPGA_PREC_BF16);
  t->spmv_per_sm = sch.spmv_per_sm;
  t->stencil_per_sm = sch.stencil_per_sm;
  t->pixel_per_sm = sch.pixel_per_sm;
  t->chunk = sch.chunk;
  t->gather_rows_fw = sch.gather_rows_fw;
  t->gather_rows_px = sch.gather_rows_px;
  return APPGA_OK;
}

extern "C" appga_status appga_batch_schedule_set(appga_matrix* mat, const appga_batch_tuning* t) {
  if (!mat || !t) return fail(APPGA_EINVAL, "null argument");
  if (t->K < 1 || t->K > 128) return fail(APPGA_EINVAL, "K must be in [1, 128]");
  if (t->a_precision != APPGA_PREC_FP32 && t->a_precision != APPGA_PREC_BF16)
    return fail(APPGA_EINVAL, "a_precision must be APPGA_PREC_FP32 or APPGA_PREC_BF16");
  for (int v : {t->spmv_per_sm, t->stencil_per_sm, t->pixel_per_sm})
    if (v < 0 || v > 16) return fail(APPGA_EINVAL, "blocks per SM must be in [0, 16]");
  if (t->chunk != 0 && t->chunk != 32 && t->chunk != 64)
    return fail(APPGA_EINVAL, "chunk must be 0, 32 or 64");
  for (int v : {t->gather_rows_fw, t->gather_rows_px})
    if (v != 0 && v != 4 && v != 8) return fail(APPGA_EINVAL, "gather rows must be 0, 4 or 8");
  BatchSchedule sch;
  sch.spmv_per_sm = t->spmv_per_sm;
  sch.stencil_per_sm = t->stencil_per_sm;
  sch.pixel_per_sm = t->pixel_per_sm;
  sch.chunk = t->chunk;
  sch.gather_rows_fw = t->gather_rows_fw == 8 ? 0 : t->gather_rows_fw;
  sch.gather_rows_px = t->gather_rows_px == 8 ? 0 : t->gather_rows_px;
  mat->tuned[padded_width(t->K) * 2 + (t->a_precision == APPGA_PREC_BF16 ? 1 : 0)] = sch;
  return APPGA_OK;
}
