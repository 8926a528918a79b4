// C ABI of the APPGA library: contexts, matrix handles, parameter checks,
// single-step entry points and the graph-driven single-slice solver.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>

#include "appga.h"
#include "appga_internal.h"
#include "handles.h"

using appga::cuda_fail;
using appga::dalloc;
using appga::DevCSR;
using appga::fail;
using appga::SolverState;
using appga::Workspace;

namespace {
thread_local std::string g_last_error;
constexpr int kDefaultGraphIters = 16;
}  // namespace

// The solver loop streams 2-byte packed column indices where the matrix
// allows (1), or 4-byte indices always (0).
#ifndef APPGA_PACK
#define APPGA_PACK 1
#endif
// The single-slice solver finalises each step in the pixel phase's first
// blocks (1) or in a separate one-block kernel (0).
#ifndef APPGA_FUSE_FIN
#define APPGA_FUSE_FIN 1
#endif

namespace appga {
void set_error(const std::string& msg) { g_last_error = msg; }

appga_status fail(appga_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

appga_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return APPGA_ENOMEM;
  if (e == cudaErrorNoDevice || e == cudaErrorInvalidDevice || e == cudaErrorInsufficientDriver)
    return APPGA_ENODEV;
  return APPGA_ECUDA;
}
}  // namespace appga

namespace appga {

#define CK(call) APPGA_CK(call)

void free_csr(DevCSR& c) {
  cudaFree(c.row_ptr);
  cudaFree(c.col);
  cudaFree(c.val);
  cudaFree(c.val_bf16);
  c = DevCSR();
}

void free_sell(DevSell& c) {
  cudaFree(c.off);
  cudaFree(c.cols);
  cudaFree(c.cols32);
  cudaFree(c.vals);
  cudaFree(c.vals_bf16);
  c = DevSell();
}

appga_status upload_sell(const appga::HostSell& h, bool bf16, DevSell* out, int64_t* bytes) {
  DevSell c;
  c.rows = h.rows;
  c.slices = h.slices;
  const size_t np = h.vals.size() / appga::PACK_ENTRIES;
  cudaError_t e = dalloc(&c.off, h.off.size(), bytes);
  if (e == cudaSuccess && !h.cols.empty()) e = dalloc(&c.cols, np, bytes);
  if (e == cudaSuccess && !h.cols32.empty()) e = dalloc(&c.cols32, np, bytes);
  if (e == cudaSuccess) e = dalloc(&c.vals, np, bytes);
  if (e == cudaSuccess && bf16) e = dalloc(&c.vals_bf16, np, bytes);
  if (e == cudaSuccess)
    e = cudaMemcpy(c.off, h.off.data(), h.off.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !h.cols.empty())
    e = cudaMemcpy(c.cols, h.cols.data(), np * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !h.cols32.empty())
    e = cudaMemcpy(c.cols32, h.cols32.data(), np * 16, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && np)
    e = cudaMemcpy(c.vals, h.vals.data(), np * 16, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && bf16 && np) {
    std::vector<uint16_t> b(h.vals.size());
    for (size_t i = 0; i < b.size(); ++i) b[i] = appga::float_to_bf16(h.vals[i]);
    e = cudaMemcpy(c.vals_bf16, b.data(), np * 8, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    free_sell(c);
    return cuda_fail(e, "sliced matrix upload");
  }
  *out = c;
  return APPGA_OK;
}

void free_workspace(Workspace& ws) {
  for (auto& kv : ws.gexec) cudaGraphExecDestroy(kv.second);
  ws.gexec.clear();
  for (auto& kv : ws.call_graphs) cudaGraphExecDestroy(kv.second);
  ws.call_graphs.clear();
  ws.call_seen.clear();
  for (auto& p : ws.f) cudaFree(p);
  for (auto& p : ws.y) cudaFree(p);
  cudaFree(ws.w);
  cudaFree(ws.gR);
  cudaFree(ws.pfreeze);
  cudaFree(ws.ft);
  cudaFree(ws.fpair);
  cudaFree(ws.partial_p);
  cudaFree(ws.partial_r);
  cudaFree(ws.partial_aux);
  cudaFree(ws.gtick);
  cudaFree(ws.scalars);
  cudaFree(ws.theta_tab);
  cudaFree(ws.st);
  cudaFree(ws.st_scratch);
  cudaFree(ws.flag);
  cudaFree(ws.d_g);
  cudaFree(ws.d_gamma);
  cudaFree(ws.d_finit);
  cudaFree(ws.d_fout);
  cudaFreeHost(ws.st_host);
  cudaFreeHost(ws.flag_host);
  cudaFreeHost(ws.scalars_host);
  ws = Workspace();
}

appga_status upload_csr(const appga::HostCSR& h, bool bf16, DevCSR* out, int64_t* bytes) {
  DevCSR c;
  c.rows = h.rows;
  c.cols = h.cols;
  c.nnz_padded = (int64_t)h.col.size();
  cudaError_t e;
  if ((e = dalloc(&c.row_ptr, h.row_ptr.size(), bytes)) != cudaSuccess ||
      (e = dalloc(&c.col, h.col.size(), bytes)) != cudaSuccess ||
      (e = dalloc(&c.val, h.val.size(), bytes)) != cudaSuccess) {
    free_csr(c);
    return cuda_fail(e, "cudaMalloc(matrix)");
  }
  if (bf16) {
    if ((e = dalloc(&c.val_bf16, h.val.size(), bytes)) != cudaSuccess) {
      free_csr(c);
      return cuda_fail(e, "cudaMalloc(matrix bf16)");
    }
  }
  e = cudaMemcpy(c.row_ptr, h.row_ptr.data(), h.row_ptr.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !h.col.empty())
    e = cudaMemcpy(c.col, h.col.data(), h.col.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !h.val.empty())
    e = cudaMemcpy(c.val, h.val.data(), h.val.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && bf16 && !h.val.empty()) {
    std::vector<uint16_t> b(h.val.size());
    for (size_t i = 0; i < b.size(); ++i) b[i] = appga::float_to_bf16(h.val[i]);
    e = cudaMemcpy(c.val_bf16, b.data(), b.size() * 2, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    free_csr(c);
    return cuda_fail(e, "cudaMemcpy(matrix)");
  }
  *out = c;
  return APPGA_OK;
}

appga_status ensure_workspace(appga_matrix* M) {
  Workspace& ws = M->ws;
  if (ws.ready) return APPGA_OK;
  const int m = M->m, d = M->d;
  const int np = appga::max_partials(m, M->n);
  cudaError_t e = cudaSuccess;
  int64_t* b = &M->bytes;
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = dalloc(&ws.f[i], (size_t)d, b);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = dalloc(&ws.y[i], (size_t)m, b);
  if (e == cudaSuccess) e = dalloc(&ws.w, (size_t)m, b);
  if (e == cudaSuccess) e = dalloc(&ws.gR, (size_t)d, b);
  if (e == cudaSuccess) e = dalloc(&ws.pfreeze, (size_t)d, b);
  if (e == cudaSuccess) e = dalloc(&ws.ft, (size_t)appga::tiled_size(M->n), b);
  if (e == cudaSuccess && M->fold_t.off != nullptr)
    e = dalloc(&ws.fpair, (size_t)appga::tiled_size(M->n), b);
  if (e == cudaSuccess) e = dalloc(&ws.partial_p, (size_t)np, b);
  if (e == cudaSuccess) e = dalloc(&ws.partial_r, (size_t)np, b);
  if (e == cudaSuccess) e = dalloc(&ws.partial_aux, (size_t)np, b);
  const int ng = appga::max_group_tickets(m, M->n);
  if (e == cudaSuccess) e = dalloc(&ws.gtick, (size_t)ng, b);
  if (e == cudaSuccess) e = cudaMemset(ws.gtick, 0, (size_t)ng * sizeof(unsigned int));
  if (e == cudaSuccess) e = dalloc(&ws.scalars, 8, b);
  if (e == cudaSuccess) e = dalloc(&ws.st, 1, b);
  if (e == cudaSuccess) e = dalloc(&ws.st_scratch, 1, b);
  if (e == cudaSuccess) e = dalloc(&ws.flag, 1, b);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ws.st_host, sizeof(SolverState));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ws.flag_host, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ws.scalars_host, 8 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(ws.st, 0, sizeof(SolverState));
  if (e == cudaSuccess) e = cudaMemset(ws.st_scratch, 0, sizeof(SolverState));
  if (e != cudaSuccess) {
    free_workspace(ws);
    return cuda_fail(e, "workspace allocation");
  }
  ws.m = m;
  ws.d = d;
  ws.ready = true;
  return APPGA_OK;
}

appga::IterParams iter_params(const appga_params* p, bool track) {
  appga::IterParams ip{};
  ip.lambda1 = (float)p->lambda1;
  ip.lambda2 = (float)p->lambda2;
  ip.eps = (float)p->eps;
  ip.beta = (float)p->beta;
  ip.omega = p->omega;
  ip.a = p->a;
  ip.b = p->b;
  ip.rel_tol = p->rel_obj_tol;
  ip.momentum = p->momentum;
  ip.freeze_iter = p->precond_freeze_iter;
  ip.track = track ? 1 : 0;
  return ip;
}

bool bf16_requested(const appga_matrix* M, const appga_params* p) {
  return p->a_precision == APPGA_PREC_BF16 && M->has_bf16;
}

bool loop_gathers_copy() { return tiled_gather_enabled(); }

void loop_layout(const appga_matrix* M, FwdArgs* fa, PixArgs* pa) {
  if (!tiled_gather_enabled()) return;  // the CSR with row-major columns
  const Workspace& ws = M->ws;
  // the loop's projector gathers f^k from its 8 x 8-tiled copy (as pairs
  // when folded)
  fa->A.col = M->A_tiled.col;
  if (M->fold_t.off != nullptr && ws.fpair != nullptr) {
    fa->S = M->fold_a;
    fa->fpair = ws.fpair;
    fa->fold_half = M->m / 2;
    fa->fold_nb = M->fold_nb;
    fa->ft = nullptr;
    pa->S = M->fold_t;
    pa->fpair = ws.fpair;
    pa->ft = nullptr;
  } else {
    fa->S = M->sell_a;
    fa->ft = ws.ft;
    pa->S = M->sell_t;
    pa->ft = ws.ft;
  }
}

cudaError_t loop_gather_copy(const appga_matrix* M, const float* f, cudaStream_t s) {
  if (!tiled_gather_enabled()) return cudaSuccess;
  if (M->fold_t.off != nullptr && M->ws.fpair != nullptr)
    return launch_to_fold_pairs(f, M->ws.fpair, M->n, s);
  return launch_to_tiled(f, M->ws.ft, M->n, s);
}

appga::FwdArgs fwd_args(appga_matrix* M, bool bf16) {
  appga::FwdArgs a{};
  a.A = M->A;
  a.use_bf16 = bf16 ? 1 : 0;
  return a;
}

// A cache key as the raw bytes of the values it depends on (exact, and no
// text formatting on the per-call path).
struct KeyBytes {
  std::string s;
  template <class T>
  KeyBytes& add(const T& v) {
    s.append(reinterpret_cast<const char*>(&v), sizeof v);
    return *this;
  }
};

std::string graph_key(const appga_params* p, bool track, bool bf16, int S) {
  KeyBytes k;
  k.add((int)track).add((int)bf16).add(S).add(p->lambda1).add(p->lambda2).add(p->eps);
  k.add(p->beta).add(p->omega).add(p->a).add(p->b).add(p->rel_obj_tol).add(p->momentum);
  k.add(p->precond_freeze_iter);
  return k.s;
}

// Device state of a run at its start (iteration index k0).  A run of zero
// maps with the objective tracked starts at done = 2: its one forward phase
// and the last finalisation still evaluate Phi(f^{k0}).
SolverState start_state(int32_t k0, const appga_params* p) {
  const bool track = p->track_objective != 0 || p->rel_obj_tol > 0.0;
  SolverState h{};
  h.k = k0;
  h.k0 = k0;
  h.k_last = k0 + p->max_iters - 1;
  h.done = p->max_iters == 0 ? (track ? 2 : 1) : 0;
  h.k_next = k0;
  h.done_next = h.done;
  h.result_k = k0;
  h.phi_cur = std::numeric_limits<double>::quiet_NaN();
  h.phi_prev = h.phi_cur;
  return h;
}

// Prepares a run on the workspace ring whose slots (k0-1)%3 and k0%3 hold
// f^{k0-1} and f^{k0} (and, if tiled_ready, whose tiled copy holds f^{k0}),
// with the device state already started: y^{k0-1} (a resumed run only; a
// fresh run has f^{k0-1} = f^{k0}), y^{k0}, w^{k0} and F(f^{k0}); fills the
// kernel argument blocks of the loop.
appga_status setup_run(appga_matrix* M, const float* g, const float* gamma, int32_t k0,
                       const appga_params* p, bool fresh, bool tiled_ready,
                       appga::FwdArgs* fa_out, appga::PixArgs* pa_out) {
  Workspace& ws = M->ws;
  cudaStream_t s = M->ctx->stream;
  const bool track = p->track_objective != 0 || p->rel_obj_tol > 0.0;
  const bool bf16 = bf16_requested(M, p);

  if (!fresh) {
    // y^{k0-1} = A f^{k0-1}, with the loop's projection (the same matrix
    // layout, gather order and accumulation), so a resumed run continues an
    // uninterrupted one bit for bit
    appga::FwdArgs init = fwd_args(M, bf16);
    init.f[0] = ws.f[(k0 + 2) % 3];
    init.y[0] = ws.y[(k0 + 1) & 1];
    init.y_out = nullptr;
    init.g = g;
    init.gamma = gamma;
    init.st = ws.st_scratch;
    init.partial = ws.partial_aux;
    init.gtick = ws.gtick;
    init.loop = 0;
    init.solver_acc = 1;
    init.n = M->n;
    appga::PixArgs unused{};
    appga::loop_layout(M, &init, &unused);
    CK(appga::loop_gather_copy(M, ws.f[(k0 + 2) % 3], s));
    CK(appga::launch_forward(init, s));
  }

  appga::FwdArgs fa = fwd_args(M, bf16);
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
  fa.want_data = track ? 1 : 0;
  fa.gR = ws.gR;
  fa.n = M->n;
  fa.ip = iter_params(p, track);
  fa.theta_tab = ws.theta_tab;

  appga::PixArgs pa{};
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
  pa.fwd_partial = ws.partial_r;
  pa.theta_tab = ws.theta_tab;
  pa.ip = iter_params(p, track);
  pa.use_bf16 = bf16 ? 1 : 0;
  pa.fuse_fin = APPGA_FUSE_FIN;
  appga::loop_layout(M, &fa, &pa);
  if (!tiled_ready) CK(appga::loop_gather_copy(M, ws.f[k0 % 3], s));
  pa.n_fwd_partial =
      appga::forward_blocks(fa.S.off != nullptr ? fa.S.rows : M->m, M->n, fa.S.off != nullptr);

  // w^{k0}, y^{k0}, B^T grad phi~(B f~^{k0}) and Phi(f^{k0})
  appga::FwdArgs first = fa;
  first.fresh_first = fresh ? 1 : 0;
  CK(appga::launch_forward(first, s));
  *fa_out = fa;
  *pa_out = pa;
  return APPGA_OK;
}

// Calls of at most this many maps (and no stopping tolerance) are captured
// whole into a call graph once their arguments repeat; at most
// kCallGraphCache such graphs are kept per matrix.
constexpr int kCallGraphMaxMaps = 64;
constexpr size_t kCallGraphCache = 8;

// Executable graph of `maps` solver maps (pixel phase, finalisation, forward
// phase) for the loop arguments of `key`, captured on first use.
appga_status loop_graph(Workspace& ws, const std::string& key, int maps,
                        const appga::FwdArgs& fa, const appga::PixArgs& pa, cudaStream_t s,
                        cudaGraphExec_t* out) {
  if (ws.gkey != key) {
    for (auto& kv : ws.gexec) cudaGraphExecDestroy(kv.second);
    ws.gexec.clear();
    ws.gkey = key;
  }
  auto it = ws.gexec.find(maps);
  if (it != ws.gexec.end()) {
    *out = it->second;
    return APPGA_OK;
  }
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < maps && e == cudaSuccess; ++i) {
    e = appga::launch_pixel(pa, s);
    if (e == cudaSuccess) e = appga::launch_forward(fa, s);
  }
  const cudaError_t e2 = cudaStreamEndCapture(s, &graph);
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(e, "graph capture");
  }
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  ws.gexec[maps] = exec;
  *out = exec;
  return APPGA_OK;
}

// Graph replays of a run of `total` maps: whole replays of S maps, then the
// remainder as replays of its binary digits (so exactly `total` maps run).
std::vector<int> replay_plan(int total, int S) {
  std::vector<int> plan((size_t)(total / S), S);
  const int rem = total % S;
  for (int b = 1 << 30; b > 0; b >>= 1)
    if (rem & b) plan.push_back(b);
  return plan;
}

// Runs the maps of a prepared run (setup_run) on ctx->stream, then the last
// finalisation of a tracked run.  With a stopping tolerance the stop flag is
// polled one replay behind, so the device never idles on the host.
appga_status run_maps(appga_matrix* M, const float* g, const float* gamma,
                      const appga_params* p, const appga::FwdArgs& fa, const appga::PixArgs& pa) {
  appga_ctx* ctx = M->ctx;
  Workspace& ws = M->ws;
  cudaStream_t s = ctx->stream;
  const bool track = p->track_objective != 0 || p->rel_obj_tol > 0.0;
  const bool bf16 = bf16_requested(M, p);
  const int S = p->graph_iters > 0 ? p->graph_iters : kDefaultGraphIters;
  if (p->max_iters > 0) {
    // the captured kernel arguments hold the g / gamma addresses
    KeyBytes kb;
    kb.s = graph_key(p, track, bf16, S);
    kb.add(g).add(gamma).add(ws.theta_tab);
    const std::string& key = kb.s;
    // the whole ladder (S and every power of two below it) is captured on
    // first use of these arguments, so later calls of any length find their
    // graphs cached
    cudaGraphExec_t unused = nullptr;
    appga_status rc0 = loop_graph(ws, key, S, fa, pa, s, &unused);
    for (int b = 1; b < S && rc0 == APPGA_OK; b *= 2) rc0 = loop_graph(ws, key, b, fa, pa, s, &unused);
    if (rc0 != APPGA_OK) return rc0;
    const std::vector<int> plan = replay_plan(p->max_iters, S);
    std::vector<cudaGraphExec_t> execs(plan.size());
    for (size_t r = 0; r < plan.size(); ++r) {
      const appga_status rc = loop_graph(ws, key, plan[r], fa, pa, s, &execs[r]);
      if (rc != APPGA_OK) return rc;
    }
    if (p->rel_obj_tol > 0.0) {
      cudaEvent_t ev[2];
      CK(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
      SolverState* hs = ws.st_host;
      hs->done = 0;
      appga_status rc = APPGA_OK;
      for (size_t r = 0; r < execs.size(); ++r) {
        cudaError_t e = cudaGraphLaunch(execs[r], s);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(&hs->done, &ws.st->done, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaEventRecord(ev[r & 1], s);
        if (e != cudaSuccess) {
          rc = cuda_fail(e, "graph replay");
          break;
        }
        if (r >= 1) {
          e = cudaEventSynchronize(ev[(r - 1) & 1]);
          if (e != cudaSuccess) {
            rc = cuda_fail(e, "cudaEventSynchronize");
            break;
          }
          if (hs->done) break;
        }
      }
      cudaEventDestroy(ev[0]);
      cudaEventDestroy(ev[1]);
      if (rc != APPGA_OK) return rc;
    } else {
      for (cudaGraphExec_t x : execs) CK(cudaGraphLaunch(x, s));
    }
  }
  if (track) CK(appga::launch_finalize(pa, s));
  return APPGA_OK;
}

// Statistics of a finished run from its final device state.
appga_status finish_stats(const SolverState& fin, int32_t k0, const appga_params* p,
                          appga_stats* stats) {
  const bool track = p->track_objective != 0 || p->rel_obj_tol > 0.0;
  if (stats) {
    stats->iters = fin.result_k - k0;
    stats->result_k = fin.result_k;
    stats->stopped_early = fin.stopped_early;
    stats->flags = fin.flags;
    stats->guard_hits = (int64_t)fin.guard_hits;
    stats->phi = track ? fin.phi_cur : std::numeric_limits<double>::quiet_NaN();
    stats->phi_prev = track ? fin.phi_prev : std::numeric_limits<double>::quiet_NaN();
  }
  if (fin.flags & APPGA_FLAG_DOMAIN)
    return fail(APPGA_EDOMAIN,
                "inputs must satisfy: g finite and >= 0, gamma finite and > 0, f finite and >= 0");
  if (fin.flags & APPGA_FLAG_TIMEOUT)
    return fail(APPGA_ETIMEOUT, "a bounded device wait ran out; the run stopped");
  if (fin.flags & APPGA_FLAG_NONFINITE)
    return fail(APPGA_ENUMERIC, "a non-finite value appeared in the iteration");
  return APPGA_OK;
}

appga_status momentum_table(appga_matrix* M, SolverState* st, int k0, const appga_params* p,
                            cudaStream_t s, const SolverState* init) {
  Workspace& ws = M->ws;
  const int need = p->max_iters + 1;
  if (ws.theta_cap < need) {
    // captured call graphs read the old table: drop them with it
    for (auto& kv : ws.call_graphs) cudaGraphExecDestroy(kv.second);
    ws.call_graphs.clear();
    cudaFree(ws.theta_tab);
    ws.theta_tab = nullptr;
    ws.theta_cap = 0;
    const int cap = need < 1024 ? 1024 : need;
    const cudaError_t e = cudaMalloc((void**)&ws.theta_tab, (size_t)cap * sizeof(ThetaEntry));
    if (e != cudaSuccess) return cuda_fail(e, "momentum table");
    ws.theta_cap = cap;
  }
  CK(launch_theta_table(st, ws.theta_tab, k0, p->max_iters, p->momentum, p->a, p->b, p->omega, s,
                        init));
  return APPGA_OK;
}

appga_status check_params_and_mat(appga_ctx* ctx, const appga_matrix* M, const appga_params* p) {
  if (ctx == nullptr || M == nullptr || p == nullptr)
    return fail(APPGA_EINVAL, "null context, matrix or params");
  if (M->ctx != ctx) return fail(APPGA_EINVAL, "matrix belongs to another context");
  return appga_params_validate(p);
}

appga_status validate_inputs(appga_matrix* M, const float* g, const float* gamma, const float* f,
                             cudaStream_t s) {
  Workspace& ws = M->ws;
  CK(cudaMemsetAsync(ws.flag, 0, sizeof(int), s));
  CK(appga::launch_validate_inputs(g, gamma, M->m, f, M->d, ws.flag, s));
  CK(cudaMemcpyAsync(ws.flag_host, ws.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (*ws.flag_host)
    return fail(APPGA_EDOMAIN,
                "inputs must satisfy: g finite and >= 0, gamma finite and > 0, f finite and >= 0");
  return APPGA_OK;
}

}  // namespace appga

using namespace appga;

namespace appga {
// Orders ctx->stream after the caller's stream.
appga_status enter_stream(appga_ctx* ctx, void* stream) {
  cudaStream_t us = (cudaStream_t)stream;
  CK(cudaSetDevice(ctx->device));
  CK(cudaEventRecord(ctx->ev_in, us));
  CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_in, 0));
  return APPGA_OK;
}
// Orders the caller's stream after ctx->stream.
appga_status leave_stream(appga_ctx* ctx, void* stream) {
  cudaStream_t us = (cudaStream_t)stream;
  CK(cudaEventRecord(ctx->ev_out, ctx->stream));
  CK(cudaStreamWaitEvent(us, ctx->ev_out, 0));
  return APPGA_OK;
}

appga_status objective_terms(appga_matrix* M, int K, const float* f, const float* g,
                             const float* gamma, const appga_params* p, bool with_reg,
                             double* dev_out, cudaStream_t s) {
  appga_status rc = ensure_workspace(M);
  if (rc != APPGA_OK) return rc;
  Workspace& ws = M->ws;
  const bool bf16 = bf16_requested(M, p);
  for (int i = 0; i < K; ++i) {
    const float* fi = f + (size_t)i * M->d;
    FwdArgs a = fwd_args(M, bf16);
    a.f[0] = fi;
    a.y[0] = nullptr;
    a.y_out = nullptr;
    a.g = g + (size_t)i * M->m;
    a.gamma = gamma + (size_t)i * M->m;
    a.st = ws.st_scratch;
    a.partial = ws.partial_aux;
    a.gtick = ws.gtick;
    a.data_out = dev_out + 2 * i;
    a.loop = 0;
    a.want_data = 1;
    a.n = M->n;
    CK(launch_forward(a, s));
    if (with_reg)
      CK(launch_reg_term(M->n, fi, (float)p->lambda1, (float)p->lambda2, (float)p->eps,
                         ws.partial_aux, ws.gtick, ws.st_scratch, dev_out + 2 * i + 1, s));
  }
  return APPGA_OK;
}

}  // namespace appga

namespace {
using appga::enter_stream;
using appga::leave_stream;

appga_status objective_on(appga_matrix* M, const float* f, const float* g, const float* gamma,
                          const appga_params* p, double* phi, cudaStream_t s) {
  Workspace& ws = M->ws;
  appga::FwdArgs a = fwd_args(M, bf16_requested(M, p));
  a.f[0] = f;
  a.y[0] = nullptr;
  a.y_out = nullptr;
  a.g = g;
  a.gamma = gamma;
  a.st = ws.st_scratch;
  a.partial = ws.partial_aux;
  a.gtick = ws.gtick;
  a.data_out = ws.scalars;
  a.loop = 0;
  a.want_data = 1;
  a.n = M->n;
  CK(appga::launch_forward(a, s));
  CK(appga::launch_reg_term(M->n, f, (float)p->lambda1, (float)p->lambda2, (float)p->eps,
                            ws.partial_aux, ws.gtick, ws.st_scratch, ws.scalars + 1, s));
  CK(cudaMemcpyAsync(ws.scalars_host, ws.scalars, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *phi = ws.scalars_host[0] + ws.scalars_host[1];
  return APPGA_OK;
}

// One solver call on ctx->stream after the caller's stream: start state and
// momentum table, input check (on the device: no host round trip), f^{k0-1}
// and f^{k0}, the first forward phase, exactly max_iters maps, the result
// copied out on the device (and to f_out_host if given), one synchronisation.
appga_status solve_common(appga_ctx* ctx, appga_matrix* M, const float* g, const float* gamma,
                          const float* f_prev, const float* f_cur, int32_t k0,
                          const appga_params* p, float* f_out_prev, float* f_out,
                          appga_stats* stats, void* stream, bool fresh,
                          float* f_out_host = nullptr) {
  appga_status rc = check_params_and_mat(ctx, M, p);
  if (rc != APPGA_OK) return rc;
  if (g == nullptr || gamma == nullptr || f_out == nullptr)
    return fail(APPGA_EINVAL, "g, gamma and f_out must be non-NULL");
  if (!fresh && (f_prev == nullptr || f_cur == nullptr))
    return fail(APPGA_EINVAL, "resume needs f_prev and f_cur");
  if (k0 < 1) return fail(APPGA_EINVAL, "k0 must be >= 1");
  if (p->precond_freeze_iter >= 0 && k0 > p->precond_freeze_iter)
    return fail(APPGA_EINVAL, "resume past the preconditioner freeze iteration is not supported");
  if ((rc = ensure_workspace(M)) != APPGA_OK) return rc;
  if ((rc = enter_stream(ctx, stream)) != APPGA_OK) return rc;
  cudaStream_t s = ctx->stream;
  Workspace& ws = M->ws;
  const size_t fb = (size_t)M->d * sizeof(float);
  // The whole call: start state and momentum table, f^{k0-1} and f^{k0},
  // the first forward phase, the maps (as graph replays, or launched one by
  // one when `direct`, inside a call graph), the last finalisation, the
  // result and the state read-back.
  auto enqueue = [&](bool direct) -> appga_status {
    const SolverState h = start_state(k0, p);
    appga_status r = momentum_table(M, ws.st, k0, p, s, &h);
    if (r != APPGA_OK) return r;
    float* slot_cur = ws.f[k0 % 3];
    float* slot_prev = ws.f[(k0 + 2) % 3];
    bool tiled_ready = false;
    if (fresh && f_cur == nullptr) {
      // TMC * 1_disk into f^{k0}, f^{k0-1} and the loop's gather copy; g
      // and gamma are checked in the same pass
      appga::FwdArgs lf{};
      appga::PixArgs lp{};
      appga::loop_layout(M, &lf, &lp);
      CK(appga::launch_initial_image(g, gamma, M->m, M->n, M->na, M->npfov, ws.partial_aux,
                                     ws.gtick, ws.st_scratch, slot_cur, s, slot_prev, lp.ft,
                                     ws.st, lp.fpair));
      tiled_ready = appga::loop_gathers_copy();
    } else {
      CK(appga::launch_check_inputs(g, gamma, M->m, f_cur, fresh ? nullptr : f_prev, M->d,
                                    ws.st, s));
      CK(cudaMemcpyAsync(slot_cur, f_cur, fb, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(slot_prev, fresh ? f_cur : f_prev, fb, cudaMemcpyDeviceToDevice, s));
    }
    appga::FwdArgs fa;
    appga::PixArgs pa;
    if ((r = setup_run(M, g, gamma, k0, p, fresh, tiled_ready, &fa, &pa)) != APPGA_OK) return r;
    if (direct) {
      for (int i = 0; i < p->max_iters; ++i) {
        CK(appga::launch_pixel(pa, s));
        CK(appga::launch_forward(fa, s));
      }
      if (p->track_objective != 0) CK(appga::launch_finalize(pa, s));
    } else if ((r = run_maps(M, g, gamma, p, fa, pa)) != APPGA_OK) {
      return r;
    }
    CK(appga::launch_copy_result(ws.st, ws.f, f_out, f_out_prev, M->d, s));
    if (f_out_host) CK(cudaMemcpyAsync(f_out_host, f_out, fb, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ws.st_host, ws.st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
    return APPGA_OK;
  };
  // A short call without a stopping tolerance whose arguments keep repeating
  // is replayed as one captured graph (one launch instead of a dozen):
  // captured on the third call with the same arguments, so every one-time
  // set-up of the kernels has run before and a single repeat does not pay
  // for the capture.  A host result buffer must be pinned.
  bool pinned_out = f_out_host == nullptr;
  if (!pinned_out) {
    cudaPointerAttributes pat{};
    pinned_out = cudaPointerGetAttributes(&pat, f_out_host) == cudaSuccess &&
                 pat.type == cudaMemoryTypeHost;
    cudaGetLastError();  // clear a failed query
  }
  const bool whole = p->max_iters > 0 && p->max_iters <= kCallGraphMaxMaps &&
                     p->rel_obj_tol <= 0.0 && pinned_out;
  std::string ckey;
  if (whole) {
    const bool track = p->track_objective != 0;
    KeyBytes kb;
    kb.s = graph_key(p, track, bf16_requested(M, p), 0);
    kb.add(k0).add((int)fresh).add(p->max_iters).add(g).add(gamma).add(f_prev).add(f_cur);
    kb.add(f_out_prev).add(f_out).add(f_out_host);
    ckey = std::move(kb.s);
  }
  auto it = whole ? ws.call_graphs.find(ckey) : ws.call_graphs.end();
  const auto seen = whole ? ws.call_seen.find(ckey) : ws.call_seen.end();
  if (whole && (it != ws.call_graphs.end() ||
                (seen != ws.call_seen.end() && seen->second >= 2))) {
    if (it == ws.call_graphs.end()) {
      // the momentum table is grown outside the capture
      const int need = p->max_iters + 1;
      if (ws.theta_cap < need && (rc = momentum_table(M, ws.st_scratch, k0, p, s)) != APPGA_OK)
        return rc;
      if (ws.call_graphs.size() >= kCallGraphCache) {
        for (auto& kv : ws.call_graphs) cudaGraphExecDestroy(kv.second);
        ws.call_graphs.clear();
      }
      cudaGraph_t graph = nullptr;
      CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      const appga_status rq = enqueue(true);
      const cudaError_t e2 = cudaStreamEndCapture(s, &graph);
      if (rq != APPGA_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rq;
      }
      if (e2 != cudaSuccess) return cuda_fail(e2, "call graph capture");
      cudaGraphExec_t exec = nullptr;
      const cudaError_t e3 = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e3 != cudaSuccess) return cuda_fail(e3, "call graph instantiation");
      it = ws.call_graphs.emplace(ckey, exec).first;
    }
    CK(cudaGraphLaunch(it->second, s));
  } else {
    if (whole) {
      if (ws.call_seen.size() >= 4 * kCallGraphCache && seen == ws.call_seen.end())
        ws.call_seen.clear();
      ++ws.call_seen[ckey];
    }
    if ((rc = enqueue(false)) != APPGA_OK) return rc;
  }
  if ((rc = leave_stream(ctx, stream)) != APPGA_OK) return rc;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  const SolverState fin = *ws.st_host;
  return finish_stats(fin, k0, p, stats);
}

}  // namespace

extern "C" {

const char* appga_status_string(appga_status s) {
  switch (s) {
    case APPGA_OK: return "ok";
    case APPGA_EINVAL: return "invalid argument";
    case APPGA_ENOMEM: return "out of memory";
    case APPGA_EDOMAIN: return "input outside the model's domain";
    case APPGA_ETIMEOUT: return "timed out";
    case APPGA_ECUDA: return "CUDA runtime error";
    case APPGA_ENODEV: return "no usable CUDA device";
    case APPGA_EBUSY: return "resource busy";
    case APPGA_ENUMERIC: return "non-finite intermediate";
  }
  return "unknown status";
}

const char* appga_last_error(void) { return g_last_error.c_str(); }

const char* appga_version(void) { return "0.1.0"; }

void appga_params_default(appga_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->lambda1 = 0.1;
  p->lambda2 = 0.05;
  p->eps = 1e-3;
  p->omega = 0.5;
  p->a = 0.125;
  p->b = 1.0;
  p->beta = 1.0;
  p->max_iters = 100;
  p->rel_obj_tol = 0.0;
  p->precond_freeze_iter = -1;
  p->a_precision = APPGA_PREC_FP32;
  p->momentum = APPGA_MOMENTUM_GN;
  p->track_objective = 0;
  p->graph_iters = 0;
}

appga_status appga_params_validate(const appga_params* p) {
  if (!p) return fail(APPGA_EINVAL, "params is NULL");
  auto fin = [](double x) { return std::isfinite(x); };
  if (!fin(p->lambda1) || p->lambda1 < 0 || !fin(p->lambda2) || p->lambda2 < 0)
    return fail(APPGA_EINVAL, "lambda1 and lambda2 must be finite and >= 0");
  if (!fin(p->eps) || !(p->eps > 0)) return fail(APPGA_EINVAL, "eps must be finite and > 0");
  if (!fin(p->beta) || !(p->beta > 0)) return fail(APPGA_EINVAL, "beta must be finite and > 0");
  if (p->max_iters < 0) return fail(APPGA_EINVAL, "max_iters must be >= 0");
  if (!fin(p->rel_obj_tol) || p->rel_obj_tol < 0)
    return fail(APPGA_EINVAL, "rel_obj_tol must be finite and >= 0");
  if (p->precond_freeze_iter < -1 || p->precond_freeze_iter == 0)
    return fail(APPGA_EINVAL, "precond_freeze_iter must be -1 or >= 1");
  if (p->a_precision != APPGA_PREC_FP32 && p->a_precision != APPGA_PREC_BF16)
    return fail(APPGA_EINVAL, "a_precision must be APPGA_PREC_FP32 or APPGA_PREC_BF16");
  if (p->graph_iters < 0 || p->graph_iters > 4096)
    return fail(APPGA_EINVAL, "graph_iters must be in [0, 4096]");
  if (p->momentum == APPGA_MOMENTUM_GN) {
    if (!fin(p->omega) || !(p->omega > 0) || p->omega > 1)
      return fail(APPGA_EINVAL, "omega must be in (0, 1]");
    if (!fin(p->a) || !(p->a > 0)) return fail(APPGA_EINVAL, "a must be > 0");
    if (p->omega == 1.0 && !(p->a < 0.5))
      return fail(APPGA_EINVAL, "a must be < 1/2 when omega = 1 (Thm. 10)");
    if (!fin(p->b)) return fail(APPGA_EINVAL, "b must be finite");
    if (p->b <= 0 && p->b > -p->a * 1e12) {
      // b must keep t_k = a k^omega + b away from zero for every k >= 1
      // (Lemma on t_k): reject b equal to -a k^omega for some k.
      const double q = std::pow(-p->b / p->a, 1.0 / p->omega);
      if (std::fabs(q - std::round(q)) < 1e-12 && std::round(q) >= 1.0)
        return fail(APPGA_EINVAL, "b = -a k^omega for some k makes t_k vanish");
    }
  } else if (p->momentum != APPGA_MOMENTUM_NONE && p->momentum != APPGA_MOMENTUM_NESTEROV) {
    return fail(APPGA_EINVAL, "unknown momentum rule");
  }
  return APPGA_OK;
}

double appga_gn_theta(int32_t k, double a, double b, double omega) {
  const double t_prev = a * std::pow((double)(k - 1), omega) + b;
  const double t = a * std::pow((double)k, omega) + b;
  return (t_prev - 1.0) / t;
}

appga_status appga_ctx_create(int32_t device, appga_ctx** out) {
  if (!out) return fail(APPGA_EINVAL, "out is NULL");
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || count == 0) return fail(APPGA_ENODEV, "no CUDA device is visible");
  if (device < 0 || device >= count) return fail(APPGA_ENODEV, "device index out of range");
  CK(cudaSetDevice(device));
  auto* ctx = new appga_ctx();
  ctx->device = device;
  e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    appga_ctx_destroy(ctx);
    return cuda_fail(e, "context setup");
  }
  *out = ctx;
  return APPGA_OK;
}

appga_status appga_ctx_destroy(appga_ctx* ctx) {
  if (!ctx) return APPGA_OK;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
  if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
  delete ctx;
  return APPGA_OK;
}

appga_status appga_matrix_create(appga_ctx* ctx, int32_t m, int32_t d, int32_t n_side,
                                 int32_t n_angles, const int32_t* row_ptr_host,
                                 const int32_t* col_host, const float* val_host, uint32_t flags,
                                 appga_matrix** out) {
  if (!ctx || !out) return fail(APPGA_EINVAL, "null context or out");
  *out = nullptr;
  if (n_side <= 0 || (int64_t)n_side * n_side != d)
    return fail(APPGA_EINVAL, "d must equal n_side * n_side");
  if (n_angles <= 0) return fail(APPGA_EINVAL, "n_angles must be > 0");
  if (m <= 0) return fail(APPGA_EINVAL, "m must be > 0");
  if ((flags & ~(APPGA_A_BF16_COPY | APPGA_A_NO_FOLD)) != 0)
    return fail(APPGA_EINVAL, "unknown flags");
  std::string why;
  appga_status rc = appga::validate_csr(m, d, row_ptr_host, col_host, val_host, &why);
  if (rc != APPGA_OK) return fail(rc, why);
  const int64_t nnz = row_ptr_host[m];
  // padded sizes must stay below 2^31 for int32 offsets
  if (nnz + 4ll * (m > d ? m : d) >= (1ll << 31))
    return fail(APPGA_EINVAL, "nnz too large for int32 row offsets");
  CK(cudaSetDevice(ctx->device));
  appga::HostCSR at, pa, pt;
  appga::transpose_csr(m, d, row_ptr_host, col_host, val_host, &at);
  appga::pad_rows(m, d, row_ptr_host, col_host, val_host, appga::ROW_PAD, &pa);
  appga::pad_rows(d, m, at.row_ptr.data(), at.col.data(), at.val.data(), appga::ROW_PAD, &pt);
  // Lambda_j = (A^T 1)_j if positive, else 1 (Eq. EM); summed in FP64, once
  // for the FP32 values and once for their BF16 rounding (the BF16 run is the
  // method applied to the rounded matrix, preconditioner included)
  const bool want_bf16 = (flags & APPGA_A_BF16_COPY) != 0;
  std::vector<float> inv(d), inv_b(want_bf16 ? d : 0);
  for (int32_t j = 0; j < d; ++j) {
    double sum = 0.0, sum_b = 0.0;
    for (int32_t p = at.row_ptr[j]; p < at.row_ptr[j + 1]; ++p) {
      sum += (double)at.val[p];
      if (want_bf16) {
        const uint32_t bits = (uint32_t)appga::float_to_bf16(at.val[p]) << 16;
        float vb;
        std::memcpy(&vb, &bits, 4);
        sum_b += (double)vb;
      }
    }
    inv[j] = (float)(1.0 / (sum > 0.0 ? sum : 1.0));
    if (want_bf16) inv_b[j] = (float)(1.0 / (sum_b > 0.0 ? sum_b : 1.0));
  }
  auto* M = new appga_matrix();
  M->ctx = ctx;
  M->m = m;
  M->d = d;
  M->n = n_side;
  M->na = n_angles;
  M->nnz = nnz;
  M->has_bf16 = (flags & APPGA_A_BF16_COPY) ? 1 : 0;
  M->npfov = appga::disk_pixels(n_side);
  rc = upload_csr(pa, M->has_bf16, &M->A, &M->bytes);
  if (rc == APPGA_OK) rc = upload_csr(pt, M->has_bf16, &M->At, &M->bytes);
  if (rc == APPGA_OK) {
    // A's column indices in the 8 x 8-tiled pixel order (row_ptr and values shared)
    std::vector<int32_t> ct(pa.col.size());
    for (size_t q = 0; q < ct.size(); ++q)
      ct[q] = appga::tiled_index(pa.col[q] / n_side, pa.col[q] % n_side, n_side);
    M->A_tiled = M->A;
    M->A_tiled.col = nullptr;
    cudaError_t e = dalloc(&M->A_tiled.col, ct.size(), &M->bytes);
    if (e == cudaSuccess && !ct.empty())
      e = cudaMemcpy(M->A_tiled.col, ct.data(), ct.size() * 4, cudaMemcpyHostToDevice);
    // the solver loop's two projections in the sliced layout (both or neither)
    if (APPGA_PACK && e == cudaSuccess && !ct.empty() && !pt.col.empty()) {
      appga::HostSell ha, ht;
      if (appga::build_sell(m, pa.row_ptr, ct, pa.val, &ha) &&
          appga::build_sell(d, pt.row_ptr, pt.col, pt.val, &ht)) {
        appga_status r1 = upload_sell(ha, want_bf16, &M->sell_a, &M->bytes);
        if (r1 == APPGA_OK) r1 = upload_sell(ht, want_bf16, &M->sell_t, &M->bytes);
        if (r1 != APPGA_OK) e = cudaErrorMemoryAllocation;
      }
    }
    // the folded loop: A's first half (its rows are a prefix of pa) and the
    // transpose of that half in orbit order
    if (M->sell_a.off != nullptr && e == cudaSuccess && (flags & APPGA_A_NO_FOLD) == 0 &&
        appga::quarter_turn_symmetric(m, n_side, n_angles, row_ptr_host, col_host, val_host)) {
      appga::HostCSR ft, pft;
      appga::fold_transpose(at, m / 2, n_side, &ft);
      appga::pad_rows(d, m / 2, ft.row_ptr.data(), ft.col.data(), ft.val.data(), appga::ROW_PAD,
                      &pft);
      appga::HostSell fa, fb;
      if (!pft.col.empty() && appga::build_sell(m / 2, pa.row_ptr, ct, pa.val, &fa) &&
          appga::build_sell(d, pft.row_ptr, pft.col, pft.val, &fb)) {
        appga_status r1 = upload_sell(fa, want_bf16, &M->fold_a, &M->bytes);
        if (r1 == APPGA_OK) r1 = upload_sell(fb, want_bf16, &M->fold_t, &M->bytes);
        if (r1 != APPGA_OK) {
          free_sell(M->fold_a);
          free_sell(M->fold_t);
          e = cudaErrorMemoryAllocation;
        }
        M->fold_nb = m / n_angles;
      }
    }
    if (e != cudaSuccess) rc = cuda_fail(e, "tiled column indices and sliced layout");
  }
  if (rc == APPGA_OK) {
    cudaError_t e = dalloc(&M->inv_lambda, (size_t)d, &M->bytes);
    if (e == cudaSuccess)
      e = cudaMemcpy(M->inv_lambda, inv.data(), (size_t)d * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && want_bf16) e = dalloc(&M->inv_lambda_bf16, (size_t)d, &M->bytes);
    if (e == cudaSuccess && want_bf16)
      e = cudaMemcpy(M->inv_lambda_bf16, inv_b.data(), (size_t)d * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) rc = cuda_fail(e, "inv_lambda");
  }
  if (rc != APPGA_OK) {
    appga_matrix_destroy(M);
    return rc;
  }
  *out = M;
  return APPGA_OK;
}

appga_status appga_matrix_destroy(appga_matrix* M) {
  if (!M) return APPGA_OK;
  if (M->ctx) cudaSetDevice(M->ctx->device);
  cudaFree(M->A_tiled.col);  // its other arrays belong to A
  free_sell(M->sell_a);
  free_sell(M->sell_t);
  free_sell(M->fold_a);
  free_sell(M->fold_t);
  free_csr(M->A);
  free_csr(M->At);
  cudaFree(M->inv_lambda);
  cudaFree(M->inv_lambda_bf16);
  free_workspace(M->ws);
  if (M->aw) {
    appga::free_afppa_workspace(M->aw);
    delete M->aw;
  }
  if (M->bw) {
    appga::free_batch_workspace(M->bw);
    delete M->bw;
  }
  delete M;
  return APPGA_OK;
}

appga_status appga_matrix_get_info(const appga_matrix* M, appga_matrix_info* out) {
  if (!M || !out) return fail(APPGA_EINVAL, "null matrix or out");
  out->m = M->m;
  out->d = M->d;
  out->n_side = M->n;
  out->n_angles = M->na;
  out->nnz = M->nnz;
  out->nnz_padded_a = M->A.nnz_padded;
  out->nnz_padded_t = M->At.nnz_padded;
  out->has_bf16 = M->has_bf16;
  out->device_bytes = M->bytes;
  out->packed_columns = M->sell_t.cols != nullptr ? 1 : 0;
  out->sliced_layout = (M->sell_t.cols != nullptr || M->sell_t.cols32 != nullptr) ? 1 : 0;
  out->quarter_turn_folded = M->fold_t.off != nullptr ? 1 : 0;
  return APPGA_OK;
}

appga_status appga_forward_ratio(appga_ctx* ctx, const appga_matrix* mat, const float* f,
                                 const float* g, const float* gamma, double* y_out, float* w_out,
                                 double* data_out, void* stream) {
  if (!ctx || !mat || !f || !g || !gamma || !y_out)
    return fail(APPGA_EINVAL, "null argument");
  auto* M = const_cast<appga_matrix*>(mat);
  appga_status rc = ensure_workspace(M);
  if (rc != APPGA_OK) return rc;
  CK(cudaSetDevice(ctx->device));
  appga::FwdArgs a = fwd_args(M, false);
  a.f[0] = f;
  a.y[0] = nullptr;
  a.y_out = y_out;
  a.w = w_out;
  a.g = g;
  a.gamma = gamma;
  a.st = M->ws.st_scratch;
  a.partial = M->ws.partial_aux;
  a.gtick = M->ws.gtick;
  a.data_out = data_out;
  a.loop = 0;
  a.want_data = data_out != nullptr ? 1 : 0;
  a.n = M->n;
  CK(appga::launch_forward(a, (cudaStream_t)stream));
  return APPGA_OK;
}

appga_status appga_backproject(appga_ctx* ctx, const appga_matrix* mat, const float* w,
                               float* out, void* stream) {
  if (!ctx || !mat || !w || !out) return fail(APPGA_EINVAL, "null argument");
  auto* M = const_cast<appga_matrix*>(mat);
  appga_status rc = ensure_workspace(M);
  if (rc != APPGA_OK) return rc;
  CK(cudaSetDevice(ctx->device));
  CK(appga::launch_backproject(mat->At, w, out, 0, (cudaStream_t)stream));
  return APPGA_OK;
}

appga_status appga_shoitv_grad(appga_ctx* ctx, int32_t n_side, const float* f, double lambda1,
                               double lambda2, double eps, float* out, void* stream) {
  if (!ctx || !f || !out) return fail(APPGA_EINVAL, "null argument");
  if (n_side <= 0) return fail(APPGA_EINVAL, "n_side must be > 0");
  if (!(lambda1 >= 0) || !(lambda2 >= 0) || !(eps > 0))
    return fail(APPGA_EINVAL, "need lambda1, lambda2 >= 0 and eps > 0");
  CK(cudaSetDevice(ctx->device));
  CK(appga::launch_stencil(n_side, f, f, 0.f, (float)lambda1, (float)lambda2, (float)eps, out,
                           (cudaStream_t)stream));
  return APPGA_OK;
}

appga_status appga_pixel_update(appga_ctx* ctx, const appga_matrix* mat, const float* f_prev,
                                const float* f_cur, const float* w, double theta,
                                const appga_params* params, float* f_next, void* stream) {
  if (!ctx || !mat || !f_prev || !f_cur || !w || !params || !f_next)
    return fail(APPGA_EINVAL, "null argument");
  appga_status rc = appga_params_validate(params);
  if (rc != APPGA_OK) return rc;
  auto* M = const_cast<appga_matrix*>(mat);
  if ((rc = ensure_workspace(M)) != APPGA_OK) return rc;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  SolverState h{};
  h.k = 1;
  h.k0 = 1;
  h.k_last = 1 << 30;
  h.theta = theta;
  h.theta_hi = (float)theta;
  h.theta_lo = (float)(theta - (double)h.theta_hi);
  h.t_cur = 1.0;
  CK(cudaMemcpyAsync(M->ws.st_scratch, &h, sizeof h, cudaMemcpyHostToDevice, s));
  // B^T grad phi~(B f~) of f~ = f_cur + theta (f_cur - f_prev)
  CK(appga::launch_stencil(M->n, f_cur, f_prev, (float)theta, (float)params->lambda1,
                           (float)params->lambda2, (float)params->eps, M->ws.gR, s));
  appga::PixArgs pa{};
  pa.At = M->At;
  pa.n = M->n;
  pa.f[0] = const_cast<float*>(f_prev);
  pa.f[1] = const_cast<float*>(f_cur);
  pa.f[2] = f_next;
  pa.w = w;
  pa.gR = M->ws.gR;
  pa.inv_lambda = bf16_requested(M, params) ? M->inv_lambda_bf16 : M->inv_lambda;
  pa.pfreeze = M->ws.pfreeze;
  pa.st = M->ws.st_scratch;
  pa.partial = M->ws.partial_aux;
  pa.gtick = M->ws.gtick;
  appga_params q = *params;
  q.precond_freeze_iter = -1;
  pa.ip = iter_params(&q, false);
  pa.use_bf16 = bf16_requested(M, params) ? 1 : 0;
  CK(appga::launch_pixel(pa, s));
  return APPGA_OK;
}

appga_status appga_objective(appga_ctx* ctx, const appga_matrix* mat, const float* f,
                             const float* g, const float* gamma, const appga_params* params,
                             double* phi_out_host, void* stream) {
  if (!ctx || !mat || !f || !g || !gamma || !params || !phi_out_host)
    return fail(APPGA_EINVAL, "null argument");
  appga_status rc = appga_params_validate(params);
  if (rc != APPGA_OK) return rc;
  auto* M = const_cast<appga_matrix*>(mat);
  if ((rc = ensure_workspace(M)) != APPGA_OK) return rc;
  CK(cudaSetDevice(ctx->device));
  return objective_on(M, f, g, gamma, params, phi_out_host, (cudaStream_t)stream);
}

appga_status appga_initial_image(appga_ctx* ctx, const appga_matrix* mat, const float* g,
                                 const float* gamma, float* f_out, void* stream) {
  if (!ctx || !mat || !g || !gamma || !f_out) return fail(APPGA_EINVAL, "null argument");
  auto* M = const_cast<appga_matrix*>(mat);
  appga_status rc = ensure_workspace(M);
  if (rc != APPGA_OK) return rc;
  CK(cudaSetDevice(ctx->device));
  CK(appga::launch_initial_image(g, gamma, M->m, M->n, M->na, M->npfov, M->ws.partial_aux, M->ws.gtick,
                                 M->ws.st_scratch, f_out, (cudaStream_t)stream));
  return APPGA_OK;
}

appga_status appga_reconstruct(appga_ctx* ctx, const appga_matrix* mat, const float* g,
                               const float* gamma, const float* f_init,
                               const appga_params* params, float* f_out,
                               appga_stats* stats_host, void* stream) {
  return solve_common(ctx, const_cast<appga_matrix*>(mat), g, gamma, nullptr, f_init, 1, params,
                      nullptr, f_out, stats_host, stream, true);
}

appga_status appga_resume(appga_ctx* ctx, const appga_matrix* mat, const float* g,
                          const float* gamma, const float* f_prev, const float* f_cur,
                          int32_t k0, const appga_params* params, float* f_out_prev,
                          float* f_out, appga_stats* stats_host, void* stream) {
  return solve_common(ctx, const_cast<appga_matrix*>(mat), g, gamma, f_prev, f_cur, k0, params,
                      f_out_prev, f_out, stats_host, stream, false);
}

appga_status appga_validate_csr_host(int32_t m, int32_t d, const int32_t* row_ptr_host,
                                     const int32_t* col_host, const float* val_host) {
  std::string why;
  appga_status rc = appga::validate_csr(m, d, row_ptr_host, col_host, val_host, &why);
  if (rc != APPGA_OK) return fail(rc, why);
  return APPGA_OK;
}

appga_status appga_kernel_times(appga_ctx* ctx, const appga_matrix* mat, const float* g,
                                const float* gamma, const appga_params* params, int32_t n_iters,
                                double* ms_pixel_host, double* ms_forward_host) {
  if (!ms_pixel_host || !ms_forward_host) return fail(APPGA_EINVAL, "null output");
  if (n_iters < 1 || n_iters > 4096) return fail(APPGA_EINVAL, "n_iters must be in [1, 4096]");
  auto* M = const_cast<appga_matrix*>(mat);
  appga_status rc = check_params_and_mat(ctx, M, params);
  if (rc != APPGA_OK) return rc;
  if (!g || !gamma) return fail(APPGA_EINVAL, "null argument");
  if ((rc = ensure_workspace(M)) != APPGA_OK) return rc;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  Workspace& ws = M->ws;
  appga_params q = *params;
  q.max_iters = n_iters;
  q.rel_obj_tol = 0.0;
  const SolverState h = start_state(1, &q);
  if ((rc = momentum_table(M, ws.st, 1, &q, s, &h)) != APPGA_OK) return rc;
  CK(appga::launch_initial_image(g, gamma, M->m, M->n, M->na, M->npfov, ws.partial_aux, ws.gtick,
                                 ws.st_scratch, ws.f[1], s, ws.f[0]));
  appga::FwdArgs fa;
  appga::PixArgs pa;
  if ((rc = setup_run(M, g, gamma, 1, &q, true, false, &fa, &pa)) != APPGA_OK) return rc;
  const bool track = q.track_objective != 0;
  std::vector<cudaEvent_t> ev((size_t)2 * n_iters + 1);
  for (auto& e : ev) CK(cudaEventCreate(&e));
  cudaError_t e = cudaEventRecord(ev[0], s);
  for (int i = 0; i < n_iters && e == cudaSuccess; ++i) {
    e = appga::launch_pixel(pa, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2 * i + 1], s);
    if (e == cudaSuccess) e = appga::launch_forward(fa, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2 * i + 2], s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  double tp = 0.0, tf = 0.0;
  for (int i = 0; i < n_iters && e == cudaSuccess; ++i) {
    float a = 0.f, b = 0.f;
    e = cudaEventElapsedTime(&a, ev[2 * i], ev[2 * i + 1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[2 * i + 1], ev[2 * i + 2]);
    tp += a;
    tf += b;
  }
  for (auto& x : ev) cudaEventDestroy(x);
  if (e != cudaSuccess) return cuda_fail(e, "kernel timing");
  *ms_pixel_host = tp / n_iters;
  *ms_forward_host = tf / n_iters;
  return APPGA_OK;
}

appga_status appga_reconstruct_host(appga_ctx* ctx, const appga_matrix* mat, const float* g_host,
                                    const float* gamma_host, const float* f_init_host,
                                    const appga_params* params, float* f_out_host,
                                    appga_stats* stats_host, void* stream) {
  if (!ctx || !mat || !g_host || !gamma_host || !params || !f_out_host)
    return fail(APPGA_EINVAL, "null argument");
  auto* M = const_cast<appga_matrix*>(mat);
  appga_status rc = ensure_workspace(M);
  if (rc != APPGA_OK) return rc;
  CK(cudaSetDevice(ctx->device));
  Workspace& ws = M->ws;
  int64_t* b = &M->bytes;
  if (ws.d_g == nullptr) {
    cudaError_t e = dalloc(&ws.d_g, (size_t)M->m, b);
    if (e == cudaSuccess) e = dalloc(&ws.d_gamma, (size_t)M->m, b);
    if (e == cudaSuccess) e = dalloc(&ws.d_finit, (size_t)M->d, b);
    if (e == cudaSuccess) e = dalloc(&ws.d_fout, (size_t)M->d, b);
    if (e != cudaSuccess) return cuda_fail(e, "host-path staging buffers");
  }
  cudaStream_t us = (cudaStream_t)stream;
  const size_t mb = (size_t)M->m * 4, db = (size_t)M->d * 4;
  CK(cudaMemcpyAsync(ws.d_g, g_host, mb, cudaMemcpyHostToDevice, us));
  CK(cudaMemcpyAsync(ws.d_gamma, gamma_host, mb, cudaMemcpyHostToDevice, us));
  if (f_init_host) CK(cudaMemcpyAsync(ws.d_finit, f_init_host, db, cudaMemcpyHostToDevice, us));
  // the result comes back to f_out_host inside the solver call, before its
  // one synchronisation
  return solve_common(ctx, M, ws.d_g, ws.d_gamma, nullptr, f_init_host ? ws.d_finit : nullptr, 1,
                      params, nullptr, ws.d_fout, stats_host, stream, true, f_out_host);
}

}  // extern "C"
