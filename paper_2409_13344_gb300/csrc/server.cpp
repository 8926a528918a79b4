// Continuous-batching reconstruction server (appga_server.h): pools of
// batched solvers per geometry, admission at step boundaries by free device
// memory, retirement of finished slots, per-request latency.
//
// Every pool has its own stream, so the replays of different pools (and of
// different geometries) overlap on the device.  A scheduling round never
// waits for a pool that is still running: a pool's replay ends with a copy
// of its slot states to pinned memory and an event; the round handles the
// pools whose event has completed (retires their finished slots, admits
// waiting requests into them, starts their next replay) and leaves the
// others running.  Retirement copies results out asynchronously and
// completes in a later round, once that copy has landed.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <limits>
#include <memory>
#include <unordered_map>
#include <vector>

#include "appga.h"
#include "appga_internal.h"
#include "appga_server.h"
#include "batched_internal.h"
#include "handles.h"

namespace appga {
namespace {

using Clock = std::chrono::steady_clock;
constexpr double kNaN = std::numeric_limits<double>::quiet_NaN();

struct Request {
  int64_t id = 0;
  int geom = 0;
  appga_params p{};
  std::vector<float> g, gamma, finit;  // host copies until admission
  std::vector<float> f;                // result once retired
  appga_request_stats st{};
  int pool = -1, slot = -1;
};

// One batched solver of one geometry: width-Kp workspace, its captured
// graph, and staging for admission and retirement.
struct Pool {
  int geom = 0;
  BatchWorkspace b;
  BFwdArgs fa{};
  BPixArgs pa{};
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t stream = nullptr;  // all of this pool's work
  cudaEvent_t ev_snap = nullptr;  // the slot-state copy after a replay has landed
  cudaEvent_t ev_start = nullptr; // start of the replay (timing)
  cudaEvent_t ev_out = nullptr;   // the retired images have landed in h_out
  bool inflight = false;          // a replay (and its slot-state copy) is running
  bool retiring = false;          // retired images on their way to h_out
  std::vector<int64_t> ret_ids;   // requests of the images on their way
  std::vector<SlotState> ret_fin; // their final slot states
  int ret_flags = 0;
  std::vector<int64_t> slot_req;  // request id per slot, -1 = free
  int used = 0;
  int gstep = 0;  // global step of the pool, as last read back
  int64_t bytes = 0;
  float* d_in = nullptr;  // [Kp][2m + d]: g, gamma, f_init of admitted slices
  float* h_in = nullptr;  // pinned mirror
  float* d_out = nullptr; // [Kp][d]: retired images
  float* h_out = nullptr; // pinned mirror
  int* d_ids = nullptr;   // [3 Kp]: admitted slots | slots with f_init | retired slots
  int* h_ids = nullptr;   // pinned mirror

  int free_slots() const { return (int)slot_req.size() - used; }
  bool idle() const { return !inflight; }
};

struct Geometry {
  const appga_matrix* M = nullptr;
  std::deque<int64_t> waiting;
};

int64_t pool_bytes(const appga_matrix* M, int Kp) {
  return batch_workspace_bytes(M->m, M->d, Kp) +
         (int64_t)Kp * (2LL * M->m + 2LL * M->d) * (int64_t)sizeof(float) +
         3LL * Kp * (int64_t)sizeof(int);
}

void free_pool(Pool* P) {
  if (!P) return;
  if (P->stream) cudaStreamSynchronize(P->stream);
  if (P->gexec) cudaGraphExecDestroy(P->gexec);
  if (P->ev_snap) cudaEventDestroy(P->ev_snap);
  if (P->ev_start) cudaEventDestroy(P->ev_start);
  if (P->ev_out) cudaEventDestroy(P->ev_out);
  if (P->stream) cudaStreamDestroy(P->stream);
  P->stream = nullptr;
  P->ev_snap = P->ev_out = P->ev_start = nullptr;
  free_batch_workspace(&P->b);
  cudaFree(P->d_in);
  cudaFree(P->d_out);
  cudaFree(P->d_ids);
  cudaFreeHost(P->h_in);
  cudaFreeHost(P->h_out);
  cudaFreeHost(P->h_ids);
  P->gexec = nullptr;
  P->d_in = P->d_out = nullptr;
  P->h_in = P->h_out = nullptr;
  P->d_ids = P->h_ids = nullptr;
}

bool finite_ge(const float* x, size_t n, float lo, bool strict) {
  for (size_t i = 0; i < n; ++i) {
    const float v = x[i];
    if (!std::isfinite(v) || v < lo || (strict && v <= lo)) return false;
  }
  return true;
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return kNaN;
  std::sort(v.begin(), v.end());
  // nearest rank: the smallest value with at least q of the samples at or below it
  size_t r = (size_t)std::ceil(q * (double)v.size());
  if (r < 1) r = 1;
  return v[r - 1];
}

}  // namespace
}  // namespace appga

using namespace appga;

struct appga_server {
  appga_ctx* ctx = nullptr;
  appga_server_config cfg{};
  std::vector<Geometry> geoms;
  std::vector<std::unique_ptr<Pool>> pools;
  std::unordered_map<int64_t, Request> reqs;
  int64_t next_id = 1;
  int64_t bytes = 0;
  int64_t submitted = 0, completed = 0, slice_iters = 0, waiting = 0, running = 0;
  int64_t pool_slot_steps = 0, live_slot_steps = 0;
  double replay_seconds = 0.0;
  std::vector<double> latencies, queue_waits;
  Clock::time_point t0;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

#define CK(call) APPGA_CK(call)

appga_status create_pool(appga_server* S, int geom, int Kp, Pool** out) {
  *out = nullptr;
  const appga_matrix* M = S->geoms[geom].M;
  auto P = std::make_unique<Pool>();
  P->geom = geom;
  P->bytes = pool_bytes(M, Kp);
  cudaError_t e = alloc_batch_workspace(P->b, M->m, M->d, Kp);
  if (e != cudaSuccess) return cuda_fail(e, "server pool workspace");
  const size_t in_len = (size_t)Kp * (2 * (size_t)M->m + M->d);
  const size_t out_len = (size_t)Kp * M->d;
  e = cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&P->ev_snap);
  if (e == cudaSuccess) e = cudaEventCreate(&P->ev_start);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = dalloc(&P->d_in, in_len);
  if (e == cudaSuccess) e = dalloc(&P->d_out, out_len);
  if (e == cudaSuccess) e = dalloc(&P->d_ids, (size_t)3 * Kp);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&P->h_in, in_len * sizeof(float));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&P->h_out, out_len * sizeof(float));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&P->h_ids, (size_t)3 * Kp * sizeof(int));
  if (e != cudaSuccess) {
    free_pool(P.get());
    return cuda_fail(e, "server pool staging");
  }
  const bool bf16 = S->cfg.a_precision == APPGA_PREC_BF16;
  make_batch_args(M->A, M->At, bf16 ? M->inv_lambda_bf16 : M->inv_lambda, M->n, P->b, bf16,
                  true, tuned_schedule(M, Kp, bf16), &P->fa, &P->pa);
  cudaStream_t s = P->stream;
  // every slot starts empty; the ring starts at step 1
  appga_params def;
  appga_params_default(&def);
  for (int i = 0; i < Kp; ++i) P->b.slots_host[i] = slot_from_params(&def, 1, false);
  BatchState hb{};
  hb.gstep = 1;
  *P->b.bst_host = hb;
  P->gstep = 1;
  e = cudaMemcpyAsync(P->b.slots, P->b.slots_host, Kp * sizeof(SlotState),
                      cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(P->b.bst, P->b.bst_host, sizeof(BatchState), cudaMemcpyHostToDevice, s);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i)
    e = cudaMemsetAsync(P->b.f[i], 0, (size_t)M->d * Kp * sizeof(float), s);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i)
    e = cudaMemsetAsync(P->b.y[i], 0, (size_t)M->m * Kp * sizeof(float), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->b.g, 0, (size_t)M->m * Kp * sizeof(float), s);
  if (e == cudaSuccess) e = launch_fill_slots(P->b.gamma, M->m, Kp, 0, Kp, 1.f, s);
  if (e == cudaSuccess) e = capture_batch_graph(P->fa, P->pa, S->cfg.steps_per_launch, s, &P->gexec);
  if (e != cudaSuccess) {
    free_pool(P.get());
    return cuda_fail(e, "server pool setup");
  }
  P->slot_req.assign(Kp, -1);
  S->bytes += P->bytes;
  // reuse a released entry so pool indices stay small
  for (auto& q : S->pools) {
    if (!q) {
      q = std::move(P);
      *out = q.get();
      return APPGA_OK;
    }
  }
  S->pools.push_back(std::move(P));
  *out = S->pools.back().get();
  return APPGA_OK;
}

int pool_index(const appga_server* S, const Pool* P) {
  for (size_t i = 0; i < S->pools.size(); ++i)
    if (S->pools[i].get() == P) return (int)i;
  return -1;
}

int live_pools(const appga_server* S) {
  int c = 0;
  for (auto& q : S->pools) c += q != nullptr;
  return c;
}

// Width of a new pool of geometry `geom`: the configured one, or (adaptive,
// slots_per_pool 0) the narrowest of 32, 64, 128 slots that holds the
// geometry's demand (its waiting requests plus those running in its pools):
// narrow pools step faster when few requests are in flight, wide pools read
// the matrix once for more slices under load.
int new_pool_width(const appga_server* S, int geom) {
  if (S->cfg.slots_per_pool > 0) return S->cfg.slots_per_pool;
  size_t demand = S->geoms[geom].waiting.size();
  for (const auto& q : S->pools)
    if (q && q->geom == geom) demand += (size_t)q->used;
  return demand <= 32 ? 32 : (demand <= 64 ? 64 : 128);
}

// Whether a new pool of geometry `geom` and width Kp fits the pool cap and
// device memory.
bool pool_fits(appga_server* S, int geom, int Kp) {
  if (S->cfg.max_pools > 0 && live_pools(S) >= S->cfg.max_pools) return false;
  if (S->cfg.max_pools_per_geometry > 0) {
    int mine = 0;
    for (const auto& q : S->pools) mine += (q && q->geom == geom) ? 1 : 0;
    if (mine >= S->cfg.max_pools_per_geometry) return false;
  }
  const int64_t need = pool_bytes(S->geoms[geom].M, Kp);
  if (S->cfg.hbm_budget_bytes > 0 && S->bytes + need > S->cfg.hbm_budget_bytes) return false;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return false;
  return (int64_t)free_b - S->cfg.hbm_reserve_bytes >= need;
}

// Releases every pool that holds no request (other than `keep_geom`'s) and
// has no work in flight (a replay, or retired images on their way out).
bool release_empty_pools(appga_server* S, int keep_geom) {
  bool any = false;
  for (auto& q : S->pools) {
    if (q && q->used == 0 && q->geom != keep_geom && !q->inflight && !q->retiring) {
      S->bytes -= q->bytes;
      free_pool(q.get());
      q.reset();
      any = true;
    }
  }
  return any;
}

// Admits up to `count` waiting requests of the pool's geometry into its free
// slots and runs their first forward phase (mode 2 of the forward kernel).
// The pool is idle: its last replay's slot states have landed, so P->gstep
// is its ring position and its staging buffers are free.
appga_status admit(appga_server* S, Pool* P, int count) {
  Geometry& G = S->geoms[P->geom];
  const appga_matrix* M = G.M;
  const int Kp = P->b.Kp, m = M->m, d = M->d;
  cudaStream_t s = P->stream;
  std::vector<int64_t> ids;
  ids.reserve(count);
  int slot = 0;
  for (int k = 0; k < count && !G.waiting.empty(); ++k) {
    while (P->slot_req[slot] != -1) ++slot;
    const int64_t id = G.waiting.front();
    G.waiting.pop_front();
    ids.push_back(id);
    P->slot_req[slot] = id;
    P->h_ids[k] = slot;
    Request& R = S->reqs[id];
    R.pool = pool_index(S, P);
    R.slot = slot;
  }
  const int K = (int)ids.size();
  if (K == 0) return APPGA_OK;
  // pack g | gamma | f_init (the slices that bring one) into the pinned staging
  int kf = 0;
  for (int k = 0; k < K; ++k) {
    Request& R = S->reqs[ids[k]];
    std::memcpy(P->h_in + (size_t)k * m, R.g.data(), (size_t)m * sizeof(float));
    std::memcpy(P->h_in + (size_t)(K + k) * m, R.gamma.data(), (size_t)m * sizeof(float));
    if (!R.finit.empty()) {
      std::memcpy(P->h_in + (size_t)2 * K * m + (size_t)kf * d, R.finit.data(),
                  (size_t)d * sizeof(float));
      P->h_ids[Kp + kf] = P->h_ids[k];
      ++kf;
    }
  }
  const int Gs = P->gstep;
  float* cur = P->b.f[Gs % 3];
  CK(cudaMemcpyAsync(P->d_in, P->h_in, ((size_t)2 * K * m + (size_t)kf * d) * sizeof(float),
                     cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(P->d_ids, P->h_ids, (size_t)2 * Kp * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(launch_to_slot_minor(P->d_in, K, m, P->b.g, Kp, 0, P->d_ids, s));
  CK(launch_to_slot_minor(P->d_in + (size_t)K * m, K, m, P->b.gamma, Kp, 0, P->d_ids, s));
  // f^{k0} = f^{k0-1}: the initial image TMC * 1_disk (Sec. 4.1), or the request's own
  CK(launch_binit_image(P->d_in, P->d_in + (size_t)K * m, m, M->n, M->na, M->npfov, K, Kp, 0,
                        P->d_ids, cur, s));
  CK(launch_to_slot_minor(P->d_in + (size_t)2 * K * m, kf, d, cur, Kp, 0, P->d_ids + Kp, s));
  CK(launch_copy_slots(cur, P->b.f[(Gs + 2) % 3], d, Kp, P->d_ids, K, s));
  for (int k = 0; k < K; ++k) {
    Request& R = S->reqs[ids[k]];
    SlotState st = slot_from_params(&R.p, 1, true);
    st.fresh = 1;
    P->b.slots_host[R.slot] = st;
    CK(cudaMemcpyAsync(P->b.slots + R.slot, P->b.slots_host + R.slot, sizeof(SlotState),
                       cudaMemcpyHostToDevice, s));
  }
  CK(launch_binit_momentum(P->b.slots, Kp, true, s));
  BFwdArgs a = P->fa;
  a.mode = 2;
  CK(launch_bforward(a, s));
  // every held slot is live at a step boundary (finished ones were retired)
  P->b.bst_host->remaining = P->used + K;
  CK(cudaMemcpyAsync(&P->b.bst->remaining, &P->b.bst_host->remaining, sizeof(int),
                     cudaMemcpyHostToDevice, s));
  const double t = S->now();
  for (int64_t id : ids) {
    Request& R = S->reqs[id];
    R.st.state = APPGA_REQ_RUNNING;
    R.st.t_admit = t;
    std::vector<float>().swap(R.g);
    std::vector<float>().swap(R.gamma);
    std::vector<float>().swap(R.finit);
  }
  P->used += K;
  S->waiting -= K;
  S->running += K;
  return APPGA_OK;
}

appga_status admit_all(appga_server* S) {
  for (int gi = 0; gi < (int)S->geoms.size(); ++gi) {
    Geometry& G = S->geoms[gi];
    bool released = false;
    while (!G.waiting.empty()) {
      // the narrowest idle pool of this geometry with a free slot; a pool of
      // the geometry that is running takes the requests once its replay ends
      Pool* P = nullptr;
      bool busy = false;
      for (auto& q : S->pools) {
        if (!q || q->geom != gi || q->free_slots() == 0) continue;
        if (!q->idle()) {
          busy = true;
          continue;
        }
        if (!P || q->b.Kp < P->b.Kp) P = q.get();
      }
      if (!P && busy) break;
      if (!P) {
        const int width = new_pool_width(S, gi);
        if (!pool_fits(S, gi, width)) {
          if (released || !release_empty_pools(S, gi)) break;  // waits for memory
          released = true;
          if (!pool_fits(S, gi, width)) break;
        }
        appga_status rc = create_pool(S, gi, width, &P);
        if (rc != APPGA_OK) return rc;
      }
      appga_status rc = admit(S, P, P->free_slots());
      if (rc != APPGA_OK) return rc;
    }
  }
  return APPGA_OK;
}

// First half of a retirement, right after the pool's slot states have
// landed: the finished slots' images are gathered out and copied to pinned
// memory on the pool's stream, the slots are reset and freed (an admission
// enqueued after this may reuse them), and the copy's event is recorded.
appga_status retire_begin(appga_server* S, Pool* P) {
  const appga_matrix* M = S->geoms[P->geom].M;
  const int Kp = P->b.Kp, d = M->d;
  cudaStream_t s = P->stream;
  const BatchState& bs = *P->b.bst_host;
  P->gstep = bs.gstep;
  std::vector<int> slots;
  for (int i = 0; i < Kp; ++i) {
    const SlotState& sl = P->b.slots_host[i];
    if (P->slot_req[i] != -1 && sl.active && sl.done) slots.push_back(i);
  }
  const int K = (int)slots.size();
  if (K == 0) return APPGA_OK;
  // a slot stopped by the test in the last pixel phase has its result one
  // ring entry back: move it into the current entry first
  CK(launch_resolve_rollback(P->fa, s));
  for (int k = 0; k < K; ++k) P->h_ids[2 * Kp + k] = slots[k];
  CK(cudaMemcpyAsync(P->d_ids + 2 * Kp, P->h_ids + 2 * Kp, K * sizeof(int),
                     cudaMemcpyHostToDevice, s));
  // a finished slot carries its result forward, so it sits in the current ring entry
  CK(launch_from_slot_minor(P->b.f[P->gstep % 3], K, d, Kp, 0, P->d_ids + 2 * Kp, P->d_out, s));
  CK(cudaMemcpyAsync(P->h_out, P->d_out, (size_t)K * d * sizeof(float), cudaMemcpyDeviceToHost,
                     s));
  appga_params def;
  appga_params_default(&def);
  P->ret_ids.resize(K);
  P->ret_fin.resize(K);
  P->ret_flags = bs.flags;
  for (int k = 0; k < K; ++k) {
    P->ret_fin[k] = P->b.slots_host[slots[k]];
    P->ret_ids[k] = P->slot_req[slots[k]];
    P->b.slots_host[slots[k]] = slot_from_params(&def, 1, false);
    CK(cudaMemcpyAsync(P->b.slots + slots[k], P->b.slots_host + slots[k], sizeof(SlotState),
                       cudaMemcpyHostToDevice, s));
    P->slot_req[slots[k]] = -1;
  }
  CK(cudaEventRecord(P->ev_out, s));
  P->used -= K;
  P->retiring = true;
  return APPGA_OK;
}

// Second half, once the images have landed in h_out: results and statistics
// of the retired requests.
void retire_finish(appga_server* S, Pool* P) {
  const int d = S->geoms[P->geom].M->d;
  const double t = S->now();
  const int K = (int)P->ret_ids.size();
  for (int k = 0; k < K; ++k) {
    const SlotState& sl = P->ret_fin[k];
    Request& R = S->reqs[P->ret_ids[k]];
    R.f.assign(P->h_out + (size_t)k * d, P->h_out + (size_t)(k + 1) * d);
    R.st.state = APPGA_REQ_DONE;
    R.st.iters = sl.result_k - sl.k0;
    R.st.result_k = sl.result_k;
    R.st.stopped_early = sl.stopped_early;
    R.st.flags = P->ret_flags;
    R.st.phi_k = sl.phi_k;
    R.st.phi_last = sl.phi_k >= 0 ? sl.phi_cur : kNaN;
    R.st.guard_hits = (int64_t)sl.guard_hits;
    R.st.t_done = t;
    R.pool = -1;
    R.slot = -1;
    S->latencies.push_back(t - R.st.t_submit);
    S->queue_waits.push_back(R.st.t_admit - R.st.t_submit);
    S->slice_iters += R.st.iters;
  }
  S->running -= K;
  S->completed += K;
  P->ret_ids.clear();
  P->ret_fin.clear();
  P->retiring = false;
}

// Handles the pools whose work has landed; true if any had.
appga_status progress(appga_server* S, bool* any) {
  *any = false;
  for (auto& q : S->pools) {
    if (!q) continue;
    if (q->retiring) {
      const cudaError_t e = cudaEventQuery(q->ev_out);
      if (e == cudaSuccess) {
        retire_finish(S, q.get());
        *any = true;
      } else if (e != cudaErrorNotReady) {
        return cuda_fail(e, "server retirement");
      }
    }
    if (q->inflight && !q->retiring) {
      const cudaError_t e = cudaEventQuery(q->ev_snap);
      if (e == cudaSuccess) {
        q->inflight = false;
        *any = true;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, q->ev_start, q->ev_snap) == cudaSuccess)
          S->replay_seconds += 1e-3 * ms;
        appga_status rc = retire_begin(S, q.get());
        if (rc != APPGA_OK) return rc;
      } else if (e != cudaErrorNotReady) {
        return cuda_fail(e, "server replay");
      }
    }
  }
  return APPGA_OK;
}

}  // namespace

extern "C" void appga_server_config_default(appga_server_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof *cfg);
  cfg->slots_per_pool = 64;
  cfg->steps_per_launch = 8;
  cfg->a_precision = APPGA_PREC_FP32;
  cfg->max_pools = 0;
  cfg->hbm_budget_bytes = 0;
  cfg->hbm_reserve_bytes = 1LL << 30;
  cfg->max_pools_per_geometry = 2;
}

extern "C" appga_status appga_server_create(appga_ctx* ctx, const appga_server_config* cfg,
                                            appga_server** out) {
  if (!ctx || !cfg || !out) return fail(APPGA_EINVAL, "null argument");
  *out = nullptr;
  const int kp = cfg->slots_per_pool;  // 0: adaptive widths
  if (kp != 0 && kp != 32 && kp != 64 && kp != 128)
    return fail(APPGA_EINVAL, "slots_per_pool must be 0 (adaptive), 32, 64 or 128");
  if (cfg->steps_per_launch < 1) return fail(APPGA_EINVAL, "steps_per_launch must be >= 1");
  if (cfg->a_precision != APPGA_PREC_FP32 && cfg->a_precision != APPGA_PREC_BF16)
    return fail(APPGA_EINVAL, "a_precision must be APPGA_PREC_FP32 or APPGA_PREC_BF16");
  if (cfg->max_pools < 0 || cfg->hbm_budget_bytes < 0 || cfg->hbm_reserve_bytes < 0 ||
      cfg->max_pools_per_geometry < 0)
    return fail(APPGA_EINVAL, "negative pool cap or memory size");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(APPGA_ENODEV, "cudaSetDevice failed");
  auto* S = new appga_server();
  S->ctx = ctx;
  S->cfg = *cfg;
  S->t0 = Clock::now();
  *out = S;
  return APPGA_OK;
}

extern "C" appga_status appga_server_destroy(appga_server* S) {
  if (!S) return APPGA_OK;
  cudaStreamSynchronize(S->ctx->stream);
  for (auto& q : S->pools)
    if (q) free_pool(q.get());
  delete S;
  return APPGA_OK;
}

extern "C" appga_status appga_server_add_geometry(appga_server* S, const appga_matrix* mat,
                                                  int32_t* geometry_out) {
  if (!S || !mat || !geometry_out) return fail(APPGA_EINVAL, "null argument");
  if (mat->ctx != S->ctx) return fail(APPGA_EINVAL, "matrix belongs to another context");
  if (S->cfg.a_precision == APPGA_PREC_BF16 && !mat->has_bf16)
    return fail(APPGA_EINVAL, "BF16 pools need a matrix created with APPGA_A_BF16_COPY");
  // the widest pool the server may create for this geometry
  const int widest = S->cfg.slots_per_pool > 0 ? S->cfg.slots_per_pool : 128;
  const appga_status rc = check_slot_width(mat, widest);
  if (rc != APPGA_OK) return rc;
  Geometry G;
  G.M = mat;
  S->geoms.push_back(G);
  *geometry_out = (int32_t)S->geoms.size() - 1;
  return APPGA_OK;
}

extern "C" appga_status appga_server_submit(appga_server* S, int32_t geometry,
                                            const float* g_host, const float* gamma_host,
                                            const float* f_init_host, const appga_params* params,
                                            int64_t* request_out) {
  if (!S || !g_host || !gamma_host || !params || !request_out)
    return fail(APPGA_EINVAL, "null argument");
  if (geometry < 0 || geometry >= (int32_t)S->geoms.size())
    return fail(APPGA_EINVAL, "unknown geometry id");
  appga_status rc = appga_params_validate(params);
  if (rc != APPGA_OK) return rc;
  const appga_matrix* M = S->geoms[geometry].M;
  if (!finite_ge(g_host, M->m, 0.f, false) || !finite_ge(gamma_host, M->m, 0.f, true) ||
      (f_init_host && !finite_ge(f_init_host, M->d, 0.f, false)))
    return fail(APPGA_EDOMAIN,
                "inputs must satisfy: g finite and >= 0, gamma finite and > 0, f finite and >= 0");
  Request R;
  R.id = S->next_id++;
  R.geom = geometry;
  R.p = *params;
  R.p.a_precision = S->cfg.a_precision;
  R.p.track_objective = 1;
  R.p.graph_iters = S->cfg.steps_per_launch;
  R.g.assign(g_host, g_host + M->m);
  R.gamma.assign(gamma_host, gamma_host + M->m);
  if (f_init_host) R.finit.assign(f_init_host, f_init_host + M->d);
  R.st.state = APPGA_REQ_WAITING;
  R.st.phi_k = -1;
  R.st.phi_last = kNaN;
  R.st.t_submit = S->now();
  R.st.t_admit = kNaN;
  R.st.t_done = kNaN;
  const int64_t id = R.id;
  S->reqs.emplace(id, std::move(R));
  S->geoms[geometry].waiting.push_back(id);
  ++S->submitted;
  ++S->waiting;
  *request_out = id;
  return APPGA_OK;
}

extern "C" appga_status appga_server_step(appga_server* S, int32_t* pending_out) {
  if (!S) return fail(APPGA_EINVAL, "null argument");
  if (cudaSetDevice(S->ctx->device) != cudaSuccess) return fail(APPGA_ENODEV, "cudaSetDevice failed");
  // retirements and replays that have landed
  bool any = false;
  appga_status rc = progress(S, &any);
  if (rc != APPGA_OK) return rc;
  // waiting requests into idle pools (or new pools)
  if ((rc = admit_all(S)) != APPGA_OK) return rc;
  // the next replay of every idle pool that holds requests, each on its own
  // stream, ending with a copy of its slot states and an event
  bool running = false, launched = false;
  for (auto& q : S->pools) {
    if (!q) continue;
    if (q->idle() && q->used > 0) {
      launched = true;
      S->pool_slot_steps += (int64_t)q->b.Kp * S->cfg.steps_per_launch;
      S->live_slot_steps += (int64_t)q->used * S->cfg.steps_per_launch;
      CK(cudaEventRecord(q->ev_start, q->stream));
      CK(cudaGraphLaunch(q->gexec, q->stream));
      CK(cudaMemcpyAsync(q->b.slots_host, q->b.slots, q->b.Kp * sizeof(SlotState),
                         cudaMemcpyDeviceToHost, q->stream));
      CK(cudaMemcpyAsync(q->b.bst_host, q->b.bst, sizeof(BatchState), cudaMemcpyDeviceToHost,
                         q->stream));
      CK(cudaEventRecord(q->ev_snap, q->stream));
      q->inflight = true;
    }
    running |= q->inflight || q->retiring;
  }
  // nothing landed or started in this round: wait for the pending work of
  // one pool instead of returning straight into another poll
  if (!any && !launched && running) {
    for (auto& q : S->pools) {
      if (!q) continue;
      if (q->retiring) {
        CK(cudaEventSynchronize(q->ev_out));
        break;
      }
      if (q->inflight) {
        CK(cudaEventSynchronize(q->ev_snap));
        break;
      }
    }
  }
  if (pending_out) *pending_out = (int32_t)(S->waiting + S->running);
  return APPGA_OK;
}

extern "C" appga_status appga_server_poll(const appga_server* S, int64_t request,
                                          appga_request_stats* stats_out) {
  if (!S || !stats_out) return fail(APPGA_EINVAL, "null argument");
  auto it = S->reqs.find(request);
  if (it == S->reqs.end()) return fail(APPGA_EINVAL, "unknown request id");
  *stats_out = it->second.st;
  return APPGA_OK;
}

extern "C" appga_status appga_server_collect(appga_server* S, int64_t request, float* f_out_host,
                                             appga_request_stats* stats_out) {
  if (!S) return fail(APPGA_EINVAL, "null argument");
  auto it = S->reqs.find(request);
  if (it == S->reqs.end()) return fail(APPGA_EINVAL, "unknown request id");
  if (it->second.st.state != APPGA_REQ_DONE) return fail(APPGA_EBUSY, "request not finished");
  if (f_out_host)
    std::memcpy(f_out_host, it->second.f.data(), it->second.f.size() * sizeof(float));
  if (stats_out) *stats_out = it->second.st;
  S->reqs.erase(it);
  return APPGA_OK;
}

extern "C" appga_status appga_server_get_summary(const appga_server* S, appga_server_summary* out) {
  if (!S || !out) return fail(APPGA_EINVAL, "null argument");
  std::memset(out, 0, sizeof *out);
  out->submitted = S->submitted;
  out->completed = S->completed;
  out->waiting = S->waiting;
  out->running = S->running;
  out->slice_iters = S->slice_iters;
  out->pools = live_pools(S);
  out->device_bytes = S->bytes;
  out->p50_latency_s = percentile(S->latencies, 0.50);
  out->p99_latency_s = percentile(S->latencies, 0.99);
  double sum = 0.0, mx = 0.0, qs = 0.0;
  for (double v : S->latencies) {
    sum += v;
    mx = std::max(mx, v);
  }
  for (double v : S->queue_waits) qs += v;
  const size_t n = S->latencies.size();
  out->mean_latency_s = n ? sum / (double)n : kNaN;
  out->max_latency_s = n ? mx : kNaN;
  out->mean_queue_s = n ? qs / (double)n : kNaN;
  out->pool_slot_steps = S->pool_slot_steps;
  out->live_slot_steps = S->live_slot_steps;
  out->replay_seconds = S->replay_seconds;
  return APPGA_OK;
}
