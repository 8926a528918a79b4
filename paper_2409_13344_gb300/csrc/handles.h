// Host-side definitions of the opaque handles and the helpers shared by the
// translation units of the C ABI (single-slice API, batched API, server).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>

#include "appga.h"
#include "appga_internal.h"
#include "batched_internal.h"

namespace appga {

// Device workspace of the single-slice solver (per matrix, allocated lazily).
struct Workspace {
  bool ready = false;
  int m = 0, d = 0;
  float* f[3] = {nullptr, nullptr, nullptr};
  float2* y[2] = {nullptr, nullptr};  // A f^k as double-float pairs
  float* w = nullptr;
  float* gR = nullptr;  // B^T grad phi~(B f~) of the current iterate
  float* pfreeze = nullptr;
  float2* partial_p = nullptr;
  float2* partial_r = nullptr;
  float2* partial_aux = nullptr;
  unsigned int* gtick = nullptr;  // group tickets of the grid reductions
  double* scalars = nullptr;      // device doubles for standalone results
  float* ft = nullptr;  // the current iterate in the 8 x 8-tiled pixel order (loop gathers)
  float2* fpair = nullptr;  // folded loop: (f_j, f_{quarter_turn(j)}) in the tiled order
  ThetaEntry* theta_tab = nullptr;  // momentum scalars of the current run
  int theta_cap = 0;                // entries of theta_tab
  SolverState* st = nullptr;
  SolverState* st_scratch = nullptr;
  SolverState* st_host = nullptr;  // pinned
  int* flag = nullptr;
  int* flag_host = nullptr;        // pinned
  double* scalars_host = nullptr;  // pinned
  // device staging for the host-buffer entry point
  float* d_g = nullptr;
  float* d_gamma = nullptr;
  float* d_finit = nullptr;
  float* d_fout = nullptr;
  // graph cache: executable graphs of n maps (n = the replay length and the
  // powers of two below it) for the parameters in gkey
  std::map<int, cudaGraphExec_t> gexec;
  std::string gkey;
  // whole-call graphs of short calls, by their arguments, and how often
  // other arguments were seen (a call graph is captured on the third call)
  std::map<std::string, cudaGraphExec_t> call_graphs;
  std::map<std::string, int> call_seen;
};

// Launch schedule of the batched kernels (0 = the kernels' defaults), as
// picked by appga_autotune_batched for one padded width and precision.
struct BatchSchedule {
  int spmv_per_sm = 0;     // forward-phase SpMV blocks per SM
  int stencil_per_sm = 0;  // stencil blocks per SM
  int pixel_per_sm = 0;    // back-projection blocks per SM
  int chunk = 0;           // slices per sub-batch (0: the whole batch at once)
  int gather_rows_fw = 0;  // rows gathered per step by the forward projection (0: 8)
  int gather_rows_px = 0;  // rows gathered per step by the back-projection (0: 8)
  bool operator==(const BatchSchedule& o) const {
    return spmv_per_sm == o.spmv_per_sm && stencil_per_sm == o.stencil_per_sm &&
           pixel_per_sm == o.pixel_per_sm && chunk == o.chunk &&
           gather_rows_fw == o.gather_rows_fw && gather_rows_px == o.gather_rows_px;
  }
};

// Dual fields of the AFPPA solver (per matrix, allocated lazily).
struct AfppaWorkspace {
  float* b[3] = {nullptr, nullptr, nullptr};  // [2][d] first-order duals, iterate ring
  float* c[3] = {nullptr, nullptr, nullptr};  // [4][d] second-order duals
  double* norms = nullptr;                    // device [2]
  double* norms_host = nullptr;               // pinned [2]
};

// Device workspace of the batched solver for one padded batch width Kp.
struct BatchWorkspace {
  int Kp = 0, m = 0, d = 0;
  float* f[3] = {nullptr, nullptr, nullptr};  // [d][Kp]
  float* y[2] = {nullptr, nullptr};           // [m][Kp]
  float* w = nullptr;                         // [m][Kp]
  float* gR = nullptr;                        // [d][Kp]
  float* pfreeze = nullptr;                   // [d][Kp]
  float* g = nullptr;                         // [m][Kp]
  float* gamma = nullptr;                     // [m][Kp]
  SlotState* slots = nullptr;                 // [Kp]
  SlotState* slots_host = nullptr;            // pinned [Kp]
  BatchState* bst = nullptr;
  BatchState* bst_host = nullptr;             // pinned
  float2* partial = nullptr;                  // (blocks + groups) x Kp
  float2* fpartial = nullptr;                 // forward-phase objective partials, blocks x Kp
  unsigned int* gtick = nullptr;
  int* flag = nullptr;
  int* flag_host = nullptr;
  float* fsm[3] = {nullptr, nullptr, nullptr};  // volume mode: slice-major iterate ring [Kp][d]
  float* gsm = nullptr;                         // volume mode: slice-major 3-D gradient
  double* vscal = nullptr;       // volume objective terms: [Kp] data terms, regulariser
  double* vscal_host = nullptr;  // pinned mirror
  cudaGraphExec_t gexec = nullptr;
  std::string gkey;
  // volume mode: the 3-D stencil's branch of the captured step (a second
  // stream forked from and joined to the solver's stream by two events)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

void free_batch_workspace(BatchWorkspace* bw);
// Device bytes of a batched workspace of width Kp for an m x d matrix.
int64_t batch_workspace_bytes(int m, int d, int Kp);
// Allocates every array of a width-Kp workspace (frees what it made on error).
cudaError_t alloc_batch_workspace(BatchWorkspace& b, int m, int d, int Kp);
// Kernel arguments of one batched step over workspace b with matrix arrays
// from (A, At, inv_lambda).
void make_batch_args(const DevCSR& A, const DevCSR& At, const float* inv_lambda, int n,
                     BatchWorkspace& b, bool bf16, bool track, const BatchSchedule& sch,
                     BFwdArgs* fa, BPixArgs* pa);
// Tuned schedule of matrix M for padded width Kp and precision (defaults if none).
BatchSchedule tuned_schedule(const appga_matrix* M, int Kp, bool bf16);
// Slot state of a problem run with `p` from iterate index k0 (active), or an
// empty slot that holds no problem (inactive).
SlotState slot_from_params(const appga_params* p, int k0, bool active);
// Captures S x (pixel update, forward phase) into an executable graph; with
// vb (volume mode) each step is pixel update, transpose of the new iterate to
// the slice-major ring, forward phase, 3-D stencil, transpose of its gradient.
struct VolumeSteps {
  Vol3Args va;
  float* slot_ring[3];
  float* slice_ring[3];
  int d, Kp, nz;
  // the stencil branch runs on `side`, forked after the iterate's transpose
  // and joined before the next pixel update, beside the forward phase
  cudaStream_t side;
  cudaEvent_t ev_fork, ev_join;
};
cudaError_t capture_batch_graph(const BFwdArgs& fa, const BPixArgs& pa, int S, cudaStream_t s,
                                cudaGraphExec_t* out, const VolumeSteps* vb = nullptr);
// APPGA on a volume of K <= 128 slices sharing the matrix (the batched solver
// in volume mode): device buffers as in appga_reconstruct_batched; on return
// the workspace's pinned slot and batch states hold the final states.
appga_status volume_solve(appga_ctx* ctx, appga_matrix* M, int32_t K, const float* g,
                          const float* gamma, const float* f_init, const appga_params* params,
                          float* f_out, void* stream);
// The batched kernels stage the offset col * Kp of every gathered slot-minor
// row in 32 bits: APPGA_OK when max(m, d) * Kp stays below 2^31, else
// APPGA_EINVAL (with the library's error message set).
appga_status check_slot_width(const appga_matrix* M, int Kp);

}  // namespace appga

struct appga_ctx {
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

struct appga_matrix {
  appga_ctx* ctx = nullptr;
  int32_t m = 0, d = 0, n = 0, na = 0;
  int64_t nnz = 0;
  appga::DevCSR A, At;
  appga::DevCSR A_tiled;  // A with column indices in the 8 x 8-tiled pixel order
                          // (shares row_ptr and values with A)
  // the solver loop's projections in the sliced layout: A with tiled
  // columns, and A^T (both or neither, cols == NULL when the matrix's
  // columns do not fit the packed words)
  appga::DevSell sell_a, sell_t;
  // the quarter-turn folded loop (when A has the symmetry bit for bit and it
  // was not turned off): the first m/2 rows of A with tiled columns, and
  // their transpose in orbit order, both sliced (off == NULL: not folded)
  appga::DevSell fold_a, fold_t;
  int32_t fold_nb = 0;  // bins per angle of the folded matrix
  float* inv_lambda = nullptr;       // 1/Lambda of the FP32 values
  float* inv_lambda_bf16 = nullptr;  // 1/Lambda of the BF16-rounded values
  int32_t has_bf16 = 0;
  int64_t bytes = 0;
  long long npfov = 0;  // pixels of the initial-image disk
  appga::Workspace ws;
  appga::BatchWorkspace* bw = nullptr;  // batched workspace (one width at a time)
  appga::AfppaWorkspace* aw = nullptr;  // AFPPA dual fields
  std::map<int, appga::BatchSchedule> tuned;  // key: padded width * 2 + BF16
};

namespace appga {

appga_status fail(appga_status s, const std::string& msg);
appga_status cuda_fail(cudaError_t e, const char* what);

template <typename T>
cudaError_t dalloc(T** p, size_t count, int64_t* bytes = nullptr) {
  *p = nullptr;
  if (count == 0) count = 1;
  const size_t b = count * sizeof(T);
  cudaError_t e = cudaMalloc((void**)p, b);
  if (e == cudaSuccess && bytes) *bytes += (int64_t)b;
  return e;
}

// Single-slice helpers shared by the solvers (api.cpp).
appga_status ensure_workspace(appga_matrix* M);
// theta_{k0+i}, i <= max_iters, of a run into ws.theta_tab (grown as needed)
// and theta_{k0} into the state st.
appga_status momentum_table(appga_matrix* M, SolverState* st, int k0, const appga_params* p,
                            cudaStream_t s, const SolverState* init = nullptr);
IterParams iter_params(const appga_params* p, bool track);
bool bf16_requested(const appga_matrix* M, const appga_params* p);
appga_status check_params_and_mat(appga_ctx* ctx, const appga_matrix* M, const appga_params* p);
appga_status validate_inputs(appga_matrix* M, const float* g, const float* gamma, const float* f,
                             cudaStream_t s);
void free_afppa_workspace(AfppaWorkspace* aw);

// The solver loop's projection layout in fa / pa: the folded sliced
// layout, the sliced layout or the CSR (its tiled columns when the loop
// gathers from the tiled copy); the gather copy is ws.fpair, ws.ft or the
// iterate ring.
void loop_layout(const appga_matrix* M, FwdArgs* fa, PixArgs* pa);
// True if the loop gathers from a copy of f (tiled or folded pairs).
bool loop_gathers_copy();
// Fills the loop's gather copy of f^k (tiled or folded pairs), if it has one.
cudaError_t loop_gather_copy(const appga_matrix* M, const float* f, cudaStream_t s);

// The objective terms of K slices (f [K][d], g and gamma [K][m]) enqueued on
// s without a host round trip, in the arithmetic of appga_objective: slice
// i's data term into dev_out[2i] (double-float projection) and, with_reg, its
// SHOITV regulariser into dev_out[2i + 1].
appga_status objective_terms(appga_matrix* M, int K, const float* f, const float* g,
                             const float* gamma, const appga_params* p, bool with_reg,
                             double* dev_out, cudaStream_t s);

// Orders ctx->stream after the caller's stream / the caller's after ctx->stream.
appga_status enter_stream(appga_ctx* ctx, void* stream);
appga_status leave_stream(appga_ctx* ctx, void* stream);

}  // namespace appga

#define APPGA_CK(call)                                               \
  do {                                                               \
    cudaError_t e_ = (call);                                         \
    if (e_ != cudaSuccess) return ::appga::cuda_fail(e_, #call);     \
  } while (0)
