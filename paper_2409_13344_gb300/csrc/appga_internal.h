// Internal declarations shared by the host API and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "appga.h"

namespace appga {

// Poisson-ratio denominator guard: den = max(y + gamma, KAPPA * gamma).
constexpr double KAPPA = 1e-3;

// Rows of a CSR stored on the device, each row padded with (col = last
// column of the row, val = 0) to a multiple of ROW_PAD entries so every row
// starts on a 16-byte boundary and streams as 4-entry packs.
constexpr int ROW_PAD = 4;

// Packed column indices: the four entries of a row-padded 4-entry pack as
// one 64-bit word, the first column in bits 0-19 and the other three as
// signed 14-bit offsets from it in bits 20-33, 34-47 and 48-61 (2 bytes per
// entry instead of 4).  A matrix whose columns do not fit (a column above
// 2^20 - 1 or an offset outside [-8192, 8191]) keeps 32-bit indices only.
constexpr int PACK_ENTRIES = ROW_PAD;
constexpr int PACK_BASE_BITS = 20;
constexpr int32_t PACK_BASE_MAX = (1 << PACK_BASE_BITS) - 1;
constexpr int32_t PACK_OFFSET_MAX = 8191;

// Device copy of a HostSell (see below), with an optional BF16 copy of the
// values (4 per pack, 8 bytes).
struct DevSell {
  int32_t rows = 0, slices = 0;
  int32_t* off = nullptr;
  uint2* cols = nullptr;    // packed words (APPGA_SELL_PACK), or
  int4* cols32 = nullptr;   // four 32-bit columns per pack
  float4* vals = nullptr;
  uint2* vals_bf16 = nullptr;
};

// Quarter-turn folding of a parallel-beam A.  With NPA angles a*pi/NPA
// (NPA even) stored angle-major (row i = a*nb + b) over an N x N image (N
// even), the ray of angle a + NPA/2 and bin nb-1-b is the ray of angle a and
// bin b turned a quarter turn about the image centre, a turn that moves pixel
// (r, c) to (N-1-c, r).  When A has this symmetry bit for bit,
//   A[fold_partner(i), quarter_turn(j)] = A[i, j]   for every i < m/2 and j,
// the solver loop streams only the first m/2 rows (and their transpose):
//   (A f)_i               = sum_j A[i,j] f_j
//   (A f)_fold_partner(i) = sum_j A[i,j] f_{quarter_turn(j)}
//   (A^T w)_j = s1(j) + s2(quarter_turn^-1(j)),  s1(p) = sum_{i<m/2} A[i,p] w_i,
//                                              s2(p) = sum_{i<m/2} A[i,p] w_{fold_partner(i)}
// so each stored entry serves two products of each projection.
__host__ __device__ inline int32_t fold_partner(int32_t i, int32_t half, int32_t nb) {
  return i + half + nb - 1 - 2 * (i % nb);
}
__host__ __device__ inline int32_t quarter_turn(int32_t j, int32_t n) {
  return (n - 1 - j % n) * n + j / n;
}
// Member r (0..3) of pixel orbit o under the quarter turn: o runs over the
// (N/2) x (N/2) top-left quadrant row-major; member r is that pixel turned r
// times.  Returns (row, column).
__host__ __device__ inline void orbit_pixel(int32_t o, int32_t r, int32_t n, int32_t* pr,
                                            int32_t* pc) {
  const int32_t h = n / 2, R = o / h, C = o % h;
  switch (r & 3) {
    case 0: *pr = R; *pc = C; break;
    case 1: *pr = n - 1 - C; *pc = R; break;
    case 2: *pr = n - 1 - R; *pc = n - 1 - C; break;
    default: *pr = C; *pc = n - 1 - R; break;
  }
}

struct DevCSR {
  int32_t rows = 0, cols = 0;
  int64_t nnz_padded = 0;
  int32_t* row_ptr = nullptr;    // rows + 1 padded offsets
  int32_t* col = nullptr;        // nnz_padded
  float* val = nullptr;          // nnz_padded
  uint16_t* val_bf16 = nullptr;  // nnz_padded (optional BF16 copy)
};

// Device-resident iteration state of one solve.  Kernels derive buffer
// indices and the momentum scalar from it, so captured graphs replay
// unchanged from one iteration to the next.
//
// Step hand-over in the solver loop: the forward phase of a step reads the
// step's index and run status from k_next / done_next (its block 0 then
// publishes them, with theta, as k / done / theta for the pixel phase), and
// the finalisation of the step -- in the pixel phase's first blocks, or in
// the one-block k_finalize -- writes the next ones.  So no kernel overwrites
// a field that blocks of the same kernel may still read.
struct SolverState {
  int32_t k;          // index of the current iterate f^k
  int32_t k_last;     // last pixel-phase index to run
  int32_t k0;         // first index of this run
  int32_t done;       // 0 running; 1 finished; 2 finished, objective of the result pending
  int32_t result_k;   // index of the returned iterate
  int32_t stopped_early;
  int32_t flags;      // APPGA_FLAG_* (sticky)
  int32_t k_next;     // index of the next forward phase
  double theta;       // theta_k for the current k (FP64)
  float theta_hi;     // theta_k as a double-float pair (for FP32-pipe arithmetic)
  float theta_lo;
  double t_cur;       // t_k (Nesterov recursion)
  double data_term;   // F(f^k) = sum y - g ln(y + gamma)
  double phi_cur;     // Phi(f^k)
  double phi_prev;    // Phi(f^{k-1})
  unsigned long long guard_hits;
  unsigned int ticket_p;
  unsigned int ticket_r;
  unsigned int ticket_aux;
  int32_t done_next;  // run status for the next forward phase
  // fixed-point proximity iteration (AFPPA): theta of the step just taken,
  // the dual step sizes from the largest preconditioner entry of that step,
  // and that largest entry as bits (positive floats order as integers)
  float theta_prev;
  float rho1, rho2;
  unsigned int pmax_bits;
};

// One momentum scalar of a run: the FP64 value and its double-float split.
struct ThetaEntry {
  double v;
  float hi, lo;
};

struct IterParams {
  float lambda1, lambda2, eps, beta;
  double omega, a, b, rel_tol;
  int32_t momentum;
  int32_t freeze_iter;
  int32_t track;  // evaluate Phi on the device each iteration
  int32_t pad;
};

// Forward-phase kernel arguments (steps a1, a2, a4 and the objective).
struct FwdArgs {
  DevCSR A;
  const float* f[3];   // iterate ring (loop) / f in slot 0 (standalone)
  float2* y[2];        // loop: projection ring A f^k as double-float pairs (hi, lo)
  double* y_out;       // standalone: A f in FP64
  float* w;            // back-projection weight 1 - g/den (may be null)
  const float* g;
  const float* gamma;
  float* gR;           // loop: B^T grad phi~(B f~) of the current iterate
  SolverState* st;
  float2* partial;     // one double-float partial per block (+ group results)
  unsigned int* gtick; // group tickets of the grid reduction (zero between launches)
  double* data_out;    // standalone: where the data term goes (may be null)
  IterParams ip;       // loop: lambda, eps, stopping tolerance
  int32_t n;           // image side
  int32_t loop;        // 1: solver loop mode, 0: standalone
  int32_t want_data;   // evaluate the objective (data term; in the loop also the regulariser)
  int32_t use_bf16;
  int32_t no_stencil;  // solver loop without the SHOITV stencil blocks (AFPPA)
  // loop: f^k in the 8 x 8-tiled pixel order; then A carries tiled column
  // indices (its projector gathers from ft, the stencil still reads f[])
  const float* ft;
  int32_t solver_acc;  // 1: accumulate y as the solver loop does, also when loop == 0
  // loop: first forward phase of a fresh run (f^{k-1} = f^k, so y~ = y and
  // the projection of f^{k-1} is not needed)
  int32_t fresh_first;
  // loop: theta_{k0+i} of the run (the forward phase takes theta_k from it)
  const ThetaEntry* theta_tab;
  // the sliced layout of A (solver projections with FP32 accumulation; its
  // columns index ft); S.cols == NULL: the CSR A
  DevSell S;
  // quarter-turn folded loop (fpair != NULL): S holds A's first fold_half
  // rows, the projector gathers fpair[t] = (f_j, f_{quarter_turn(j)}) at the
  // tiled index t of pixel j, and w is written as pairs (w_i,
  // w_{fold_partner(i)}) for the stored rows i
  const float2* fpair;
  int32_t fold_half;  // m / 2
  int32_t fold_nb;    // bins per angle
};

// Fused pixel-phase arguments (steps a0, a3, a4, a5).
struct PixArgs {
  DevCSR At;
  int32_t n;           // image side
  float* f[3];         // iterate ring: f^{k-1}, f^k read; f^{k+1} written
  const float* w;      // back-projection weight
  const float* gR;     // B^T grad phi~(B f~^k)
  const float* inv_lambda;
  float* pfreeze;      // frozen f^{K_P} (may be null)
  SolverState* st;
  float2* partial;
  unsigned int* gtick;
  // block partials of Phi(f^k) left by the forward phase of the same step
  // (ip.track): reduced here, where the stopping test runs
  const float2* fwd_partial;
  int32_t n_fwd_partial;
  // theta_{k0+i} of the run (launch_theta_table); NULL for a standalone
  // update, which then has no step to finalise
  const ThetaEntry* theta_tab;
  IterParams ip;
  int32_t use_bf16;
  int32_t want_pmax;  // also reduce the largest preconditioner entry (AFPPA step sizes)
  float* ft;          // if set: f^{k+1} also written in the 8 x 8-tiled pixel order
  // 1: the pixel phase's first blocks finalise the step (Phi(f^k) from the
  // forward phase's partials, stopping test, next index); 0: k_finalize does
  int32_t fuse_fin;
  // the sliced layout of A^T (S.cols == NULL: the CSR At)
  DevSell S;
  // quarter-turn folded loop (fpair != NULL): S holds the folded A^T (slice o
  // = the four pixels of orbit o, columns the stored rows), w holds pairs
  // (w_i, w_{fold_partner(i)}), and f^{k+1} is also written as the gather
  // pairs of the next forward phase
  float2* fpair;
};

// ---- launchers (kernels.cu) ----
int stencil_tiles(int n);
// grid of the solver-loop forward phase (sliced: A in the sliced layout)
int forward_blocks(int m, int n, bool sliced);
int max_partials(int m, int n);
int max_group_tickets(int m, int n);

cudaError_t launch_forward(const FwdArgs& a, cudaStream_t s);
cudaError_t launch_pixel(const PixArgs& a, cudaStream_t s);
cudaError_t launch_backproject(const DevCSR& At, const float* w, float* out, int use_bf16,
                               cudaStream_t s);
cudaError_t launch_stencil(int n, const float* f_cur, const float* f_prev, float theta,
                           float lam1, float lam2, float eps, float* out, cudaStream_t s);
cudaError_t launch_reg_term(int n, const float* f, float lam1, float lam2, float eps,
                            float2* partial, unsigned int* gtick, SolverState* st, double* out,
                            cudaStream_t s);
cudaError_t launch_validate_inputs(const float* g, const float* gamma, int m, const float* f,
                                   int d, int* flag, cudaStream_t s);
// Solver-run input check without a host round trip: on a bad g, gamma, fa or
// fb (fa, fb may be NULL) sets APPGA_FLAG_DOMAIN in st->flags and st->done.
cudaError_t launch_check_inputs(const float* g, const float* gamma, int m, const float* fa,
                                const float* fb, int d, SolverState* st, cudaStream_t s);
// One more finalisation of the solver loop: after the last forward phase of a
// tracked run it turns that phase's partials into Phi of the result.
cudaError_t launch_finalize(const PixArgs& a, cudaStream_t s);
// out = f^{result_k}, out_prev = f^{result_k - 1} (may be NULL) from the ring
// f[3], selected on the device from st; nothing is written if the run's
// inputs failed the check.
cudaError_t launch_copy_result(const SolverState* st, float* const f[3], float* out,
                               float* out_prev, int d, cudaStream_t s);
// theta_{k0+i}, i = 0..n, into tab and theta_{k0} into the state
// Pixel (r, c) of an n x n image in the 8 x 8-tiled order: tiles row-major,
// pixels row-major inside a tile; tiled_size(n) entries cover the image.
__host__ __device__ inline int64_t tiled_size(int n) {
  return (int64_t)((n + 7) / 8) * ((n + 7) / 8) * 64;
}
__host__ __device__ inline int32_t tiled_index(int r, int c, int n) {
  return (((r >> 3) * ((n + 7) / 8) + (c >> 3)) << 6) + ((r & 7) << 3) + (c & 7);
}
// ft[tiled_index(j)] = f[j] for the d = n * n pixels
cudaError_t launch_to_tiled(const float* f, float* ft, int n, cudaStream_t s);
// fpair[tiled_index(j)] = (f[j], f[quarter_turn(j)]) for the d = n * n pixels
cudaError_t launch_to_fold_pairs(const float* f, float2* fpair, int n, cudaStream_t s);
bool tiled_gather_enabled();  // the solver loop gathers from the tiled copy
// (with init: *st = *init first, so one launch starts a run)
cudaError_t launch_theta_table(SolverState* st, ThetaEntry* tab, int k0, int n, int momentum,
                               double a, double b, double omega, cudaStream_t s,
                               const SolverState* init = nullptr);
long long disk_pixels(int n);
// f_out = TMC * 1_disk; also into f_out2, (8 x 8-tiled) ft and the folded
// gather pairs fpair when not NULL (the disk is invariant under the quarter
// turn); with check_st set, g and gamma are checked as launch_check_inputs does.
cudaError_t launch_initial_image(const float* g, const float* gamma, int m, int n, int n_angles,
                                 long long npfov, float2* partial, unsigned int* gtick,
                                 SolverState* st, float* f_out, cudaStream_t s,
                                 float* f_out2 = nullptr, float* ft = nullptr,
                                 SolverState* check_st = nullptr, float2* fpair = nullptr);

// ---- host CSR helpers (csr_host.cpp) ----
struct HostCSR {
  int32_t rows = 0, cols = 0;
  std::vector<int32_t> row_ptr, col;
  std::vector<float> val;
};
// Checks a CSR and returns APPGA_OK or EINVAL/EDOMAIN with a message.
appga_status validate_csr(int32_t m, int32_t d, const int32_t* row_ptr, const int32_t* col,
                          const float* val, std::string* why);
// Stable transpose (counting sort by column): rows of the result keep the
// original row order.
void transpose_csr(int32_t m, int32_t d, const int32_t* row_ptr, const int32_t* col,
                   const float* val, HostCSR* out);
// Pads each row to a multiple of `mult` entries (col = last col, val = 0).
void pad_rows(int32_t rows, int32_t cols, const int32_t* row_ptr, const int32_t* col,
              const float* val, int mult, HostCSR* out);

// True if the CSR A (m x n*n) has the quarter-turn symmetry above bit for
// bit: n and n_angles even, m = n_angles * nb, no repeated column in a row,
// and every row i < m/2 equal to row fold_partner(i) with its columns turned.
bool quarter_turn_symmetric(int32_t m, int32_t n, int32_t n_angles, const int32_t* row_ptr,
                            const int32_t* col, const float* val);
// Transposed first half of A in orbit order: row 4*o + r lists the entries
// (i, A[i, p]) with i < half of pixel p = orbit_pixel(o, r), in ascending i,
// from the stable transpose `at` of the whole A.
void fold_transpose(const HostCSR& at, int32_t half, int32_t n, HostCSR* out);

// Round-to-nearest-even FP32 -> BF16 bits.
uint16_t float_to_bf16(float x);
// Packs a row-padded column array (a multiple of PACK_ENTRIES entries) into
// 64-bit words (layout above); false if some pack does not fit.
bool pack_columns(const std::vector<int32_t>& col, std::vector<uint64_t>* out);
// One pack of PACK_ENTRIES columns into a word; false if it does not fit.
bool encode_pack(const int32_t* c, uint64_t* word);

// Sliced layout of a row-padded CSR for the solver loop's projections
// (sliced ELLPACK over 4-entry packs): rows in slices of SELL_ROWS; each row
// owns SELL_LANES lanes of a warp, which take its packs in turn (pack k to
// lane k mod SELL_LANES at step k / SELL_LANES); a slice runs for as many
// steps as its longest row needs, and every step is one pack per lane, the
// 32 packs of a step stored consecutively.  Positions are counted in packs;
// padding packs have value 0 (and column 0).
#ifndef APPGA_SELL_LANES
#define APPGA_SELL_LANES 4
#endif
constexpr int SELL_LANES = APPGA_SELL_LANES;  // 1, 2, 4, 8, 16 or 32
static_assert(SELL_LANES >= 1 && SELL_LANES <= 32 && 32 % SELL_LANES == 0, "lanes per row");
constexpr int SELL_ROWS = 32 / SELL_LANES;
// Columns of the sliced layout as packed words (1) or as four 32-bit
// indices per pack (0).
#ifndef APPGA_SELL_PACK
#define APPGA_SELL_PACK 1
#endif
struct HostSell {
  int32_t rows = 0, slices = 0;
  std::vector<int32_t> off;    // slices + 1 pack offsets (a multiple of 32 apart)
  std::vector<uint64_t> cols;  // one packed word per pack (APPGA_SELL_PACK)
  std::vector<int32_t> cols32; // PACK_ENTRIES columns per pack (otherwise)
  std::vector<float> vals;     // PACK_ENTRIES values per pack
};
// false if some pack's columns do not fit the packed word or the layout
// exceeds 2^31 packs
bool build_sell(int32_t rows, const std::vector<int32_t>& row_ptr, const std::vector<int32_t>& col,
                const std::vector<float>& val, HostSell* out);

void set_error(const std::string& msg);

}  // namespace appga
