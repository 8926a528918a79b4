// Device structures and launchers of the batched (multi-slice) kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "appga_internal.h"

namespace appga {

// Per-slot device state: iteration index, momentum, objective, stop flag and
// the slot's model parameters.  Slots are independent problems sharing A.
struct SlotState {
  int32_t k;          // index of the slot's current iterate
  int32_t k0;         // first index of the slot's run
  int32_t k_last;     // last step index to run
  int32_t done;       // finished (iteration cap or stopping test)
  int32_t result_k;   // index of the slot's result
  int32_t stopped_early;
  int32_t active;     // the slot holds a problem
  int32_t freeze_iter;
  int32_t momentum;
  int32_t fresh;      // just admitted: f^{k-1} = f^k, needs its first forward phase
  int32_t phi_k;      // iterate index whose objective is in phi_cur (-1: none)
  int32_t rollback;   // stopped one step back: the result is the previous ring entry
  float theta_hi, theta_lo;  // theta_k as a double-float pair
  float lambda1, lambda2, eps, beta;
  double theta, t_cur, phi_cur, phi_prev;
  double omega, a, b, rel_tol;
  unsigned long long guard_hits;
};

struct BatchState {
  int32_t gstep;      // global step: ring slot of the current iterates
  int32_t remaining;  // live slots
  int32_t flags;
  int32_t phi_tot_k;  // volume mode: iterate index of phi_tot_cur (-1: none)
  unsigned int ticket_r, ticket_p, ticket_aux, pad2;
  double phi_tot_cur, phi_tot_prev;  // volume mode: objective of the whole volume
};

struct BFwdArgs {
  DevCSR A;
  int32_t n, Kp;
  int32_t mode;  // 0: solver step; 1: project the previous iterate only;
                 // 2: first forward phase of the fresh slots only (admission)
  int32_t track;
  int32_t use_bf16;
  int32_t n_spmv_blocks;  // set by the launcher
  int32_t spmv_per_sm;    // SpMV blocks per SM (0: default); tuned by the autotuner
  int32_t stencil_per_sm; // stencil blocks per SM (0: default)
  int32_t no_stencil;     // volume mode: the 3-D stencil runs in its own kernel
  int32_t gather_rows;    // image rows gathered per step: 8 (0: default) or 4; tuned
  float* f[3];
  float* y[2];
  float* w;
  const float* g;
  const float* gamma;
  float* gR;
  SlotState* slots;
  BatchState* bst;
  float2* fpartial;  // per-slot objective partials, one row of Kp per block
};

struct BPixArgs {
  DevCSR At;
  int32_t n, Kp;
  int32_t use_bf16;
  int32_t blocks_per_sm;  // 0: default; tuned by the autotuner
  int32_t gather_rows;    // weight rows gathered per step: 8 (0: default) or 4; tuned
  int32_t pad;
  float* f[3];
  const float* w;
  const float* gR;
  const float* inv_lambda;
  float* pfreeze;
  SlotState* slots;
  BatchState* bst;
  float2* partial;
  unsigned int* gtick;
  // objective partials left by the forward phase of the same step (track):
  // reduced here, where the stopping test runs
  const float2* fpartial;
  int32_t n_fpartial;
  int32_t track;
  int32_t joint;  // volume mode: one stopping test on the sum of the slots' objectives
};

// 3-D SHOITV stencil (kernels_vol.cu) on slice-major volumes: voxel
// (z, r, c) at z n^2 + r n + c.  Solver mode (bst != null): f^k and f^{k-1}
// are the slice-major ring entries of the current step (f[G % 3] and
// f[(G + 2) % 3]), theta, lambda and eps come from slot z; stand-alone mode:
// f[0] is the volume, f~ = f, lam1/lam2/eps as given.
struct Vol3Args {
  int32_t n, nz;
  const float* f[3];
  const SlotState* slots;
  const BatchState* bst;
  float lam1, lam2, eps;
  int32_t want_reg;       // also the regulariser at f^k: one row of pstride
  int32_t pstride;        // per-slice double-float sums per block in partial
  int32_t pad;
  float* gR;              // out: B^T grad phi~(B f~), slice-major
  float2* partial;        // out (want_reg): stencil3d_grid rows of pstride
};
int stencil3d_max_slices();
int stencil3d_grid(int n, int nz);
cudaError_t launch_stencil3d(const Vol3Args& a, cudaStream_t s);
// *out = sum of rows x cols double-float pairs (row stride pstride), in FP64
cudaError_t launch_sum_pairs(const float2* p, int rows, int cols, int pstride, double* out,
                             cudaStream_t s);
// Volume mode: the current ring entry (bst->gstep) of the slot-minor iterate
// ring [d][Kp] into the slice-major ring [nz][d] (every entry if all != 0),
// and a slice-major gradient [nz][d] into the slot-minor [d][Kp].  Both do
// nothing once no slot is live.
cudaError_t launch_slots_to_slices(float* const* slot_ring, float* const* slice_ring, int d,
                                   int Kp, int nz, const BatchState* bst, int all,
                                   cudaStream_t s);
cudaError_t launch_slices_to_slots(const float* in, float* out, int d, int Kp, int nz,
                                   const BatchState* bst, cudaStream_t s);

int batch_max_blocks();
// Grid of the forward phase for these arguments (the launcher's own choice).
int bforward_grid(const BFwdArgs& a);
// Slots whose result sits one ring entry back (stopped by the test in the
// last pixel phase): copy it into the current entry and clear the mark.
cudaError_t launch_resolve_rollback(const BFwdArgs& a, cudaStream_t s);
cudaError_t launch_bforward(const BFwdArgs& a, cudaStream_t s);
// The batched projectors' inner loop alone over M (rows reduced against the
// Kp-wide rows of x, [cols][Kp]; no epilogue) in the row order of the forward
// projection (forward) or of the back-projection, with blocks_per_sm (1..16)
// blocks per SM; sink: at least (SMs x 16) floats, written only in a case
// that does not arise.
cudaError_t launch_gather_probe(const DevCSR& M, bool forward, const float* x, int Kp,
                                float* sink, int blocks_per_sm, cudaStream_t s);
cudaError_t launch_bpixel(const BPixArgs& a, cudaStream_t s);
// Slot lists: where `ids` is given, slice k goes to slot ids[k] (a device
// array of K ints); otherwise to slot s0 + k.
cudaError_t launch_binit_momentum(SlotState* slots, int Kp, bool only_fresh, cudaStream_t s);
cudaError_t launch_to_slot_minor(const float* in, int K, int len, float* out, int Kp, int s0,
                                 const int* ids, cudaStream_t s);
cudaError_t launch_from_slot_minor(const float* in, int K, int len, int Kp, int s0,
                                   const int* ids, float* out, cudaStream_t s);
cudaError_t launch_copy_slots(const float* src, float* dst, int len, int Kp, const int* ids,
                              int K, cudaStream_t s);
cudaError_t launch_fill_slots(float* out, int len, int Kp, int s0, int s1, float v, cudaStream_t s);
cudaError_t launch_binit_image(const float* g, const float* gamma, int m, int n, int n_angles,
                               long long npfov, int K, int Kp, int s0, const int* ids,
                               float* f_out, cudaStream_t s);

}  // namespace appga
