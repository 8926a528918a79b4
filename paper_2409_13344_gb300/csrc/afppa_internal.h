// Device arguments and launchers of the AFPPA kernels (kernels_afppa.cu).
#pragma once

#include <cuda_runtime.h>

#include "appga_internal.h"

namespace appga {

struct DualArgs {
  int32_t n;               // image side
  float lambda1, lambda2;  // ball radii of the dual groups
  const float* f[3];       // iterate ring
  float* b[3];             // first-order dual ring, [2][d] (field-major)
  float* c[3];             // second-order dual ring, [4][d]
  float* gR;               // out: B1^T b~ + B2^T c~ for the next pixel phase
  const SolverState* st;   // k (index of the newest iterate), theta, rho
};

cudaError_t launch_afppa_dual(const DualArgs& a, cudaStream_t s);
// out[0] = ||x - y||^2, out[1] = ||x||^2 in FP64 (device doubles)
cudaError_t launch_norms2(int d, const float* x, const float* y, double* out, cudaStream_t s);

}  // namespace appga
