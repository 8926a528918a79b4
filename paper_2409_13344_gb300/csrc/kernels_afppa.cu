// CUDA kernels of the accelerated fixed-point proximity algorithm (AFPPA) for
// the non-smooth HOITV model (the paper's extension of the GN momentum,
// Sec. 4.4):
//
//   k_afppa_dual : after the pixel phase of step k has produced f^{k+1}, the
//                  dual updates
//                    b^{k+1} = rho1 (I - prox_{(lam1/rho1)||.||})(b~/rho1 + B1 u)
//                            = proj_{ball(lam1)}(b~ + rho1 B1 u),
//                    c^{k+1} = proj_{ball(lam2)}(c~ + rho2 B2 u),
//                  u = 2 f^{k+1} - f~^k, group by group, and the term
//                  B1^T b~^{k+1} + B2^T c~^{k+1} that the next pixel phase adds
//                  to the gradient (b~, c~ the momentum extrapolations).
//   k_norms2     : ||x - y||^2 and ||x||^2 (double-float), for the relative
//                  error RE = ||f^{k+1} - f^k|| / ||f^{k+1}||.
//
// The forward and pixel phases are the APPGA kernels (the forward phase
// without its smoothed-TV stencil; the pixel phase also reduces the largest
// preconditioner entry, from which rho1 = 1/(16 p_max), rho2 = 1/(128 p_max)).
//
// Tile: 4 x 32 pixels per block.  u is staged with a 2-pixel halo so that the
// six difference fields, and so the new duals, are known on a 1-pixel halo,
// which the adjoint needs; every block writes the duals of its own pixels only.
#include <cuda_runtime.h>

#include "afppa_internal.h"
#include "appga_internal.h"
#include "device_common.cuh"

namespace appga {
namespace {

constexpr int DR = 4, DC = 32, DT = DR * DC;
constexpr int TWD = DC + 4, VWD = DC + 2;

// Projects the group z (len components) onto the l2 ball of radius r.
template <int L>
__device__ __forceinline__ void ball_project(float (&z)[L], float r) {
  float n2 = 0.f;
#pragma unroll
  for (int q = 0; q < L; ++q) n2 = fmaf(z[q], z[q], n2);
  if (n2 > r * r) {
    const float s = r / sqrtf(n2);
#pragma unroll
    for (int q = 0; q < L; ++q) z[q] *= s;
  }
}

__global__ void __launch_bounds__(DT) k_afppa_dual(DualArgs a) {
  __shared__ float T[DR + 4][TWD];
  __shared__ float V[6][DR + 2][VWD];
  const SolverState* st = a.st;
  const int k1 = st->k;  // index of f^{k+1}, the iterate the pixel phase just wrote
  const float th_k = st->theta_prev, th_k1 = st->theta_hi;
  const float rho1 = st->rho1, rho2 = st->rho2;
  const int n = a.n, d = n * n, tid = threadIdx.x;
  const float* f1 = a.f[k1 % 3];
  const float* f0 = a.f[(k1 + 2) % 3];
  const float* fm = a.f[(k1 + 1) % 3];
  float* bn = a.b[k1 % 3];
  const float* b0 = a.b[(k1 + 2) % 3];
  const float* bm = a.b[(k1 + 1) % 3];
  float* cn = a.c[k1 % 3];
  const float* c0 = a.c[(k1 + 2) % 3];
  const float* cm = a.c[(k1 + 1) % 3];
  const int ntx = (n + DC - 1) / DC;
  const int r0 = (blockIdx.x / ntx) * DR, c0x = (blockIdx.x % ntx) * DC;

  // u = 2 f^{k+1} - f~^k on the tile with a 2-pixel halo (0 outside the image)
  for (int t = tid; t < (DR + 4) * TWD; t += DT) {
    const int ii = t / TWD, jj = t % TWD;
    const int r = r0 - 2 + ii, c = c0x - 2 + jj;
    float v = 0.f;
    if (r >= 0 && r < n && c >= 0 && c < n) {
      const int j = r * n + c;
      const float ft = fmaf(th_k, f0[j] - fm[j], f0[j]);
      v = fmaf(2.f, f1[j], -ft);
    }
    T[ii][jj] = v;
  }
  __syncthreads();
  // new duals on the 1-pixel halo ring and the tile, then their extrapolation
  for (int t = tid; t < (DR + 2) * VWD; t += DT) {
    const int ii = t / VWD, jj = t % VWD;
    const int r = r0 - 1 + ii, c = c0x - 1 + jj;
    float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (r >= 0 && r < n && c >= 0 && c < n) {
      const int j = r * n + c;
      float u[6];
      diff_fields<TWD>(T, ii + 1, jj + 1, r, c, n, u);
      float zb[2], bk[2], zc[4], ck[4];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        bk[q] = b0[q * d + j];
        const float bt = fmaf(th_k, bk[q] - bm[q * d + j], bk[q]);
        zb[q] = fmaf(rho1, u[q], bt);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        ck[q] = c0[q * d + j];
        const float ct = fmaf(th_k, ck[q] - cm[q * d + j], ck[q]);
        zc[q] = fmaf(rho2, u[2 + q], ct);
      }
      ball_project<2>(zb, a.lambda1);
      ball_project<4>(zc, a.lambda2);
      if (ii >= 1 && ii <= DR && jj >= 1 && jj <= DC) {
#pragma unroll
        for (int q = 0; q < 2; ++q) bn[q * d + j] = zb[q];
#pragma unroll
        for (int q = 0; q < 4; ++q) cn[q * d + j] = zc[q];
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) v[q] = fmaf(th_k1, zb[q] - bk[q], zb[q]);
#pragma unroll
      for (int q = 0; q < 4; ++q) v[2 + q] = fmaf(th_k1, zc[q] - ck[q], zc[q]);
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) V[q][ii][jj] = v[q];
  }
  __syncthreads();
  // B1^T b~^{k+1} + B2^T c~^{k+1} at the tile pixels (the adjoint forms of B)
  for (int t = tid; t < DR * DC; t += DT) {
    const int ii = t / DC, jj = t % DC;
    const int r = r0 + ii, c = c0x + jj;
    if (r < n && c < n) {
      const int i = ii + 1, j = jj + 1;
      const bool r_lo = r >= 1, r_hi = r <= n - 2, c_lo = c >= 1, c_hi = c <= n - 2;
      float g = 0.f;
      if (c_lo) g += V[0][i][j];
      if (c_hi) g -= V[0][i][j + 1];
      if (r_lo) g += V[1][i][j];
      if (r_hi) g -= V[1][i + 1][j];
      g += form_u3<VWD>(V[2], i, j, c_lo, c_hi);
      g += form_u6<VWD>(V[3], i, j, r_lo, c_lo, c_hi);
      g += form_u5<VWD>(V[4], i, j, r_lo, r_hi);
      g += form_u4<VWD>(V[5], i, j, r_lo, r_hi, c_lo);
      a.gR[r * n + c] = g;
    }
  }
}

// out[0] = ||x - y||^2, out[1] = ||x||^2 (one block, fixed order)
__global__ void __launch_bounds__(1024) k_norms2(int d, const float* __restrict__ x,
                                                 const float* __restrict__ y, double* out) {
  float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    df e;
    two_sum(x[j], -y[j], e.hi, e.lo);
    const df e2 = df_mul(e, e);
    acc_add(h0, l0, e2.hi, e2.lo);
    const df xx = df_mul({x[j], 0.f}, {x[j], 0.f});
    acc_add(h1, l1, xx.hi, xx.lo);
  }
  const df s0 = block_sum_acc(h0, l0);
  const df s1 = block_sum_acc(h1, l1);
  if (threadIdx.x == 0) {
    out[0] = (double)s0.hi + (double)s0.lo;
    out[1] = (double)s1.hi + (double)s1.lo;
  }
}

}  // namespace

cudaError_t launch_afppa_dual(const DualArgs& a, cudaStream_t s) {
  const int tiles = ((a.n + DC - 1) / DC) * ((a.n + DR - 1) / DR);
  k_afppa_dual<<<tiles, DT, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_norms2(int d, const float* x, const float* y, double* out, cudaStream_t s) {
  k_norms2<<<1, 1024, 0, s>>>(d, x, y, out);
  return cudaGetLastError();
}

}  // namespace appga
