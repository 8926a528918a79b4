// 3-D SHOITV stencil (sm_103a): B^T grad phi~(B f~) of the volume regulariser
// and the regulariser's value, for volumes of nz slices of n x n pixels.
//
// The paper gives HOITV in 2-D (Sec. 2.1, Eq. gradenvL2); the 3-D operators
// here are the Kronecker generalisation: per voxel three first-order
// differences (Dc, Dr, Dz) and nine second-order fields (the paper's four 2-D
// blocks -Dc^T Dc, -Dr^T Dc, -Dr^T Dr, -Dr Dc^T, then -Dz^T Dz, -Dz^T Dc,
// -Dz Dc^T, -Dz^T Dr, -Dz Dr^T), D the backward difference with a zero first
// row along each axis.  grad phi~ scales the triple by lambda1 / max(||.||,
// eps) and the 9-vector by lambda2 / max(||.||, eps).
//
// Layout: voxel (z, r, c) of a volume sits at (r n + c) ps + z zs, so the
// same kernel serves the solver's slot-minor blocks (ps = Kp, zs = 1: slice z
// is slot z) and slice-major volumes (ps = 1, zs = n^2).
//
// Tiles of 2 x 32 pixels x 8 slices, one thread per (column, slice); f~ and
// f^k are staged with a 2-voxel halo in every axis, the twelve gradient
// fields with a 1-voxel halo, so each block writes only its own voxels.
// Blocks are persistent over the tiles and leave one row of per-slice
// regulariser sums (double-float pairs) each, in a fixed order.
#include <cuda_runtime.h>

#include "appga_internal.h"
#include "batched_internal.h"
#include "device_common.cuh"

namespace appga {
namespace {

constexpr int VR = 2, VC = 32, VS = 8;  // tile: rows x columns x slices
constexpr int VT = VC * VS;             // threads: one per (column, slice)
constexpr int HR = VR + 4, HC = VC + 4, HS = VS + 4;  // f tiles, halo 2
constexpr int WR = VR + 2, WC = VC + 2, WS = VS + 2;  // gradient fields, halo 1
constexpr int NF = 12;                                // 3 + 9 components
constexpr int MAXZ = 128;                             // slices (slots) at most

struct Vol3Smem {
  float T[HR][HC][HS];      // f~
  float K[HR][HC][HS];      // f^k (regulariser value)
  float W[NF][WR][WC][WS];  // grad phi~ fields
  float reg_hi[MAXZ], reg_lo[MAXZ];
};

struct Edges {
  bool c_lo, c_hi, r_lo, r_hi, z_lo, z_hi;
};
__device__ __forceinline__ Edges edges(int z, int r, int c, int nz, int n) {
  return {c >= 1, c <= n - 2, r >= 1, r <= n - 2, z >= 1, z <= nz - 2};
}

// Component Q of B x at a voxel, X(dz, dr, dc) reading x at the offset.
// The forms are the matrix rows written out from the definition of D.
template <int Q, class F>
__device__ __forceinline__ float comp(const F& X, const Edges& e) {
  const float x = X(0, 0, 0);
  if constexpr (Q == 0) return e.c_lo ? x - X(0, 0, -1) : 0.f;  // Dc
  if constexpr (Q == 1) return e.r_lo ? x - X(0, -1, 0) : 0.f;  // Dr
  if constexpr (Q == 2) return e.z_lo ? x - X(-1, 0, 0) : 0.f;  // Dz
  if constexpr (Q == 3)  // -Dc^T Dc
    return (e.c_lo ? -(x - X(0, 0, -1)) : 0.f) + (e.c_hi ? X(0, 0, 1) - x : 0.f);
  if constexpr (Q == 4)  // -Dr^T Dc
    return e.c_lo ? ((e.r_lo ? -(x - X(0, 0, -1)) : 0.f) +
                     (e.r_hi ? X(0, 1, 0) - X(0, 1, -1) : 0.f))
                  : 0.f;
  if constexpr (Q == 5)  // -Dr^T Dr
    return (e.r_lo ? -(x - X(0, -1, 0)) : 0.f) + (e.r_hi ? X(0, 1, 0) - x : 0.f);
  if constexpr (Q == 6)  // -Dr Dc^T
    return e.r_lo ? ((e.c_lo ? -(x - X(0, -1, 0)) : 0.f) +
                     (e.c_hi ? X(0, 0, 1) - X(0, -1, 1) : 0.f))
                  : 0.f;
  if constexpr (Q == 7)  // -Dz^T Dz
    return (e.z_lo ? -(x - X(-1, 0, 0)) : 0.f) + (e.z_hi ? X(1, 0, 0) - x : 0.f);
  if constexpr (Q == 8)  // -Dz^T Dc
    return e.c_lo ? ((e.z_lo ? -(x - X(0, 0, -1)) : 0.f) +
                     (e.z_hi ? X(1, 0, 0) - X(1, 0, -1) : 0.f))
                  : 0.f;
  if constexpr (Q == 9)  // -Dz Dc^T
    return e.z_lo ? ((e.c_lo ? -(x - X(-1, 0, 0)) : 0.f) +
                     (e.c_hi ? X(0, 0, 1) - X(-1, 0, 1) : 0.f))
                  : 0.f;
  if constexpr (Q == 10)  // -Dz^T Dr
    return e.r_lo ? ((e.z_lo ? -(x - X(0, -1, 0)) : 0.f) +
                     (e.z_hi ? X(1, 0, 0) - X(1, -1, 0) : 0.f))
                  : 0.f;
  if constexpr (Q == 11)  // -Dz Dr^T
    return e.z_lo ? ((e.r_lo ? -(x - X(-1, 0, 0)) : 0.f) +
                     (e.r_hi ? X(0, 1, 0) - X(-1, 1, 0) : 0.f))
                  : 0.f;
  return 0.f;
}

template <class F>
__device__ __forceinline__ void all_comps(const F& X, const Edges& e, float (&u)[NF]) {
  u[0] = comp<0>(X, e);
  u[1] = comp<1>(X, e);
  u[2] = comp<2>(X, e);
  u[3] = comp<3>(X, e);
  u[4] = comp<4>(X, e);
  u[5] = comp<5>(X, e);
  u[6] = comp<6>(X, e);
  u[7] = comp<7>(X, e);
  u[8] = comp<8>(X, e);
  u[9] = comp<9>(X, e);
  u[10] = comp<10>(X, e);
  u[11] = comp<11>(X, e);
}

__device__ __forceinline__ void norms(const float (&u)[NF], float& n1, float& n2) {
  n1 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  n2 = 0.f;
#pragma unroll
  for (int q = 3; q < NF; ++q) n2 = fmaf(u[q], u[q], n2);
}

__global__ void __launch_bounds__(VT) k_stencil3d(Vol3Args a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Vol3Smem& S = *reinterpret_cast<Vol3Smem*>(smem_raw);
  if (a.bst != nullptr && a.bst->remaining == 0) return;  // uniform over the grid
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = a.n, nz = a.nz;
  const long long ps = a.ps, zs = a.zs;
  const float *fk, *fkm;
  if (a.bst != nullptr) {
    const int G = a.bst->gstep;
    fk = a.f[G % 3];
    fkm = a.f[(G + 2) % 3];
  } else {
    fk = a.f[0];
    fkm = nullptr;
  }
  for (int s = tid; s < MAXZ; s += VT) {
    S.reg_hi[s] = 0.f;
    S.reg_lo[s] = 0.f;
  }
  const int ntx = (n + VC - 1) / VC, nty = (n + VR - 1) / VR, ntz = (nz + VS - 1) / VS;
  const int items = ntx * nty * ntz;
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    const int tz = it % ntz, txy = it / ntz;
    const int z0 = tz * VS, r0 = (txy / ntx) * VR, c0 = (txy % ntx) * VC;
    __syncthreads();  // the previous item's fields are no longer read
    // f~ = f^k + theta_z (f^k - f^{k-1}) and f^k on the tile with a 2-voxel halo
    for (int t = tid; t < HR * HC * HS; t += VT) {
      int iz, ic, ir;
      if (a.zs == 1) {  // slices adjacent in memory: slice fastest
        iz = t % HS;
        ic = (t / HS) % HC;
        ir = t / (HS * HC);
      } else {          // pixels of a row adjacent: column fastest
        ic = t % HC;
        iz = (t / HC) % HS;
        ir = t / (HC * HS);
      }
      const int z = z0 - 2 + iz, r = r0 - 2 + ir, c = c0 - 2 + ic;
      float vk = 0.f, vt = 0.f;
      if (z >= 0 && z < nz && r >= 0 && r < n && c >= 0 && c < n) {
        const long long o = (long long)(r * n + c) * ps + (long long)z * zs;
        vk = fk[o];
        vt = vk;
        if (fkm != nullptr) vt = fmaf(a.slots[z].theta_hi, vk - fkm[o], vk);
      }
      S.T[ir][ic][iz] = vt;
      S.K[ir][ic][iz] = vk;
    }
    __syncthreads();
    // grad phi~(B f~) on the tile and a 1-voxel ring around it
    for (int t = tid; t < WR * WC * WS; t += VT) {
      const int iz = t % WS, ic = (t / WS) % WC, ir = t / (WS * WC);
      const int z = z0 - 1 + iz, r = r0 - 1 + ir, c = c0 - 1 + ic;
      float v[NF];
#pragma unroll
      for (int q = 0; q < NF; ++q) v[q] = 0.f;
      if (z >= 0 && z < nz && r >= 0 && r < n && c >= 0 && c < n) {
        const Edges e = edges(z, r, c, nz, n);
        auto X = [&](int dz, int dr, int dc) { return S.T[ir + 1 + dr][ic + 1 + dc][iz + 1 + dz]; };
        all_comps(X, e, v);
        float n1, n2;
        norms(v, n1, n2);
        const float lam1 = a.slots ? a.slots[z].lambda1 : a.lam1;
        const float lam2 = a.slots ? a.slots[z].lambda2 : a.lam2;
        const float eps = a.slots ? a.slots[z].eps : a.eps;
        const float s1 = lam1 / fmaxf(sqrtf(n1), eps);
        const float s2 = lam2 / fmaxf(sqrtf(n2), eps);
#pragma unroll
        for (int q = 0; q < 3; ++q) v[q] *= s1;
#pragma unroll
        for (int q = 3; q < NF; ++q) v[q] *= s2;
      }
#pragma unroll
      for (int q = 0; q < NF; ++q) S.W[q][ir][ic][iz] = v[q];
    }
    __syncthreads();
    // B^T applied to the fields at the tile voxels: D^T for the first-order
    // fields; each second-order block's transpose is the block of the same
    // form (symmetric ones) or of its partner (4 <-> 6, 8 <-> 9, 10 <-> 11)
    const int col = tid % VC, zq = tid / VC;
    const int z = z0 + zq, c = c0 + col;
    float reg = 0.f;
    if (z < nz && c < n) {
#pragma unroll
      for (int ii = 0; ii < VR; ++ii) {
        const int r = r0 + ii;
        if (r >= n) continue;
        const Edges e = edges(z, r, c, nz, n);
        const int wr = ii + 1, wc = col + 1, wz = zq + 1;
        auto Wf = [&](int q) {
          return [&, q](int dz, int dr, int dc) { return S.W[q][wr + dr][wc + dc][wz + dz]; };
        };
        float g = 0.f;
        if (e.c_lo) g += S.W[0][wr][wc][wz];
        if (e.c_hi) g -= S.W[0][wr][wc + 1][wz];
        if (e.r_lo) g += S.W[1][wr][wc][wz];
        if (e.r_hi) g -= S.W[1][wr + 1][wc][wz];
        if (e.z_lo) g += S.W[2][wr][wc][wz];
        if (e.z_hi) g -= S.W[2][wr][wc][wz + 1];
        g += comp<3>(Wf(3), e);
        g += comp<6>(Wf(4), e);
        g += comp<5>(Wf(5), e);
        g += comp<4>(Wf(6), e);
        g += comp<7>(Wf(7), e);
        g += comp<9>(Wf(8), e);
        g += comp<8>(Wf(9), e);
        g += comp<11>(Wf(10), e);
        g += comp<10>(Wf(11), e);
        a.gR[(long long)(r * n + c) * ps + (long long)z * zs] = g;
        if (a.want_reg) {
          auto Xk = [&](int dz, int dr, int dc) {
            return S.K[ii + 2 + dr][col + 2 + dc][zq + 2 + dz];
          };
          float u[NF];
          all_comps(Xk, e, u);
          float n1, n2;
          norms(u, n1, n2);
          const float lam1 = a.slots ? a.slots[z].lambda1 : a.lam1;
          const float lam2 = a.slots ? a.slots[z].lambda2 : a.lam2;
          const float eps = a.slots ? a.slots[z].eps : a.eps;
          reg += lam1 * s_eps_f(n1, eps) + lam2 * s_eps_f(n2, eps);
        }
      }
    }
    if (a.want_reg) {
      // warp zq holds slice z0 + zq: fold its 32 columns in a fixed order
      float h = reg, l = 0.f;
      warp_sum_acc(h, l);
      if (lane == 0 && z0 + warp < nz) acc_add(S.reg_hi[z0 + warp], S.reg_lo[z0 + warp], h, l);
    }
  }
  if (!a.want_reg) return;
  __syncthreads();
  for (int s = tid; s < a.pstride; s += VT)
    a.partial[(long long)blockIdx.x * a.pstride + s] =
        s < MAXZ ? make_float2(S.reg_hi[s], S.reg_lo[s]) : make_float2(0.f, 0.f);
}

// out = sum of rows x cols double-float pairs (row stride pstride), one block,
// fixed order
__global__ void __launch_bounds__(256) k_sum_pairs(const float2* __restrict__ p, int rows,
                                                   int cols, int pstride, double* out) {
  float h = 0.f, l = 0.f;
  const int total = rows * cols;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const float2 v = p[(long long)(i / cols) * pstride + i % cols];
    acc_add(h, l, v.x, v.y);
  }
  const df s = block_sum_acc(h, l);
  if (threadIdx.x == 0) *out = (double)s.hi + (double)s.lo;
}

int sm_count_vol() {
  static const int sms = [] {
    int dev = 0, s = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
    return s > 0 ? s : 1;
  }();
  return sms;
}

}  // namespace

int stencil3d_max_slices() { return MAXZ; }

int stencil3d_grid(int n, int nz) {
  const int items = ((n + VC - 1) / VC) * ((n + VR - 1) / VR) * ((nz + VS - 1) / VS);
  const int cap = 2 * sm_count_vol();
  return items < cap ? items : cap;
}

cudaError_t launch_stencil3d(const Vol3Args& a, cudaStream_t s) {
  if (a.nz < 1 || a.nz > MAXZ || a.n < 1) return cudaErrorInvalidValue;
  static cudaError_t attr = cudaFuncSetAttribute(
      k_stencil3d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Vol3Smem));
  if (attr != cudaSuccess) return attr;
  k_stencil3d<<<stencil3d_grid(a.n, a.nz), VT, sizeof(Vol3Smem), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sum_pairs(const float2* p, int rows, int cols, int pstride, double* out,
                             cudaStream_t s) {
  k_sum_pairs<<<1, 256, 0, s>>>(p, rows, cols, pstride, out);
  return cudaGetLastError();
}

}  // namespace appga
