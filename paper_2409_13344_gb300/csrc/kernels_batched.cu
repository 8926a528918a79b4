// Batched CUDA kernels: K independent slices (slots) that share one system
// matrix run the APPGA iteration together, so every nonzero of A and A^T is
// read once per iteration for all K right-hand sides (CSR SpMM).
//
// Layout (slot-minor): images f[j][s], sinograms y[i][s], w[i][s], g[i][s]
// with K padded to Kp = 32 V (V = 1, 2 or 4 slots per lane).  One warp owns
// a CSR row: lanes load 32 (column, value) pairs at a time and stage them in
// shared memory; every lane reads them back with broadcast loads and, for
// each nonzero, gathers its 4V-byte piece of the Kp-wide image row (one
// coalesced row per warp) and accumulates V products in FP32.  The
// back-projection's blocks own contiguous runs of pixels, whose rays overlap,
// so the gathered weight rows are reused from L1; the forward projection
// deals rays to the warps of the whole grid in turn, so the grid works on
// neighbouring rays at once and the image rows they gather stay in L2 (each
// order is a per-projection switch).  The per-(row, slot) epilogues match the
// single-slice kernels (Eq. APPGAiter, Eq. EM, Sec. 2.2); the SHOITV stencil
// runs on shared-memory tiles of 2 x 32 pixels x 8 slots.
//
// Every slot carries its own device state (iteration index, momentum scalar,
// objective, stop flag, parameters), so slots may sit at different
// iterations (continuous batching).  The iterate rings are indexed by a
// global step counter shared by all slots.  Per-slot objective sums use the
// deterministic two-level grid reduction, so results do not depend on which
// other slots are in the batch.
#include <cuda_runtime.h>
#include <math.h>

#include "appga_internal.h"
#include "batched_internal.h"
#include "device_common.cuh"

namespace appga {
namespace {

constexpr int B_THREADS = 256;
constexpr int B_WARPS = B_THREADS / 32;
constexpr int MAXK = 128;                    // largest padded batch (V = 4)
// Default grids: more blocks than fit at once (measured faster on GB300 than
// grids that are all resident: blocks own contiguous row ranges, and the
// block scheduler balances the tail).
constexpr int kSpmvPerSm = 8;                // SpMV / back-projection blocks per SM
constexpr int kStencilPerSm = 4;             // stencil blocks per SM
constexpr int kMaxPerSm = 16;                // upper bound of either tuned value
__host__ __forceinline__ int clamp_per_sm(int v, int dflt) {
  return v <= 0 ? dflt : (v > kMaxPerSm ? kMaxPerSm : v);
}
// Blocks per SM when no tuned schedule is given: at 64 slots the
// autotuner's choice on 64 slices of 256^2 (forward 4, pixel 5, stencil 8),
// other widths the caps above.
__host__ __forceinline__ int default_spmv_per_sm(int Kp) { return Kp == 64 ? 4 : kSpmvPerSm; }
__host__ __forceinline__ int default_pixel_per_sm(int Kp) { return Kp == 64 ? 5 : kSpmvPerSm; }
__host__ __forceinline__ int default_stencil_per_sm(int Kp) {
  return Kp == 64 ? 8 : kStencilPerSm;
}
constexpr int BST_R = 2, BST_C = 32, BST_S = 8;  // stencil item: 2 x 32 pixels x 8 slots
constexpr int BTW = BST_C + 4, BVW = BST_C + 2;
static_assert(BST_C * BST_S == B_THREADS, "stencil: one thread per (column, slot)");

template <int V>
__device__ __forceinline__ void vload(const float* p, float (&x)[V]) {
  if constexpr (V == 1) {
    x[0] = __ldg(p);
  } else if constexpr (V == 2) {
    const float2 t = __ldg(reinterpret_cast<const float2*>(p));
    x[0] = t.x;
    x[1] = t.y;
  } else {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    x[0] = t.x;
    x[1] = t.y;
    x[2] = t.z;
    x[3] = t.w;
  }
}
template <int V>
__device__ __forceinline__ void vstore(float* p, const float (&x)[V]) {
  if constexpr (V == 1) {
    p[0] = x[0];
  } else if constexpr (V == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(x[0], x[1]);
  } else {
    *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
  }
}

#ifndef APPGA_BDOT
#define APPGA_BDOT 2
#endif
// Row order of each projection: a contiguous run of rows per block (1) or
// rows dealt to the warps of the whole grid in turn (0).  The forward
// projection gathers image rows faster dealt in turn (the whole grid works
// on neighbouring rays at once, so the rows it gathers stay in L2); the
// back-projection keeps contiguous runs of pixels (their weight rows are
// reused from L1).
#ifndef APPGA_BCONTIG_FW
#define APPGA_BCONTIG_FW 0
#endif
#ifndef APPGA_BCONTIG_PX
#define APPGA_BCONTIG_PX 1
#endif

// One CSR row of M times the Kp-wide columns of X ([cols][Kp]): lane holds
// the V sums of slots lane*V .. lane*V + V - 1.  Each lane loads one of 32
// (column, value) pairs; the warp stages them in shared memory (the column
// as an element offset col * Kp) and every lane reads them back four at a
// time with broadcast loads, gathering GR image rows per step (8 or 4: more
// loads in flight against fewer registers; a launch-schedule choice).  The
// next 32 pairs are loaded while the current ones are consumed.  Products
// are accumulated in the row's entry order whatever GR, so the sums do not
// depend on it.
template <int V, bool BF16, int GR = 8>
__device__ __forceinline__ void brow_dot(const DevCSR& M, int row, const float* __restrict__ X,
                                         int Kp, int lane, bool lane_on, uint64_t pol,
                                         int* s_off, float* s_val, float (&acc)[V]) {
#if APPGA_BDOT == 2
#pragma unroll
  for (int t = 0; t < V; ++t) acc[t] = 0.f;
  const int s = __ldg(M.row_ptr + row), e = __ldg(M.row_ptr + row + 1);
  const float* xl = X + lane * V;
  int c = 0;
  float v = 0.f;
  if (s + lane < e) {
    c = ld_stream_i1(M.col + s + lane, pol);
    v = BF16 ? ld_stream_bf16_1(M.val_bf16 + s + lane, pol) : ld_stream_f1(M.val + s + lane, pol);
  }
  for (int p0 = s; p0 < e; p0 += 32) {
    const int cnt = min(32, e - p0);  // a multiple of 4 (rows are padded)
    __syncwarp();
    s_off[lane] = c * Kp;
    s_val[lane] = v;
    __syncwarp();
    const int pn = p0 + 32 + lane;
    if (pn < e) {
      c = ld_stream_i1(M.col + pn, pol);
      v = BF16 ? ld_stream_bf16_1(M.val_bf16 + pn, pol) : ld_stream_f1(M.val + pn, pol);
    }
    if (!lane_on) continue;
    int q = 0;
    if constexpr (GR == 8) {
      for (; q + 8 <= cnt; q += 8) {
        const int4 o0 = *reinterpret_cast<const int4*>(s_off + q);
        const int4 o1 = *reinterpret_cast<const int4*>(s_off + q + 4);
        const float4 w0 = *reinterpret_cast<const float4*>(s_val + q);
        const float4 w1 = *reinterpret_cast<const float4*>(s_val + q + 4);
        float x[8][V];
        vload<V>(xl + o0.x, x[0]);
        vload<V>(xl + o0.y, x[1]);
        vload<V>(xl + o0.z, x[2]);
        vload<V>(xl + o0.w, x[3]);
        vload<V>(xl + o1.x, x[4]);
        vload<V>(xl + o1.y, x[5]);
        vload<V>(xl + o1.z, x[6]);
        vload<V>(xl + o1.w, x[7]);
        const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int t = 0; t < V; ++t) acc[t] = fmaf(w[u], x[u][t], acc[t]);
      }
    }
    static_assert(GR == 8 || GR == 4, "image rows gathered per step");
    for (; q < cnt; q += 4) {  // cnt is a multiple of 4 (rows are padded)
      const int4 o0 = *reinterpret_cast<const int4*>(s_off + q);
      const float4 w0 = *reinterpret_cast<const float4*>(s_val + q);
      float x[4][V];
      vload<V>(xl + o0.x, x[0]);
      vload<V>(xl + o0.y, x[1]);
      vload<V>(xl + o0.z, x[2]);
      vload<V>(xl + o0.w, x[3]);
      const float w[4] = {w0.x, w0.y, w0.z, w0.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int t = 0; t < V; ++t) acc[t] = fmaf(w[u], x[u][t], acc[t]);
    }
  }
#else
  (void)s_off;
  (void)s_val;
#pragma unroll
  for (int t = 0; t < V; ++t) acc[t] = 0.f;
  const int s = __ldg(M.row_ptr + row), e = __ldg(M.row_ptr + row + 1);
  const float* xl = X + lane * V;
  for (int p0 = s; p0 < e; p0 += 32) {
    const int p = p0 + lane;
    int c = 0;
    float v = 0.f;
    if (p < e) {
      c = ld_stream_i1(M.col + p, pol);
      v = BF16 ? ld_stream_bf16_1(M.val_bf16 + p, pol) : ld_stream_f1(M.val + p, pol);
    }
    const int cnt = min(32, e - p0);  // a multiple of 4 (rows are padded)
    for (int q = 0; q < cnt; q += 4) {
      int cq[4];
      float vq[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        cq[u] = __shfl_sync(0xffffffffu, c, q + u);
        vq[u] = __shfl_sync(0xffffffffu, v, q + u);
      }
      float x[4][V];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (lane_on) {
          vload<V>(xl + (size_t)cq[u] * Kp, x[u]);
        } else {
#pragma unroll
          for (int t = 0; t < V; ++t) x[u][t] = 0.f;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int t = 0; t < V; ++t) acc[t] = fmaf(vq[u], x[u][t], acc[t]);
    }
  }
#endif
}

// ------------------------------------------------- per-slot grid reduction
// Two-level deterministic reduction of Kp double-float values per block
// (p_hi/p_lo in shared memory).  True in the final block, where tot_hi /
// tot_lo (shared) hold the per-slot totals.  Partial layout: block b at
// partial[b*Kp .. ), group g result at partial[(nb + g)*Kp .. ).
__device__ bool grid_reduce_slots(float2* partial, unsigned int* gtick, unsigned int* ftick,
                                  const float* p_hi, const float* p_lo, int Kp, float* tot_hi,
                                  float* tot_lo) {
  __shared__ int s_flag;
  __shared__ float r_hi[B_THREADS], r_lo[B_THREADS];
  const int nb = gridDim.x, b = blockIdx.x, g = b / RED_GROUP, tid = threadIdx.x;
  const int ngroups = (nb + RED_GROUP - 1) / RED_GROUP;
  const int gsize = min(RED_GROUP, nb - g * RED_GROUP);
  for (int s = tid; s < Kp; s += blockDim.x) partial[(size_t)b * Kp + s] = make_float2(p_hi[s], p_lo[s]);
  __threadfence();
  __syncthreads();
  if (tid == 0) s_flag = (atomicAdd(&gtick[g], 1u) == (unsigned)(gsize - 1));
  __syncthreads();
  if (!s_flag) return false;
  __threadfence();
  const int P = blockDim.x / Kp;  // parts per slot
  auto reduce_rows = [&](const float2* base, int count) {
    const int s = tid % Kp, part = tid / Kp;
    float h = 0.f, l = 0.f;
    if (part < P) {
      for (int i = part; i < count; i += P) {
        const float2 v = __ldcg(base + (size_t)i * Kp + s);
        acc_add(h, l, v.x, v.y);
      }
    }
    r_hi[tid] = h;
    r_lo[tid] = l;
    __syncthreads();
    if (tid < Kp) {
      float hh = 0.f, ll = 0.f;
      for (int q = 0; q < P; ++q) acc_add(hh, ll, r_hi[q * Kp + tid], r_lo[q * Kp + tid]);
      tot_hi[tid] = hh;
      tot_lo[tid] = ll;
    }
    __syncthreads();
  };
  reduce_rows(partial + (size_t)g * RED_GROUP * Kp, gsize);
  for (int s = tid; s < Kp; s += blockDim.x)
    partial[(size_t)(nb + g) * Kp + s] = make_float2(tot_hi[s], tot_lo[s]);
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    gtick[g] = 0;
    s_flag = (atomicAdd(ftick, 1u) == (unsigned)(ngroups - 1));
  }
  __syncthreads();
  if (!s_flag) return false;
  __threadfence();
  reduce_rows(partial + (size_t)nb * Kp, ngroups);
  if (tid == 0) *ftick = 0;
  return true;
}

// --------------------------------------------------------------- stencil

struct BStencilSmem {
  float T[BST_R + 4][BTW][BST_S];
  float K[BST_R + 4][BTW][BST_S];
  float V[6][BST_R + 2][BVW][BST_S];
};

// One stencil item: tile (r0, c0) for slots s0 .. s0+7.  Thread (col, q) =
// (tid % 32, tid / 32).  Writes gR and returns this thread's regulariser
// share of Phi(f^k) for slot s0 + q (both tile rows).
__device__ float bstencil_item(BStencilSmem& S, const float* __restrict__ fk,
                               const float* __restrict__ fkm, const SlotState* slots, int Kp,
                               int r0, int c0, int s0, int n, float* __restrict__ gR,
                               bool want_reg, int mode) {
  const int tid = threadIdx.x;
  // load the halo tile, slots fastest (32-byte runs)
  for (int t = tid; t < (BST_R + 4) * BTW * BST_S; t += blockDim.x) {
    const int q = t % BST_S, pix = t / BST_S;
    const int ii = pix / BTW, jj = pix % BTW;
    const int r = r0 - 2 + ii, c = c0 - 2 + jj;
    float vk = 0.f, vt = 0.f;
    if (r >= 0 && r < n && c >= 0 && c < n) {
      const size_t o = (size_t)(r * n + c) * Kp + s0 + q;
      vk = fk[o];
      vt = mode == 2 ? vk : fmaf(slots[s0 + q].theta_hi, vk - fkm[o], vk);
    }
    S.K[ii][jj][q] = vk;
    S.T[ii][jj][q] = vt;
  }
  __syncthreads();
  for (int t = tid; t < (BST_R + 2) * BVW * BST_S; t += blockDim.x) {
    const int q = t % BST_S, pix = t / BST_S;
    const int ii = pix / BVW, jj = pix % BVW;
    const int r = r0 - 1 + ii, c = c0 - 1 + jj;
    float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (r >= 0 && r < n && c >= 0 && c < n) {
      const SlotState& sl = slots[s0 + q];
      // the six fields of B at (r, c) of slot s0 + q (same forms as the single-slice stencil)
      const int i = ii + 1, j = jj + 1;
      const bool r_lo = r >= 1, r_hi = r <= n - 2, c_lo = c >= 1, c_hi = c <= n - 2;
      auto X = [&](int a, int b) { return S.T[a][b][q]; };
      float u[6];
      u[0] = c_lo ? X(i, j) - X(i, j - 1) : 0.f;
      u[1] = r_lo ? X(i, j) - X(i - 1, j) : 0.f;
      u[2] = (c_lo ? -(X(i, j) - X(i, j - 1)) : 0.f) + (c_hi ? X(i, j + 1) - X(i, j) : 0.f);
      u[3] = c_lo ? ((r_lo ? -(X(i, j) - X(i, j - 1)) : 0.f) +
                     (r_hi ? X(i + 1, j) - X(i + 1, j - 1) : 0.f))
                  : 0.f;
      u[4] = (r_lo ? -(X(i, j) - X(i - 1, j)) : 0.f) + (r_hi ? X(i + 1, j) - X(i, j) : 0.f);
      u[5] = r_lo ? ((c_lo ? -(X(i, j) - X(i - 1, j)) : 0.f) +
                     (c_hi ? X(i, j + 1) - X(i - 1, j + 1) : 0.f))
                  : 0.f;
      const float n1 = u[0] * u[0] + u[1] * u[1];
      const float n2 = u[2] * u[2] + u[3] * u[3] + u[4] * u[4] + u[5] * u[5];
      const float s1 = sl.lambda1 / fmaxf(sqrtf(n1), sl.eps);
      const float s2 = sl.lambda2 / fmaxf(sqrtf(n2), sl.eps);
      v[0] = s1 * u[0];
      v[1] = s1 * u[1];
      v[2] = s2 * u[2];
      v[3] = s2 * u[3];
      v[4] = s2 * u[4];
      v[5] = s2 * u[5];
    }
#pragma unroll
    for (int f = 0; f < 6; ++f) S.V[f][ii][jj][q] = v[f];
  }
  __syncthreads();
  const int col = tid % BST_C, q = tid / BST_C;
  const SlotState& sl = slots[s0 + q];
  const bool part = mode == 2 ? sl.fresh : (sl.active && !sl.done);
  float reg = 0.f;
#pragma unroll
  for (int ii = 0; ii < BST_R; ++ii) {
    const int r = r0 + ii, c = c0 + col;
    if (part && r < n && c < n) {
      const int i = ii + 1, j = col + 1;
      const bool r_lo = r >= 1, r_hi = r <= n - 2, c_lo = c >= 1, c_hi = c <= n - 2;
      auto W = [&](int f, int a, int b) { return S.V[f][a][b][q]; };
      float gsum = 0.f;
      if (c_lo) gsum += W(0, i, j);
      if (c_hi) gsum -= W(0, i, j + 1);
      if (r_lo) gsum += W(1, i, j);
      if (r_hi) gsum -= W(1, i + 1, j);
      // u3-form of v3, u6-form of v4, u5-form of v5, u4-form of v6
      gsum += (c_lo ? -(W(2, i, j) - W(2, i, j - 1)) : 0.f) + (c_hi ? W(2, i, j + 1) - W(2, i, j) : 0.f);
      gsum += r_lo ? ((c_lo ? -(W(3, i, j) - W(3, i - 1, j)) : 0.f) +
                      (c_hi ? W(3, i, j + 1) - W(3, i - 1, j + 1) : 0.f))
                   : 0.f;
      gsum += (r_lo ? -(W(4, i, j) - W(4, i - 1, j)) : 0.f) + (r_hi ? W(4, i + 1, j) - W(4, i, j) : 0.f);
      gsum += c_lo ? ((r_lo ? -(W(5, i, j) - W(5, i, j - 1)) : 0.f) +
                      (r_hi ? W(5, i + 1, j) - W(5, i + 1, j - 1) : 0.f))
                   : 0.f;
      gR[(size_t)(r * n + c) * Kp + s0 + q] = gsum;
      if (want_reg) {
        auto Kf = [&](int a, int b) { return S.K[a][b][q]; };
        const int a = ii + 2, b = col + 2;
        float u[6];
        u[0] = c_lo ? Kf(a, b) - Kf(a, b - 1) : 0.f;
        u[1] = r_lo ? Kf(a, b) - Kf(a - 1, b) : 0.f;
        u[2] = (c_lo ? -(Kf(a, b) - Kf(a, b - 1)) : 0.f) + (c_hi ? Kf(a, b + 1) - Kf(a, b) : 0.f);
        u[3] = c_lo ? ((r_lo ? -(Kf(a, b) - Kf(a, b - 1)) : 0.f) +
                       (r_hi ? Kf(a + 1, b) - Kf(a + 1, b - 1) : 0.f))
                    : 0.f;
        u[4] = (r_lo ? -(Kf(a, b) - Kf(a - 1, b)) : 0.f) + (r_hi ? Kf(a + 1, b) - Kf(a, b) : 0.f);
        u[5] = r_lo ? ((c_lo ? -(Kf(a, b) - Kf(a - 1, b)) : 0.f) +
                       (c_hi ? Kf(a, b + 1) - Kf(a - 1, b + 1) : 0.f))
                    : 0.f;
        const float n1 = u[0] * u[0] + u[1] * u[1];
        const float n2 = u[2] * u[2] + u[3] * u[3] + u[4] * u[4] + u[5] * u[5];
        reg += sl.lambda1 * s_eps_f(n1, sl.eps) + sl.lambda2 * s_eps_f(n2, sl.eps);
      }
    }
  }
  __syncthreads();  // the tile buffers are reused by the next item
  return reg;
}

__device__ double bgn_t(int k, double a, double b, double omega) {
  return a * pow((double)k, omega) + b;
}
__device__ void bset_theta(SlotState& s, double theta) {
  s.theta = theta;
  const float h = (float)theta;
  s.theta_hi = h;
  s.theta_lo = (float)(theta - (double)h);
}

// -------------------------------------------------------------- k_bforward

// Shared memory of the forward phase: the per-slot objective partials of the
// block, and with stencil blocks in the grid the stencil tiles.  A launch
// without stencil blocks (the first projection, volume mode) leaves out the
// stencil's ~40 KB, so more blocks fit per SM and more of the unified L1
// serves the gathers of image rows.
struct BFwdEpi {
  float dhi[B_WARPS][MAXK];
  float dlo[B_WARPS][MAXK];
};
template <bool ST>
struct BFwdSmem {
  BFwdEpi e;
};
template <>
struct BFwdSmem<true> {
  union {
    BFwdEpi e;
    BStencilSmem st;
  };
};

// ST false: SpMV blocks only (grid n_spmv_blocks); ST true: the SpMV blocks
// followed by the stencil blocks in one grid, so the stencil blocks fill the
// SMs as the SpMV blocks finish.
template <int V, bool BF16, bool ST, int GR>
__global__ void __launch_bounds__(B_THREADS) k_bforward(BFwdArgs a) {
  __shared__ __align__(16) int s_off[B_WARPS][32];
  __shared__ __align__(16) float s_val[B_WARPS][32];
  __shared__ BFwdSmem<ST> sm;
  BatchState* bs = a.bst;
  if (a.mode == 0 && bs->remaining == 0) return;  // uniform over the grid
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Kp = a.Kp, n = a.n;
  const int G = bs->gstep;
  const bool proj_only = a.mode == 1;
  const float* f = proj_only ? a.f[(G + 2) % 3] : a.f[G % 3];
  float* y_out = proj_only ? a.y[(G + 1) & 1] : a.y[G & 1];
  const float* y_prev = a.y[(G + 1) & 1];
  const bool want = !proj_only && a.track;
  // which of this lane's slots take part: every slot (projection), the live
  // slots (step), or the fresh slots (admission, where f^{k-1} = f^k so the
  // extrapolated projection is y itself)
  int on[V];
  float th_h[V];
  bool lane_on = false;
#pragma unroll
  for (int t = 0; t < V; ++t) {
    const SlotState& sl = a.slots[lane * V + t];
    on[t] = proj_only ? 1 : (a.mode == 2 ? sl.fresh : (sl.active && !sl.done));
    th_h[t] = a.mode == 2 ? 0.f : sl.theta_hi;
    lane_on = lane_on || on[t];
  }
  float dh[V], dl[V];
  int hits[V];
#pragma unroll
  for (int t = 0; t < V; ++t) {
    dh[t] = 0.f;
    dl[t] = 0.f;
    hits[t] = 0;
  }
  if (!ST || (int)blockIdx.x < a.n_spmv_blocks) {
    const uint64_t pol = evict_first_policy();
#if APPGA_BCONTIG_FW
    // each block owns a contiguous run of rows (neighbouring rays share
    // pixels, so the gathered image rows are reused from L1)
    const int per = (a.A.rows + a.n_spmv_blocks - 1) / a.n_spmv_blocks;
    const int r0 = blockIdx.x * per, r1 = min(a.A.rows, r0 + per);
    for (int row = r0 + warp; row < r1; row += B_WARPS) {
#else
    const int stride = a.n_spmv_blocks * B_WARPS;
    for (int row = blockIdx.x * B_WARPS + warp; row < a.A.rows; row += stride) {
#endif
      float acc[V];
      brow_dot<V, BF16, GR>(a.A, row, f, Kp, lane, lane_on, pol, s_off[warp], s_val[warp], acc);
      if (!lane_on) continue;
      const size_t o = (size_t)row * Kp + lane * V;
      float yp[V], gg[V], gm[V], yo[V], wo[V];
      vload<V>(y_out + o, yo);
      if (!proj_only) {
        vload<V>(y_prev + o, yp);
        vload<V>(a.g + o, gg);
        vload<V>(a.gamma + o, gm);
        vload<V>(a.w + o, wo);
      }
#pragma unroll
      for (int t = 0; t < V; ++t) {
        if (!on[t]) continue;
        yo[t] = acc[t];
        if (proj_only) continue;
        // y~ = y + theta (y - y_prev); den = max(y~ + gamma, kappa gamma); w = (den - g)/den
        const float yt = a.mode == 2 ? acc[t] : fmaf(th_h[t], acc[t] - yp[t], acc[t]);
        float den = yt + gm[t];
        const float fl = 1e-3f * gm[t];
        if (den < fl) {
          den = fl;
          ++hits[t];
        }
        wo[t] = __fdiv_rn(den - gg[t], den);
        if (want) {
          // data term y - g ln(y + gamma) in double-float
          df yg;
          two_sum(acc[t], gm[t], yg.hi, yg.lo);
          const df term = df_add_f(df_neg(df_mul_f(df_log(yg), gg[t])), acc[t]);
          acc_add(dh[t], dl[t], term.hi, term.lo);
        }
      }
      vstore<V>(y_out + o, yo);
      if (!proj_only) vstore<V>(a.w + o, wo);
    }
  } else if constexpr (ST) {
    if (!proj_only) {
      // stencil items: (tile, 8-slot chunk) pairs, persistent over the stencil blocks
      const int nsb = gridDim.x - a.n_spmv_blocks;
      const int ntx = (n + BST_C - 1) / BST_C, nty = (n + BST_R - 1) / BST_R;
      const int nchunks = Kp / BST_S;
      const int ntiles = ntx * nty;
      __shared__ float sreg_hi[MAXK], sreg_lo[MAXK];  // per-slot regulariser sums
      __shared__ int chunk_on[MAXK / BST_S];
      for (int s = tid; s < MAXK; s += blockDim.x) {
        sreg_hi[s] = 0.f;
        sreg_lo[s] = 0.f;
      }
      for (int c = tid; c < nchunks; c += blockDim.x) {
        int any = 0;
        for (int q = 0; q < BST_S; ++q) {
          const SlotState& sl = a.slots[c * BST_S + q];
          any |= a.mode == 2 ? sl.fresh : (sl.active && !sl.done);
        }
        chunk_on[c] = any;
      }
      __syncthreads();
      // Each block owns the same tiles for every slot chunk, so a slot's
      // regulariser sum is grouped the same way whatever its slot index.
      for (int tile = blockIdx.x - a.n_spmv_blocks; tile < ntiles; tile += nsb)
      for (int chunk = 0; chunk < nchunks; ++chunk) {
        if (!chunk_on[chunk]) continue;  // uniform over the block
        const int r0 = (tile / ntx) * BST_R, c0 = (tile % ntx) * BST_C;
        const float reg = bstencil_item(sm.st, f, a.f[(G + 2) % 3], a.slots, Kp, r0, c0,
                                        chunk * BST_S, n, a.gR, want, a.mode);
        if (want) {
          // warp q holds slot chunk*8 + q: fold the warp's 32 columns
          float h = reg, l = 0.f;
          warp_sum_acc(h, l);
          if (lane == 0) {
            const int s = chunk * BST_S + warp;
            acc_add(sreg_hi[s], sreg_lo[s], h, l);
          }
        }
      }
      __syncthreads();
      if (want && warp == 0) {
        // hand the per-slot sums to the lanes that own the slots in warp 0
  #pragma unroll
        for (int t = 0; t < V; ++t) {
          dh[t] = sreg_hi[lane * V + t];
          dl[t] = sreg_lo[lane * V + t];
        }
      }
    }
  }
  if (!proj_only) {
#pragma unroll
    for (int t = 0; t < V; ++t)
      if (hits[t]) atomicAdd(&a.slots[lane * V + t].guard_hits, (unsigned long long)hits[t]);
  }
  if (!want) return;
  // block partial per slot (fixed order over warps), left for the pixel
  // phase of this step; an admission pass writes only the fresh slots' columns
  __syncthreads();
#pragma unroll
  for (int t = 0; t < V; ++t) {
    sm.e.dhi[warp][lane * V + t] = dh[t];
    sm.e.dlo[warp][lane * V + t] = dl[t];
  }
  __syncthreads();
  for (int s = tid; s < Kp; s += blockDim.x) {
    const SlotState& sl = a.slots[s];
    if (a.mode == 2 ? !sl.fresh : !(sl.active && !sl.done)) continue;
    float h = 0.f, l = 0.f;
    for (int w = 0; w < B_WARPS; ++w) acc_add(h, l, sm.e.dhi[w][s], sm.e.dlo[w][s]);
    a.fpartial[(size_t)blockIdx.x * Kp + s] = make_float2(h, l);
  }
}

// --------------------------------------------------------------- k_bpixel

template <int V, bool BF16, int GR>
__global__ void __launch_bounds__(B_THREADS) k_bpixel(BPixArgs a) {
  __shared__ __align__(16) int s_off[B_WARPS][32];
  __shared__ __align__(16) float s_val[B_WARPS][32];
  __shared__ float r_hi[MAXK], r_lo[MAXK], t_hi[MAXK], t_lo[MAXK];
  BatchState* bs = a.bst;
  if (bs->remaining == 0) return;  // uniform over the grid
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Kp = a.Kp;
  const int G = bs->gstep;
  const float* fk = a.f[G % 3];
  const float* fkm = a.f[(G + 2) % 3];
  float* fn = a.f[(G + 1) % 3];
  // this lane's slot parameters
  float th[V], beta[V];
  int live[V], kk[V], frz[V], back[V];
#pragma unroll
  for (int t = 0; t < V; ++t) {
    const SlotState& sl = a.slots[lane * V + t];
    th[t] = sl.theta_hi;
    beta[t] = sl.beta;
    live[t] = sl.active && !sl.done;
    kk[t] = sl.k;
    frz[t] = sl.freeze_iter;
    back[t] = sl.rollback;
  }
  bool lane_live = false;
#pragma unroll
  for (int t = 0; t < V; ++t) lane_live = lane_live || live[t];
  const uint64_t pol = evict_first_policy();
  int bad = 0;
#if APPGA_BCONTIG_PX
  // each block owns a contiguous run of pixels (neighbouring pixels lie on
  // the same rays, so the gathered weight rows are reused from L1)
  const int per = (a.At.rows + gridDim.x - 1) / gridDim.x;
  const int j0 = blockIdx.x * per, j1 = min(a.At.rows, j0 + per);
  for (int j = j0 + warp; j < j1; j += B_WARPS) {
#else
  const int stride = gridDim.x * B_WARPS;
  for (int j = blockIdx.x * B_WARPS + warp; j < a.At.rows; j += stride) {
#endif
    float bp[V];
    brow_dot<V, BF16, GR>(a.At, j, a.w, Kp, lane, lane_live, pol, s_off[warp], s_val[warp], bp);
    const size_t o = (size_t)j * Kp + lane * V;
    float vk[V], vm[V], gr[V], out[V];
    vload<V>(fk + o, vk);
    vload<V>(fkm + o, vm);
    vload<V>(a.gR + o, gr);
    const float il = __ldg(a.inv_lambda + j);
#pragma unroll
    for (int t = 0; t < V; ++t) {
      if (!live[t]) {
        // finished or empty slot: carry the image (the previous entry when
        // the slot stopped one step back)
        out[t] = back[t] ? vm[t] : vk[t];
        continue;
      }
      const float ft = fmaf(th[t], vk[t] - vm[t], vk[t]);
      float pk = vk[t];
      if (frz[t] >= 0) {
        if (kk[t] == frz[t]) {
          a.pfreeze[o + t] = vk[t];
        } else if (kk[t] > frz[t]) {
          pk = a.pfreeze[o + t];
        }
      }
      const float p = beta[t] * pk * il;
      const float xv = __fmaf_rn(-p, bp[t] + gr[t], ft);
      if (!isfinite(xv)) bad = 1;
      out[t] = fmaxf(xv, 0.f);
    }
    vstore<V>(fn + o, out);
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&bs->flags, APPGA_FLAG_NONFINITE);
  // This block's share of every slot's Phi(f^k): forward partial rows
  // b, b + G, ... (fixed order).
  for (int s = tid; s < Kp; s += blockDim.x) {
    float h = 0.f, l = 0.f;
    if (a.track)
      for (int i = blockIdx.x; i < a.n_fpartial; i += gridDim.x) {
        const float2 v = a.fpartial[(size_t)i * Kp + s];
        acc_add(h, l, v.x, v.y);
      }
    r_hi[s] = h;
    r_lo[s] = l;
  }
  // Finalise the step in the last block: Phi and the stopping test of every
  // live slot, then its next index and momentum; the global step advances.
  __syncthreads();
  if (grid_reduce_slots(a.partial, a.gtick, &bs->ticket_p, r_hi, r_lo, Kp, t_hi, t_lo)) {
    __shared__ int s_rem[B_THREADS];
    __shared__ int s_jstop;
    if (a.joint) {
      // volume: the slices are one problem; its objective is the sum of the
      // slots' shares, summed in FP64 in slot order, and one test stops all
      if (tid == 0) {
        double tot = 0.0;
        int kk = -1, k0 = 0;
        double tol = 0.0;
        for (int s = 0; s < Kp; ++s) {
          const SlotState& sl = a.slots[s];
          if (!sl.active || sl.done) continue;
          tot += (double)t_hi[s] + (double)t_lo[s];
          kk = sl.k;
          k0 = sl.k0;
          tol = sl.rel_tol;
        }
        int stop = 0;
        if (kk >= 0 && a.track && bs->phi_tot_k != kk) {
          const double prev = bs->phi_tot_cur;
          const bool consecutive = bs->phi_tot_k == kk - 1;
          bs->phi_tot_prev = prev;
          bs->phi_tot_cur = tot;
          bs->phi_tot_k = kk;
          stop = tol > 0.0 && kk > k0 && consecutive && fabs(tot - prev) <= tol * fabs(prev);
        }
        s_jstop = stop;
      }
      __syncthreads();
    }
    int rem = 0;
    for (int s = tid; s < Kp; s += blockDim.x) {
      SlotState& sl = a.slots[s];
      sl.fresh = 0;
      if (!sl.active || sl.done) {
        sl.rollback = 0;  // its carry above used the previous entry
        continue;
      }
      if (a.track && sl.phi_k != sl.k) {
        const double phi = (double)t_hi[s] + (double)t_lo[s];
        const double prev = sl.phi_cur;
        const bool consecutive = sl.phi_k == sl.k - 1;
        sl.phi_prev = prev;
        sl.phi_cur = phi;
        sl.phi_k = sl.k;
        if (!a.joint && sl.rel_tol > 0.0 && sl.k > sl.k0 && consecutive &&
            fabs(phi - prev) <= sl.rel_tol * fabs(prev)) {
          // f^k is the result; the f^{k+1} written above is not used
          sl.done = 1;
          sl.result_k = sl.k;
          sl.stopped_early = 1;
          sl.rollback = 1;
          continue;
        }
      }
      if (a.joint && s_jstop) {
        // the volume's test fired: f^k of every slice is the result
        sl.done = 1;
        sl.result_k = sl.k;
        sl.stopped_early = 1;
        sl.rollback = 1;
        continue;
      }
      if (sl.k >= sl.k_last) {
        sl.done = 1;
        sl.result_k = sl.k + 1;
      } else {
        ++rem;
      }
      const int k = sl.k;
      sl.k = k + 1;
      double th_next = 0.0;
      if (sl.momentum == APPGA_MOMENTUM_GN) {
        th_next = (bgn_t(k, sl.a, sl.b, sl.omega) - 1.0) / bgn_t(k + 1, sl.a, sl.b, sl.omega);
      } else if (sl.momentum == APPGA_MOMENTUM_NESTEROV) {
        const double t = sl.t_cur;
        const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        th_next = (t - 1.0) / tn;
        sl.t_cur = tn;
      }
      bset_theta(sl, th_next);
    }
    s_rem[tid] = rem;
    __syncthreads();
    if (tid == 0) {
      int tot = 0;
      for (int i = 0; i < (int)blockDim.x; ++i) tot += s_rem[i];
      bs->gstep = G + 1;
      bs->remaining = tot;
    }
  }
}

// ----------------------------------------------------------- setup kernels

// Slots marked rollback: copy the previous ring entry into the current one
// (the ring entries of the current global step, read on the device).
__global__ void k_resolve_rollback(const SlotState* slots, const BatchState* bs, float* f0,
                                   float* f1, float* f2, int len, int Kp) {
  const int s = blockIdx.y;
  if (!slots[s].rollback) return;  // uniform over the block
  float* ring[3] = {f0, f1, f2};
  const int G = bs->gstep;
  const float* prev = ring[(G + 2) % 3];
  float* cur = ring[G % 3];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x)
    cur[(size_t)i * Kp + s] = prev[(size_t)i * Kp + s];
}
__global__ void k_clear_rollback(SlotState* slots, int Kp) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < Kp) slots[s].rollback = 0;
}

// theta_{k0} of every slot, or of the fresh slots only (same device
// arithmetic as the step kernel).
__global__ void k_binit_momentum(SlotState* slots, int Kp, int only_fresh) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Kp) return;
  SlotState& sl = slots[s];
  if (only_fresh && !sl.fresh) return;
  double theta = 0.0, t = 1.0;
  if (sl.momentum == APPGA_MOMENTUM_GN) {
    theta = (bgn_t(sl.k - 1, sl.a, sl.b, sl.omega) - 1.0) / bgn_t(sl.k, sl.a, sl.b, sl.omega);
  } else if (sl.momentum == APPGA_MOMENTUM_NESTEROV) {
    for (int k = 1; k <= sl.k; ++k) {
      const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
      theta = (t - 1.0) / tn;
      t = tn;
    }
  }
  bset_theta(sl, theta);
  sl.t_cur = t;
}

// Slot of the k-th slice: ids[k] when a slot list is given, else s0 + k.
__device__ __forceinline__ int slot_of(const int* ids, int s0, int k) {
  return ids ? __ldg(ids + k) : s0 + k;
}

// [K][len] slice-major -> [len][Kp] slot-minor: out[i*Kp + slot(s)] = in[s*len + i].
// Padding slots are written separately.
__global__ void k_to_slot_minor(const float* __restrict__ in, int K, int len, float* __restrict__ out,
                                int Kp, int s0, const int* __restrict__ ids) {
  __shared__ float tile[32][33];
  const int i0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r, i = i0 + threadIdx.x;
    tile[r][threadIdx.x] = (k < K && i < len) ? in[(size_t)k * len + i] : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + r, k = k0 + threadIdx.x;
    if (i < len && k < K) out[(size_t)i * Kp + slot_of(ids, s0, k)] = tile[threadIdx.x][r];
  }
}
// out[s*len + i] = in[i*Kp + slot(s)] for s < K.
__global__ void k_from_slot_minor(const float* __restrict__ in, int K, int len, int Kp, int s0,
                                  const int* __restrict__ ids, float* __restrict__ out) {
  __shared__ float tile[32][33];
  const int i0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + r, k = k0 + threadIdx.x;
    tile[r][threadIdx.x] = (i < len && k < K) ? in[(size_t)i * Kp + slot_of(ids, s0, k)] : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r, i = i0 + threadIdx.x;
    if (k < K && i < len) out[(size_t)k * len + i] = tile[threadIdx.x][r];
  }
}
// Copies the listed columns of one [len][Kp] array into another.
__global__ void k_copy_slots(const float* __restrict__ src, float* __restrict__ dst, int len,
                             int Kp, const int* __restrict__ ids, int K) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)len * K;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t o = (t / K) * Kp + __ldg(ids + t % K);
    dst[o] = src[o];
  }
}
// Sets column s of a [len][Kp] array to v for s in [s0, s1).
__global__ void k_fill_slots(float* out, int len, int Kp, int s0, int s1, float v) {
  const int w = s1 - s0;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)len * w;
       t += (size_t)gridDim.x * blockDim.x)
    out[(t / w) * Kp + s0 + t % w] = v;
}

// Per-slot initial image TMC_s * 1_disk (Sec. 4.1) for the slots of K slices
// (s0 + k, or ids[k]) from slice-major g, gamma ([K][m]): one block per slice.
__global__ void __launch_bounds__(256) k_binit_image(const float* __restrict__ g,
                                                     const float* __restrict__ gamma, int m, int n,
                                                     int n_angles, long long npfov, int Kp, int s0,
                                                     const int* __restrict__ ids,
                                                     float* __restrict__ f_out) {
  const int k = blockIdx.x;
  const int slot = slot_of(ids, s0, k);
  float h = 0.f, l = 0.f;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    acc_add(h, l, g[(size_t)k * m + i], 0.f);
    acc_add(h, l, -gamma[(size_t)k * m + i], 0.f);
  }
  const df t = block_sum_acc(h, l);
  __shared__ float s_tmc;
  if (threadIdx.x == 0)
    s_tmc = (float)(((double)t.hi + (double)t.lo) / ((double)npfov * (double)n_angles));
  __syncthreads();
  const float v = s_tmc;
  for (int j = threadIdx.x; j < n * n; j += blockDim.x) {
    const int r = j / n, c = j % n;
    const long long dx = 2ll * c + 1 - n, dy = 2ll * r + 1 - n;
    f_out[(size_t)j * Kp + slot] = (dx * dx + dy * dy <= (long long)n * n) ? v : 0.f;
  }
}


int sm_count() { return current_sm_count(); }

int bforward_grid_n(const BFwdArgs& a, int* n_spmv) {
  const int sms = sm_count();
  int nsp = (a.A.rows + B_WARPS - 1) / B_WARPS;
  const int cap = sms * clamp_per_sm(a.spmv_per_sm, default_spmv_per_sm(a.Kp));
  if (nsp > cap) nsp = cap;
  int nst = 0;
  if (a.mode != 1 && !a.no_stencil) {
    // equal tile counts per stencil block
    const int tiles = ((a.n + BST_C - 1) / BST_C) * ((a.n + BST_R - 1) / BST_R);
    const int scap = sms * clamp_per_sm(a.stencil_per_sm, default_stencil_per_sm(a.Kp));
    const int per = (tiles + scap - 1) / scap;
    nst = (tiles + per - 1) / per;
  }
  if (n_spmv) *n_spmv = nsp;
  return nsp + nst;
}

// Gather probe: the batched projectors' inner loop alone.  Every row of M
// is reduced against the Kp-wide slot-minor rows of x by brow_dot, in the
// row order of the projection it stands for (contig: a contiguous run of
// rows per block, else rows dealt to the grid's warps in turn), with no
// epilogue, stencil or pixel update: the time of the column/value stream and
// the gathers by themselves.
template <int V>
__global__ void __launch_bounds__(B_THREADS) k_gather_probe(DevCSR M, const float* __restrict__ x,
                                                            int Kp, int contig,
                                                            float* __restrict__ sink) {
  __shared__ __align__(16) int s_off[B_WARPS][32];
  __shared__ __align__(16) float s_val[B_WARPS][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t pol = evict_first_policy();
  const int per = (M.rows + gridDim.x - 1) / gridDim.x;
  const int r0 = contig ? blockIdx.x * per : blockIdx.x * B_WARPS;
  const int r1 = contig ? min(M.rows, r0 + per) : M.rows;
  const int step = contig ? B_WARPS : gridDim.x * B_WARPS;
  float s = 0.f;
  for (int row = r0 + warp; row < r1; row += step) {
    float acc[V];
    brow_dot<V, false>(M, row, x, Kp, lane, true, pol, s_off[warp], s_val[warp], acc);
#pragma unroll
    for (int t = 0; t < V; ++t) s += acc[t];
  }
  if (s == 1.0e38f) sink[blockIdx.x] = s;  // keeps the loads; the value is never used
}

template <int V>
cudaError_t bforward_v(const BFwdArgs& a0, cudaStream_t s) {
  BFwdArgs a = a0;
  const int sms = sm_count();
  (void)sms;
  int nsp = 0;
  const int grid = bforward_grid_n(a, &nsp);
  a.n_spmv_blocks = nsp;
  const bool st = grid > nsp, g4 = a.gather_rows == 4;
  void (*kern)(BFwdArgs);
  if (a.use_bf16)
    kern = st ? (g4 ? k_bforward<V, true, true, 4> : k_bforward<V, true, true, 8>)
              : (g4 ? k_bforward<V, true, false, 4> : k_bforward<V, true, false, 8>);
  else
    kern = st ? (g4 ? k_bforward<V, false, true, 4> : k_bforward<V, false, true, 8>)
              : (g4 ? k_bforward<V, false, false, 4> : k_bforward<V, false, false, 8>);
  kern<<<grid, B_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}
template <int V>
cudaError_t bpixel_v(const BPixArgs& a, cudaStream_t s) {
  const int sms = sm_count();
  int nb = (a.At.rows + B_WARPS - 1) / B_WARPS;
  const int cap = sms * clamp_per_sm(a.blocks_per_sm, default_pixel_per_sm(a.Kp));
  if (nb > cap) nb = cap;
  const bool g4 = a.gather_rows == 4;
  void (*kern)(BPixArgs) = a.use_bf16 ? (g4 ? k_bpixel<V, true, 4> : k_bpixel<V, true, 8>)
                                      : (g4 ? k_bpixel<V, false, 4> : k_bpixel<V, false, 8>);
  kern<<<nb, B_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

// Largest grid of the batched kernels: at most kMaxPerSm SpMV and kMaxPerSm
// stencil blocks per SM (the launchers clamp the tuned values).
int batch_max_blocks() { return sm_count() * 2 * kMaxPerSm + 64; }

int bforward_grid(const BFwdArgs& a) { return bforward_grid_n(a, nullptr); }

cudaError_t launch_resolve_rollback(const BFwdArgs& a, cudaStream_t s) {
  const int len = a.n * a.n;
  dim3 grid((len + 255) / 256 < 64 ? (len + 255) / 256 : 64, a.Kp);
  k_resolve_rollback<<<grid, 256, 0, s>>>(a.slots, a.bst, a.f[0], a.f[1], a.f[2], len, a.Kp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // cleared by a second launch: every block above has read the mark first
  k_clear_rollback<<<(a.Kp + 127) / 128, 128, 0, s>>>(a.slots, a.Kp);
  return cudaGetLastError();
}

cudaError_t launch_bforward(const BFwdArgs& a, cudaStream_t s) {
  cudaError_t e = ensure_tables();
  if (e != cudaSuccess) return e;
  switch (a.Kp / 32) {
    case 1: return bforward_v<1>(a, s);
    case 2: return bforward_v<2>(a, s);
    case 4: return bforward_v<4>(a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_gather_probe(const DevCSR& M, bool forward, const float* x, int Kp,
                                float* sink, int blocks_per_sm, cudaStream_t s) {
  if (blocks_per_sm < 1 || blocks_per_sm > kMaxPerSm) return cudaErrorInvalidValue;
  const int grid = sm_count() * blocks_per_sm;
  const int contig = forward ? APPGA_BCONTIG_FW : APPGA_BCONTIG_PX;
  switch (Kp / 32) {
    case 1: k_gather_probe<1><<<grid, B_THREADS, 0, s>>>(M, x, Kp, contig, sink); break;
    case 2: k_gather_probe<2><<<grid, B_THREADS, 0, s>>>(M, x, Kp, contig, sink); break;
    case 4: k_gather_probe<4><<<grid, B_THREADS, 0, s>>>(M, x, Kp, contig, sink); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_bpixel(const BPixArgs& a, cudaStream_t s) {
  switch (a.Kp / 32) {
    case 1: return bpixel_v<1>(a, s);
    case 2: return bpixel_v<2>(a, s);
    case 4: return bpixel_v<4>(a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_binit_momentum(SlotState* slots, int Kp, bool only_fresh, cudaStream_t s) {
  k_binit_momentum<<<(Kp + 127) / 128, 128, 0, s>>>(slots, Kp, only_fresh ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_to_slot_minor(const float* in, int K, int len, float* out, int Kp, int s0,
                                 const int* ids, cudaStream_t s) {
  if (K <= 0) return cudaSuccess;
  dim3 grid((len + 31) / 32, (K + 31) / 32), block(32, 8);
  k_to_slot_minor<<<grid, block, 0, s>>>(in, K, len, out, Kp, s0, ids);
  return cudaGetLastError();
}

cudaError_t launch_from_slot_minor(const float* in, int K, int len, int Kp, int s0,
                                   const int* ids, float* out, cudaStream_t s) {
  if (K <= 0) return cudaSuccess;
  dim3 grid((len + 31) / 32, (K + 31) / 32), block(32, 8);
  k_from_slot_minor<<<grid, block, 0, s>>>(in, K, len, Kp, s0, ids, out);
  return cudaGetLastError();
}

cudaError_t launch_copy_slots(const float* src, float* dst, int len, int Kp, const int* ids,
                              int K, cudaStream_t s) {
  if (K <= 0) return cudaSuccess;
  k_copy_slots<<<256, 256, 0, s>>>(src, dst, len, Kp, ids, K);
  return cudaGetLastError();
}

cudaError_t launch_fill_slots(float* out, int len, int Kp, int s0, int s1, float v,
                              cudaStream_t s) {
  if (s1 <= s0) return cudaSuccess;
  k_fill_slots<<<256, 256, 0, s>>>(out, len, Kp, s0, s1, v);
  return cudaGetLastError();
}

cudaError_t launch_binit_image(const float* g, const float* gamma, int m, int n, int n_angles,
                               long long npfov, int K, int Kp, int s0, const int* ids,
                               float* f_out, cudaStream_t s) {
  if (K <= 0) return cudaSuccess;
  k_binit_image<<<K, 256, 0, s>>>(g, gamma, m, n, n_angles, npfov, Kp, s0, ids, f_out);
  return cudaGetLastError();
}

}  // namespace appga
