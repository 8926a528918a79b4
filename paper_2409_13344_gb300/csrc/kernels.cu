// Single-slice CUDA kernels of the APPGA hot path (sm_103a).
//
//   k_forward  : y = A f (double-float accumulation), y~ = y + theta (y - y_prev),
//                w = 1 - g / max(y~ + gamma, kappa gamma), FP64 data term
//                (steps a1, a2, a6-data; Sec. 2.2 grad F, Eq. FidelityTerm)
//   k_pixel    : f~ = f^k + theta (f^k - f^{k-1}); B^T grad phi~(B f~) by a
//                shared-memory halo-tiled stencil; A^T w through the
//                transposed CSR (no atomics); EM-preconditioned projected
//                update; FP64 regulariser term of Phi(f^k); momentum scalar
//                for the next iteration (steps a0, a3, a4, a5, a6-reg;
//                Eq. APPGAiter, Eq. EM, Eq. GNtheta)
//
// Both kernels read the iteration index and theta from a device-resident
// SolverState, so a captured graph of (k_pixel, k_forward) pairs replays
// without host involvement.  Block partial sums are combined by the last
// block to finish (ticket counter), in a fixed order, so every reduction is
// deterministic.
#include <cuda_runtime.h>
#include <math.h>

#include "appga_internal.h"

namespace appga {
namespace {

constexpr int THREADS = 256;
constexpr int WARPS = THREADS / 32;
constexpr int ROWS_PER_WARP = 8;   // forward: rows handled by one warp
constexpr int TILE_R = 2;          // pixel kernel tile: TILE_R x TILE_C pixels
constexpr int TILE_C = 32;
constexpr int PIX_PER_WARP = TILE_R * TILE_C / WARPS;  // 8
static_assert(PIX_PER_WARP <= 32, "one lane per pixel in the epilogue");

// ----------------------------------------------------------------- loads

// A and A^T are streamed once per iteration: bypass L1 and tag the lines
// evict-first in L2 (an L2 cache-policy operand) so the gathered vectors
// (f, w) stay cached.
__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ int4 ld_stream_i4(const int32_t* p, uint64_t pol) {
  int4 r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0,%1,%2,%3}, [%4], %5;"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
      : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ float4 ld_stream_f4(const float* p, uint64_t pol) {
  float4 r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
      : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
      : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ float4 ld_stream_bf16x4(const uint16_t* p, uint64_t pol) {
  uint2 u;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u32 {%0,%1}, [%2], %3;"
      : "=r"(u.x), "=r"(u.y)
      : "l"(p), "l"(pol));
  // BF16 -> FP32 is exact: the 16 bits are the high half of the float.
  float4 r;
  r.x = __uint_as_float(u.x << 16);
  r.y = __uint_as_float(u.x & 0xffff0000u);
  r.z = __uint_as_float(u.y << 16);
  r.w = __uint_as_float(u.y & 0xffff0000u);
  return r;
}

template <bool BF16>
__device__ __forceinline__ float4 ld_vals(const DevCSR& M, int p, uint64_t pol) {
  if constexpr (BF16) {
    return ld_stream_bf16x4(M.val_bf16 + p, pol);
  } else {
    return ld_stream_f4(M.val + p, pol);
  }
}

// ------------------------------------------------- double-float arithmetic
// Error-free transformations (Knuth TwoSum, FMA-based TwoProduct).  The
// explicit _rn intrinsics keep the compiler from contracting them.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (hi, lo) += a * x with the product and the sum error kept in lo.
__device__ __forceinline__ void df_fma(float& hi, float& lo, float a, float x) {
  const float p = __fmul_rn(a, x);
  const float pe = __fmaf_rn(a, x, -p);
  float s, e;
  two_sum(hi, p, s, e);
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(e, pe));
}
__device__ __forceinline__ void df_add(float& hi, float& lo, float h2, float l2) {
  float s, e;
  two_sum(hi, h2, s, e);
  hi = s;
  lo = __fadd_rn(__fadd_rn(lo, l2), e);
}
// Butterfly reductions: every lane ends with the same (bitwise) value.
__device__ __forceinline__ void warp_sum_df(float& hi, float& lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    df_add(hi, lo, h2, l2);
  }
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum of one double per thread (fixed tree).
__device__ double block_sum_d(double v) {
  __shared__ double red[WARPS];
  v = warp_sum_d(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < WARPS ? red[lane] : 0.0;
    t = warp_sum_d(t);
  }
  return t;  // valid in warp 0
}
__device__ int block_sum_i(int v) {
  __shared__ int redi[WARPS];
  v = warp_sum_i(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) redi[warp] = v;
  __syncthreads();
  int t = 0;
  if (warp == 0) {
    t = lane < WARPS ? redi[lane] : 0;
    t = warp_sum_i(t);
  }
  return t;
}

// Publishes this block's partial and returns true in the block that
// finishes last; that block then sums all partials in index order.
__device__ bool publish_and_check_last(double* partial, double mine, unsigned int* ticket) {
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    partial[blockIdx.y * gridDim.x + blockIdx.x] = mine;
    __threadfence();
    const unsigned int nb = gridDim.x * gridDim.y;
    const unsigned int t = atomicAdd(ticket, 1u);
    s_last = (t == nb - 1);
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last;
}
__device__ double sum_partials(const double* partial) {
  const int nb = gridDim.x * gridDim.y;
  double v = 0.0;
  for (int i = threadIdx.x; i < nb; i += THREADS) v += __ldcg(partial + i);
  return block_sum_d(v);
}

// ------------------------------------------------------------ projectors
//
// A warp owns R consecutive CSR rows, whose (row-padded) entries form one
// contiguous range.  It streams that range linearly in 128-entry chunks
// (one 4-entry pack per lane; row padding keeps every pack inside a single
// row), loading chunk t+1 while it gathers and accumulates chunk t.  Each
// lane accumulates into its current row and, when its row changes, parks the
// partial in a per-warp shared-memory slot [row][lane]; lane q then sums the
// 32 slots of row q in a fixed order.  No per-row shuffle reductions and no
// idle lanes on short rows; deterministic.

// Shared-memory slot row stride (33: the per-row sums read without bank conflicts).
constexpr int SLOT_W = 33;

// Row of entry p among rows q = 0..nrows-1 with starts bnd[0..nrows-1]
// (the last row starting at or before p; empty rows are skipped).
template <int R>
__device__ __forceinline__ int row_of(int p, const int (&bnd)[R + 1], int nrows) {
  int q = 0;
#pragma unroll
  for (int k = 1; k < R; ++k) q += (k < nrows && bnd[k] <= p) ? 1 : 0;
  return q;
}

template <int R>
__device__ __forceinline__ void load_bounds(const DevCSR& M, int row0, int nrows, int lane,
                                            int (&bnd)[R + 1]) {
  const int b = lane <= nrows ? M.row_ptr[row0 + lane] : 0;
#pragma unroll
  for (int k = 0; k <= R; ++k) bnd[k] = __shfl_sync(0xffffffffu, b, k <= nrows ? k : nrows);
}

// Double-float rows: returns row (lane) sums in lanes 0..nrows-1.
// slot_hi / slot_lo: this warp's R*32 floats each of shared memory.
template <bool BF16, int R>
__device__ __forceinline__ void warp_rows_dot_df(const DevCSR& M, int row0, int nrows,
                                                 const float* __restrict__ x, int lane,
                                                 float* slot_hi, float* slot_lo, float& out_hi,
                                                 float& out_lo) {
  out_hi = 0.f;
  out_lo = 0.f;
  if (nrows <= 0) return;
  int bnd[R + 1];
  load_bounds<R>(M, row0, nrows, lane, bnd);
#pragma unroll
  for (int q = 0; q < R; ++q) {
    slot_hi[q * SLOT_W + lane] = 0.f;
    slot_lo[q * SLOT_W + lane] = 0.f;
  }
  const uint64_t pol = evict_first_policy();
  const int P1 = bnd[nrows];
  int p = bnd[0] + lane * 4;
  int4 c = make_int4(0, 0, 0, 0);
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (p < P1) {
    c = ld_stream_i4(M.col + p, pol);
    v = ld_vals<BF16>(M, p, pol);
  }
  float hi = 0.f, lo = 0.f;
  int cur = -1;
  for (int base = bnd[0]; base < P1; base += 128, p += 128) {
    const int pn = p + 128;
    int4 cn = make_int4(0, 0, 0, 0);
    float4 vn = make_float4(0.f, 0.f, 0.f, 0.f);
    if (pn < P1) {
      cn = ld_stream_i4(M.col + pn, pol);
      vn = ld_vals<BF16>(M, pn, pol);
    }
    if (p < P1) {
      const int q = row_of<R>(p, bnd, nrows);
      if (q != cur) {
        if (cur >= 0) {
          slot_hi[cur * SLOT_W + lane] = hi;
          slot_lo[cur * SLOT_W + lane] = lo;
        }
        cur = q;
        hi = 0.f;
        lo = 0.f;
      }
      const float x0 = __ldg(x + c.x), x1 = __ldg(x + c.y), x2 = __ldg(x + c.z), x3 = __ldg(x + c.w);
      df_fma(hi, lo, v.x, x0);
      df_fma(hi, lo, v.y, x1);
      df_fma(hi, lo, v.z, x2);
      df_fma(hi, lo, v.w, x3);
    }
    c = cn;
    v = vn;
  }
  if (cur >= 0) {
    slot_hi[cur * SLOT_W + lane] = hi;
    slot_lo[cur * SLOT_W + lane] = lo;
  }
  __syncwarp();
  if (lane < nrows) {
    float h = 0.f, l = 0.f;
#pragma unroll 8
    for (int i = 0; i < 32; ++i) df_add(h, l, slot_hi[lane * SLOT_W + i], slot_lo[lane * SLOT_W + i]);
    out_hi = h;
    out_lo = l;
  }
  __syncwarp();
}

// FP32 rows: returns row (lane) sums in lanes 0..nrows-1.
template <bool BF16, int R>
__device__ __forceinline__ float warp_rows_dot_f(const DevCSR& M, int row0, int nrows,
                                                 const float* __restrict__ x, int lane,
                                                 float* slot) {
  if (nrows <= 0) return 0.f;
  int bnd[R + 1];
  load_bounds<R>(M, row0, nrows, lane, bnd);
#pragma unroll
  for (int q = 0; q < R; ++q) slot[q * SLOT_W + lane] = 0.f;
  const uint64_t pol = evict_first_policy();
  const int P1 = bnd[nrows];
  int p = bnd[0] + lane * 4;
  int4 c = make_int4(0, 0, 0, 0);
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (p < P1) {
    c = ld_stream_i4(M.col + p, pol);
    v = ld_vals<BF16>(M, p, pol);
  }
  float acc = 0.f;
  int cur = -1;
  for (int base = bnd[0]; base < P1; base += 128, p += 128) {
    const int pn = p + 128;
    int4 cn = make_int4(0, 0, 0, 0);
    float4 vn = make_float4(0.f, 0.f, 0.f, 0.f);
    if (pn < P1) {
      cn = ld_stream_i4(M.col + pn, pol);
      vn = ld_vals<BF16>(M, pn, pol);
    }
    if (p < P1) {
      const int q = row_of<R>(p, bnd, nrows);
      if (q != cur) {
        if (cur >= 0) slot[cur * SLOT_W + lane] = acc;
        cur = q;
        acc = 0.f;
      }
      const float x0 = __ldg(x + c.x), x1 = __ldg(x + c.y), x2 = __ldg(x + c.z), x3 = __ldg(x + c.w);
      acc = fmaf(v.x, x0, acc);
      acc = fmaf(v.y, x1, acc);
      acc = fmaf(v.z, x2, acc);
      acc = fmaf(v.w, x3, acc);
    }
    c = cn;
    v = vn;
  }
  if (cur >= 0) slot[cur * SLOT_W + lane] = acc;
  __syncwarp();
  float out = 0.f;
  if (lane < nrows) {
#pragma unroll 8
    for (int i = 0; i < 32; ++i) out += slot[lane * SLOT_W + i];
  }
  __syncwarp();
  return out;
}

// Forward projection with the Poisson-ratio epilogue (steps a1, a2) and the
// FP64 data term of the objective.  Each warp projects ROWS_PER_WARP rows;
// the epilogue runs once per block on 64 consecutive rows with full warps
// (FP64 is scarce on this part, so it is issued as few times as possible).
template <bool BF16, bool DATA>
__global__ void __launch_bounds__(THREADS) k_forward(FwdArgs a) {
  SolverState* st = a.st;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float* f;
  double* y_out;
  const double* y_prev = nullptr;
  double theta = 0.0;
  if (a.loop) {
    if (st->done) return;  // uniform over the grid
    const int kk = st->k;
    theta = st->theta;
    f = a.f[kk % 3];
    y_out = a.y[kk & 1];
    y_prev = a.y[(kk + 1) & 1];
  } else {
    f = a.f[0];
    y_out = a.y[0];
  }
  __shared__ float s_hi[WARPS][ROWS_PER_WARP * SLOT_W];
  __shared__ float s_lo[WARPS][ROWS_PER_WARP * SLOT_W];
  __shared__ float r_hi[WARPS * ROWS_PER_WARP], r_lo[WARPS * ROWS_PER_WARP];
  const int m = a.A.rows;
  const int block_row0 = blockIdx.x * WARPS * ROWS_PER_WARP;
  const int row0 = block_row0 + warp * ROWS_PER_WARP;
  const int nrows = max(0, min(ROWS_PER_WARP, m - row0));
  float hi, lo;
  warp_rows_dot_df<BF16, ROWS_PER_WARP>(a.A, row0, nrows, f, lane, s_hi[warp], s_lo[warp], hi, lo);
  if (lane < ROWS_PER_WARP) {
    r_hi[warp * ROWS_PER_WARP + lane] = hi;
    r_lo[warp * ROWS_PER_WARP + lane] = lo;
  }
  __syncthreads();
  double data = 0.0;
  int hits = 0, bad = 0;
  const int t = threadIdx.x;
  const int row = block_row0 + t;
  if (t < WARPS * ROWS_PER_WARP && row < m) {
    const double y = (double)r_hi[t] + (double)r_lo[t];
    y_out[row] = y;
    const double gam = (double)a.gamma[row];
    const double gg = (double)a.g[row];
    if (a.w != nullptr) {
      double yt = y;
      if (theta != 0.0) yt = fma(theta, y - y_prev[row], y);
      double den = yt + gam;
      const double floor_ = KAPPA * gam;
      if (den < floor_) {
        den = floor_;
        hits = 1;
      }
      // w = 1 - g/den = (den - g)/den: the numerator is formed in FP64 so the
      // weight keeps its relative accuracy when den ~ g.
      const float wv = __fdiv_rn((float)(den - gg), (float)den);
      a.w[row] = wv;
      if (!isfinite(wv)) bad = 1;
    }
    if (!isfinite(y)) bad = 1;
    if (DATA) data = y - gg * log(y + gam);
  }
  if (a.loop || a.want_data) {
    const int bhits = block_sum_i(hits);
    const int bbad = block_sum_i(bad);
    double bdata = 0.0;
    if (DATA) bdata = block_sum_d(data);
    if (threadIdx.x == 0) {
      if (bhits) atomicAdd(&st->guard_hits, (unsigned long long)bhits);
      if (bbad) atomicOr(&st->flags, (int)APPGA_FLAG_NONFINITE);
    }
    if (DATA) {
      if (publish_and_check_last(a.partial, bdata, &st->ticket_r)) {
        const double tot = sum_partials(a.partial);
        if (threadIdx.x == 0) {
          if (a.loop) st->data_term = tot;
          if (a.data_out) *a.data_out = tot;
          st->ticket_r = 0;
        }
      }
    }
  }
}

// ------------------------------------------------------------- stencil
// Row-major image, pixel (r, c).  D acts along c for I (x) D and along r
// for D (x) I (Sec. 2.1).  With [.] the Iverson bracket:
//   (D x)_i   = [i >= 1] (x_i - x_{i-1})
//   (D^T y)_i = [i >= 1] y_i - [i <= N-2] y_{i+1}
// The six fields of B = [B1; B2] at (r, c), with X the tile and (i, j) the
// position of (r, c) in it:
//   u1 = Dc X,  u2 = Dr X,  u3 = -DTc Dc X,  u4 = -DTr Dc X,
//   u5 = -DTr Dr X,  u6 = -Dr DTc X
// and the adjoint B^T v = DTc v1 + DTr v2 - DTc Dc v3 - Dr DTc v4
//                        - DTr Dr v5 - DTr Dc v6,
// i.e. the u3-, u6-, u5- and u4-forms applied to v3, v4, v5, v6.

template <int W>
__device__ __forceinline__ float form_u3(const float (*X)[W], int i, int j, bool c_lo, bool c_hi) {
  float t = 0.f;
  if (c_lo) t -= X[i][j] - X[i][j - 1];
  if (c_hi) t += X[i][j + 1] - X[i][j];
  return t;
}
template <int W>
__device__ __forceinline__ float form_u5(const float (*X)[W], int i, int j, bool r_lo, bool r_hi) {
  float t = 0.f;
  if (r_lo) t -= X[i][j] - X[i - 1][j];
  if (r_hi) t += X[i + 1][j] - X[i][j];
  return t;
}
template <int W>
__device__ __forceinline__ float form_u4(const float (*X)[W], int i, int j, bool r_lo, bool r_hi,
                                         bool c_lo) {
  if (!c_lo) return 0.f;
  float t = 0.f;
  if (r_lo) t -= X[i][j] - X[i][j - 1];
  if (r_hi) t += X[i + 1][j] - X[i + 1][j - 1];
  return t;
}
template <int W>
__device__ __forceinline__ float form_u6(const float (*X)[W], int i, int j, bool r_lo, bool c_lo,
                                         bool c_hi) {
  if (!r_lo) return 0.f;
  float t = 0.f;
  if (c_lo) t -= X[i][j] - X[i - 1][j];
  if (c_hi) t += X[i][j + 1] - X[i - 1][j + 1];
  return t;
}

template <int W>
__device__ __forceinline__ void diff_fields(const float (*X)[W], int i, int j, int r, int c, int n,
                                            float u[6]) {
  const bool r_lo = r >= 1, r_hi = r <= n - 2, c_lo = c >= 1, c_hi = c <= n - 2;
  u[0] = c_lo ? X[i][j] - X[i][j - 1] : 0.f;
  u[1] = r_lo ? X[i][j] - X[i - 1][j] : 0.f;
  u[2] = form_u3<W>(X, i, j, c_lo, c_hi);
  u[3] = form_u4<W>(X, i, j, r_lo, r_hi, c_lo);
  u[4] = form_u5<W>(X, i, j, r_lo, r_hi);
  u[5] = form_u6<W>(X, i, j, r_lo, c_lo, c_hi);
}

// s_eps of a group (Eq. def:smoothL2) given its squared norm.
__device__ __forceinline__ float s_eps_f(float nrm2, float eps) {
  const float nrm = sqrtf(nrm2);
  return nrm > eps ? nrm - 0.5f * eps : nrm2 / (2.f * eps);
}

constexpr int TW = TILE_C + 4;  // f tile width (halo 2)
constexpr int VW = TILE_C + 2;  // v tile width (halo 1)

struct StencilSmem {
  float T[TILE_R + 4][TW];      // f~ (or f) with halo 2
  float K[TILE_R + 4][TW];      // f^k with halo 2
  float V[6][TILE_R + 2][VW];   // grad phi~ fields with halo 1
  float G[TILE_R * TILE_C];     // B^T grad phi~(B f~) at the tile pixels
};

// v = grad phi~(B X) on the (TILE_R+2) x (TILE_C+2) points around the tile.
__device__ void stencil_v(StencilSmem& S, int r0, int c0, int n, float lam1, float lam2,
                          float eps) {
  for (int t = threadIdx.x; t < (TILE_R + 2) * VW; t += THREADS) {
    const int ii = t / VW, jj = t % VW;
    const int r = r0 - 1 + ii, c = c0 - 1 + jj;
    float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (r >= 0 && r < n && c >= 0 && c < n) {
      float u[6];
      diff_fields<TW>(S.T, ii + 1, jj + 1, r, c, n, u);
      const float n1 = u[0] * u[0] + u[1] * u[1];
      const float n2 = u[2] * u[2] + u[3] * u[3] + u[4] * u[4] + u[5] * u[5];
      // grad s_eps(x) = x / max(||x||, eps), scaled by lambda (Sec. 2.2)
      const float s1 = lam1 / fmaxf(sqrtf(n1), eps);
      const float s2 = lam2 / fmaxf(sqrtf(n2), eps);
      v[0] = s1 * u[0];
      v[1] = s1 * u[1];
      v[2] = s2 * u[2];
      v[3] = s2 * u[3];
      v[4] = s2 * u[4];
      v[5] = s2 * u[5];
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) S.V[q][ii][jj] = v[q];
  }
}

// B^T v at tile pixel (r, c), located at (i, j) = (ii + 1, jj + 1) in V.
__device__ __forceinline__ float stencil_adjoint(const StencilSmem& S, int i, int j, int r, int c,
                                                 int n) {
  const bool r_lo = r >= 1, r_hi = r <= n - 2, c_lo = c >= 1, c_hi = c <= n - 2;
  float t = 0.f;
  if (c_lo) t += S.V[0][i][j];
  if (c_hi) t -= S.V[0][i][j + 1];
  if (r_lo) t += S.V[1][i][j];
  if (r_hi) t -= S.V[1][i + 1][j];
  t += form_u3<VW>(S.V[2], i, j, c_lo, c_hi);
  t += form_u6<VW>(S.V[3], i, j, r_lo, c_lo, c_hi);
  t += form_u5<VW>(S.V[4], i, j, r_lo, r_hi);
  t += form_u4<VW>(S.V[5], i, j, r_lo, r_hi, c_lo);
  return t;
}

// lam1 s_eps(pair) + lam2 s_eps(quad) at pixel (r, c) of X (position (i, j)).
__device__ __forceinline__ float reg_at(const float (*X)[TW], int i, int j, int r, int c, int n,
                                        float lam1, float lam2, float eps) {
  float u[6];
  diff_fields<TW>(X, i, j, r, c, n, u);
  const float n1 = u[0] * u[0] + u[1] * u[1];
  const float n2 = u[2] * u[2] + u[3] * u[3] + u[4] * u[4] + u[5] * u[5];
  return lam1 * s_eps_f(n1, eps) + lam2 * s_eps_f(n2, eps);
}

// Momentum scalar for index k (Eq. GNtheta) -- FP64 on the device.
__device__ double gn_t_dev(int k, double a, double b, double omega) {
  return a * pow((double)k, omega) + b;
}

// theta_{k0} and t_{k0} of the first iteration of a run, with the same device
// arithmetic the pixel kernel uses for later indices (so a resumed run
// replays an uninterrupted one bit for bit).
__global__ void k_init_momentum(SolverState* st, int k0, int momentum, double a, double b,
                                double omega) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double theta = 0.0, t = 1.0;
  if (momentum == APPGA_MOMENTUM_GN) {
    theta = (gn_t_dev(k0 - 1, a, b, omega) - 1.0) / gn_t_dev(k0, a, b, omega);
  } else if (momentum == APPGA_MOMENTUM_NESTEROV) {
    for (int k = 1; k <= k0; ++k) {  // t_0 = 1
      const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
      theta = (t - 1.0) / tn;
      t = tn;
    }
  }
  st->theta = theta;
  st->t_cur = t;
}

// Fused pixel phase: steps a0, a3, a4, a5 (+ the regulariser term of Phi(f^k)).
template <bool BF16, bool TRACK>
__global__ void __launch_bounds__(THREADS) k_pixel(PixArgs a) {
  SolverState* st = a.st;
  if (st->done) return;  // uniform over the grid
  const int kk = st->k;
  const double theta = st->theta;
  const float* __restrict__ fk = a.f[kk % 3];
  const float* __restrict__ fkm = a.f[(kk + 2) % 3];
  float* __restrict__ fnext = a.f[(kk + 1) % 3];
  const int n = a.n;
  const int r0 = blockIdx.y * TILE_R, c0 = blockIdx.x * TILE_C;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ StencilSmem S;
  __shared__ float s_slot[WARPS][PIX_PER_WARP * SLOT_W];
  const float th = (float)theta;

  // a3: grad F = A^T w for this warp's PIX_PER_WARP consecutive pixels (their
  // rows of the transposed CSR are contiguous); issued first so the stream
  // starts at once
  float keep = 0.f;
  {
    const int t0 = warp * PIX_PER_WARP;
    const int r = r0 + t0 / TILE_C, c = c0 + t0 % TILE_C;
    const int np = r < n ? max(0, min(PIX_PER_WARP, n - c)) : 0;
    keep = warp_rows_dot_f<BF16, PIX_PER_WARP>(a.At, r * n + c, np, a.w, lane, s_slot[warp]);
  }

  // a0: f~ = f^k + theta (f^k - f^{k-1}) on the tile with halo 2
  for (int t = threadIdx.x; t < (TILE_R + 4) * TW; t += THREADS) {
    const int ii = t / TW, jj = t % TW;
    const int r = r0 - 2 + ii, c = c0 - 2 + jj;
    float vk = 0.f, vt = 0.f;
    if (r >= 0 && r < n && c >= 0 && c < n) {
      vk = fk[r * n + c];
      const float vm = fkm[r * n + c];
      vt = fmaf(th, vk - vm, vk);
    }
    S.K[ii][jj] = vk;
    S.T[ii][jj] = vt;
  }
  __syncthreads();
  // a4: grad phi~(B f~) around the tile, then B^T at the tile pixels
  stencil_v(S, r0, c0, n, a.ip.lambda1, a.ip.lambda2, a.ip.eps);
  __syncthreads();
  float reg = 0.f;
  for (int t = threadIdx.x; t < TILE_R * TILE_C; t += THREADS) {
    const int ii = t / TILE_C, jj = t % TILE_C;
    const int r = r0 + ii, c = c0 + jj;
    float gr = 0.f;
    if (r < n && c < n) {
      gr = stencil_adjoint(S, ii + 1, jj + 1, r, c, n);
      if (TRACK) reg += reg_at(S.K, ii + 2, jj + 2, r, c, n, a.ip.lambda1, a.ip.lambda2, a.ip.eps);
    }
    S.G[t] = gr;
  }
  __syncthreads();  // S.G complete
  // a5: f^{k+1} = max(f~ - beta (f^k / Lambda) (grad F + grad R), 0)
  int bad = 0;
  if (lane < PIX_PER_WARP) {
    const int t = warp * PIX_PER_WARP + lane;
    const int ii = t / TILE_C, jj = t % TILE_C;
    const int r = r0 + ii, c = c0 + jj;
    if (r < n && c < n) {
      const int j = r * n + c;
      const float ft = S.T[ii + 2][jj + 2];
      float pk = S.K[ii + 2][jj + 2];
      if (a.ip.freeze_iter >= 0) {
        if (kk == a.ip.freeze_iter) {
          a.pfreeze[j] = pk;
        } else if (kk > a.ip.freeze_iter) {
          pk = a.pfreeze[j];
        }
      }
      const float p = a.ip.beta * pk * a.inv_lambda[j];
      const float grad = keep + S.G[t];
      const float x = __fmaf_rn(-p, grad, ft);
      if (!isfinite(x)) bad = 1;
      fnext[j] = fmaxf(x, 0.f);
    }
  }
  // Finalise the iteration in the last block: Phi(f^k), the stopping test,
  // the next index and the next momentum scalar.
  const int bbad = block_sum_i(bad);
  if (threadIdx.x == 0 && bbad) atomicOr(&st->flags, (int)APPGA_FLAG_NONFINITE);
  double breg = 0.0;
  if (TRACK) breg = block_sum_d((double)reg);
  if (publish_and_check_last(a.partial, breg, &st->ticket_p)) {
    double reg_tot = 0.0;
    if (TRACK) reg_tot = sum_partials(a.partial);
    if (threadIdx.x == 0) {
      st->ticket_p = 0;
      bool stop = false;
      if (TRACK) {
        const double phi = st->data_term + reg_tot;
        const double prev = st->phi_cur;
        st->phi_prev = prev;
        st->phi_cur = phi;
        if (a.ip.rel_tol > 0.0 && kk > st->k0 && fabs(phi - prev) <= a.ip.rel_tol * fabs(prev)) {
          stop = true;
          st->done = 1;
          st->result_k = kk;
          st->stopped_early = 1;
        }
      }
      if (!stop) {
        if (kk >= st->k_last) {
          st->done = 1;
          st->result_k = kk + 1;
        }
        st->k = kk + 1;
        double th_next = 0.0;
        if (a.ip.momentum == APPGA_MOMENTUM_GN) {
          th_next = (gn_t_dev(kk, a.ip.a, a.ip.b, a.ip.omega) - 1.0) /
                    gn_t_dev(kk + 1, a.ip.a, a.ip.b, a.ip.omega);
        } else if (a.ip.momentum == APPGA_MOMENTUM_NESTEROV) {
          const double t = st->t_cur;
          const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
          th_next = (t - 1.0) / tn;
          st->t_cur = tn;
        }
        st->theta = th_next;
      }
    }
  }
}

// Standalone back-projection (step a3): out = A^T w.
template <bool BF16>
__global__ void __launch_bounds__(THREADS) k_backproject(DevCSR At, const float* __restrict__ w,
                                                         float* __restrict__ out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ float s_slot[WARPS][ROWS_PER_WARP * SLOT_W];
  const int row0 = (blockIdx.x * WARPS + warp) * ROWS_PER_WARP;
  const int nrows = max(0, min(ROWS_PER_WARP, At.rows - row0));
  const float s = warp_rows_dot_f<BF16, ROWS_PER_WARP>(At, row0, nrows, w, lane, s_slot[warp]);
  if (lane < nrows) out[row0 + lane] = s;
}

// Standalone SHOITV gradient (step a4): out = B^T grad phi~(B f).
__global__ void __launch_bounds__(THREADS) k_shoitv(int n, const float* __restrict__ f, float lam1,
                                                    float lam2, float eps, float* __restrict__ out) {
  const int r0 = blockIdx.y * TILE_R, c0 = blockIdx.x * TILE_C;
  __shared__ StencilSmem S;
  for (int t = threadIdx.x; t < (TILE_R + 4) * TW; t += THREADS) {
    const int ii = t / TW, jj = t % TW;
    const int r = r0 - 2 + ii, c = c0 - 2 + jj;
    S.T[ii][jj] = (r >= 0 && r < n && c >= 0 && c < n) ? f[r * n + c] : 0.f;
  }
  __syncthreads();
  stencil_v(S, r0, c0, n, lam1, lam2, eps);
  __syncthreads();
  for (int t = threadIdx.x; t < TILE_R * TILE_C; t += THREADS) {
    const int ii = t / TILE_C, jj = t % TILE_C;
    const int r = r0 + ii, c = c0 + jj;
    if (r < n && c < n) out[r * n + c] = stencil_adjoint(S, ii + 1, jj + 1, r, c, n);
  }
}

// Regulariser term phi~(B f) in FP64 (objective, step a6).
__global__ void __launch_bounds__(THREADS) k_reg_term(int n, const float* __restrict__ f, float lam1,
                                                      float lam2, float eps, double* partial,
                                                      SolverState* st, double* out) {
  const int r0 = blockIdx.y * TILE_R, c0 = blockIdx.x * TILE_C;
  __shared__ float X[TILE_R + 4][TW];
  for (int t = threadIdx.x; t < (TILE_R + 4) * TW; t += THREADS) {
    const int ii = t / TW, jj = t % TW;
    const int r = r0 - 2 + ii, c = c0 - 2 + jj;
    X[ii][jj] = (r >= 0 && r < n && c >= 0 && c < n) ? f[r * n + c] : 0.f;
  }
  __syncthreads();
  double reg = 0.0;
  for (int t = threadIdx.x; t < TILE_R * TILE_C; t += THREADS) {
    const int ii = t / TILE_C, jj = t % TILE_C;
    const int r = r0 + ii, c = c0 + jj;
    if (r < n && c < n) reg += (double)reg_at(X, ii + 2, jj + 2, r, c, n, lam1, lam2, eps);
  }
  const double b = block_sum_d(reg);
  if (publish_and_check_last(partial, b, &st->ticket_aux)) {
    const double tot = sum_partials(partial);
    if (threadIdx.x == 0) {
      *out = tot;
      st->ticket_aux = 0;
    }
  }
}

// Input validation: g finite and >= 0, gamma finite and > 0, f finite and >= 0.
__global__ void k_validate(const float* __restrict__ g, const float* __restrict__ gamma, int m,
                           const float* __restrict__ f, int d, int* flag) {
  int bad = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const float gi = g[i], ci = gamma[i];
    if (!(isfinite(gi) && gi >= 0.f && isfinite(ci) && ci > 0.f)) bad = 1;
  }
  if (f != nullptr) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x) {
      const float x = f[i];
      if (!(isfinite(x) && x >= 0.f)) bad = 1;
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

// Initial image (Sec. 4.1): TMC * 1_disk, TMC = (sum g - sum gamma)/(NPFOV * NPA).
__global__ void __launch_bounds__(THREADS) k_actc(const float* __restrict__ g,
                                                  const float* __restrict__ gamma, int m,
                                                  double* partial, SolverState* st,
                                                  double* actc_out) {
  double v = 0.0;
  for (int i = blockIdx.x * THREADS + threadIdx.x; i < m; i += gridDim.x * THREADS)
    v += (double)g[i] - (double)gamma[i];
  const double b = block_sum_d(v);
  if (publish_and_check_last(partial, b, &st->ticket_aux)) {
    const double tot = sum_partials(partial);
    if (threadIdx.x == 0) {
      *actc_out = tot;
      st->ticket_aux = 0;
    }
  }
}
// Pixel centre (c + 1/2 - N/2, r + 1/2 - N/2) inside x^2 + y^2 <= (N/2)^2, in
// exact integer arithmetic (both sides scaled by 4).
__device__ __forceinline__ bool in_disk(int r, int c, int n) {
  const long long dx = 2ll * c + 1 - n, dy = 2ll * r + 1 - n;
  return dx * dx + dy * dy <= (long long)n * n;
}
__global__ void k_fill_disk(int n, int n_angles, int npfov, const double* actc, float* f_out) {
  const double tmc = *actc / ((double)npfov * (double)n_angles);
  const float v = (float)tmc;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n * n; j += gridDim.x * blockDim.x)
    f_out[j] = in_disk(j / n, j % n, n) ? v : 0.f;
}

}  // namespace

// ------------------------------------------------------------- launchers

int fwd_grid(int m) { return (m + WARPS * ROWS_PER_WARP - 1) / (WARPS * ROWS_PER_WARP); }
int pix_grid_x(int n) { return (n + TILE_C - 1) / TILE_C; }
int pix_grid_y(int n) { return (n + TILE_R - 1) / TILE_R; }
int max_partials(int m, int n) {
  const int a = fwd_grid(m), b = pix_grid_x(n) * pix_grid_y(n);
  return (a > b ? a : b) + 1024;
}

cudaError_t launch_forward(const FwdArgs& a, int track, cudaStream_t s) {
  const int grid = fwd_grid(a.A.rows);
  if (grid == 0) return cudaSuccess;
  const bool data = track || a.want_data;
  if (a.use_bf16) {
    if (data)
      k_forward<true, true><<<grid, THREADS, 0, s>>>(a);
    else
      k_forward<true, false><<<grid, THREADS, 0, s>>>(a);
  } else {
    if (data)
      k_forward<false, true><<<grid, THREADS, 0, s>>>(a);
    else
      k_forward<false, false><<<grid, THREADS, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_pixel(const PixArgs& a, cudaStream_t s) {
  dim3 grid(pix_grid_x(a.n), pix_grid_y(a.n));
  if (a.use_bf16) {
    if (a.ip.track)
      k_pixel<true, true><<<grid, THREADS, 0, s>>>(a);
    else
      k_pixel<true, false><<<grid, THREADS, 0, s>>>(a);
  } else {
    if (a.ip.track)
      k_pixel<false, true><<<grid, THREADS, 0, s>>>(a);
    else
      k_pixel<false, false><<<grid, THREADS, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_backproject(const DevCSR& At, const float* w, float* out, int use_bf16,
                               cudaStream_t s) {
  const int grid = fwd_grid(At.rows);
  if (grid == 0) return cudaSuccess;
  if (use_bf16)
    k_backproject<true><<<grid, THREADS, 0, s>>>(At, w, out);
  else
    k_backproject<false><<<grid, THREADS, 0, s>>>(At, w, out);
  return cudaGetLastError();
}

cudaError_t launch_shoitv_grad(int n, const float* f, float lam1, float lam2, float eps,
                               float* out, cudaStream_t s) {
  dim3 grid(pix_grid_x(n), pix_grid_y(n));
  k_shoitv<<<grid, THREADS, 0, s>>>(n, f, lam1, lam2, eps, out);
  return cudaGetLastError();
}

cudaError_t launch_reg_term(int n, const float* f, float lam1, float lam2, float eps,
                            double* partial, SolverState* st, double* out, cudaStream_t s) {
  dim3 grid(pix_grid_x(n), pix_grid_y(n));
  k_reg_term<<<grid, THREADS, 0, s>>>(n, f, lam1, lam2, eps, partial, st, out);
  return cudaGetLastError();
}

cudaError_t launch_validate_inputs(const float* g, const float* gamma, int m, const float* f,
                                   int d, int* flag, cudaStream_t s) {
  k_validate<<<256, 256, 0, s>>>(g, gamma, m, f, d, flag);
  return cudaGetLastError();
}

cudaError_t launch_init_momentum(SolverState* st, int k0, int momentum, double a, double b,
                                 double omega, cudaStream_t s) {
  k_init_momentum<<<1, 32, 0, s>>>(st, k0, momentum, a, b, omega);
  return cudaGetLastError();
}

long long disk_pixels(int n) {
  // pixels with centres in the inscribed disk (same integer test as in_disk)
  long long npfov = 0;
  for (long long r = 0; r < n; ++r)
    for (long long c = 0; c < n; ++c) {
      const long long dx = 2 * c + 1 - n, dy = 2 * r + 1 - n;
      npfov += (dx * dx + dy * dy <= (long long)n * n) ? 1 : 0;
    }
  return npfov;
}

cudaError_t launch_initial_image(const float* g, const float* gamma, int m, int n, int n_angles,
                                 long long npfov, double* partial, SolverState* st, float* f_out,
                                 cudaStream_t s) {
  // the ACTc scalar is parked in the last partial slot
  double* actc = partial + 1023;
  k_actc<<<256, THREADS, 0, s>>>(g, gamma, m, partial, st, actc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_fill_disk<<<pix_grid_x(n) * 8, 256, 0, s>>>(n, n_angles, (int)npfov, actc, f_out);
  return cudaGetLastError();
}

}  // namespace appga
