// Single-slice CUDA kernels of the APPGA hot path (sm_103a).
//
//   k_forward : y = A f^k (double-float accumulation), y~ = y + theta_k (y - y^{k-1})
//               (the projection of f~^k by linearity), w = 1 - g / max(y~ + gamma,
//               kappa gamma), data term of the objective; in the solver loop
//               the same launch also runs the SHOITV stencil of
//               f~^k = f^k + theta_k (f^k - f^{k-1}) (B^T grad phi~(B f~^k)), the
//               regulariser term of Phi(f^k) and the stopping test
//               (steps a0, a1, a2, a4, a6; Sec. 2.2, Eq. FidelityTerm,
//               Eq. gradenvL2, Eq. def:phi)
//   k_pixel   : grad F = A^T w through the transposed CSR (no atomics) and the
//               EM-preconditioned projected update f^{k+1} = max(f~ - beta
//               (f^k / Lambda)(grad F + B^T grad phi~), 0); next index and FP64
//               momentum scalar (steps a3, a5; Eq. APPGAiter, Eq. EM, Eq. GNtheta)
//
// Projector layout: a warp owns 8 consecutive CSR rows, whose row-padded
// entries form one contiguous range, and streams it linearly in 128-entry
// chunks (a 16-byte pack of columns and one of values per lane), keeping PF
// chunks in flight in registers.  Lanes accumulate into their current row and
// park partials in per-warp shared-memory slots; lane q sums row q.  No
// block-wide barrier sits on the streaming path.
//
// The per-row epilogue runs on the FP32 pipe only: double-float (FP32 pair)
// arithmetic for y, y~, the guarded denominator, and a double-float natural
// logarithm for the data term -- this part's FP64 pipe is a small fraction of
// its FP32 rate, so FP64 is used only for a handful of scalars per launch.
//
// Kernels read the iteration index and theta from a device-resident
// SolverState, so a captured graph of (k_pixel, k_forward) pairs replays
// without host involvement.  Block partials (double-float pairs) are combined
// by the last block to finish (ticket counter) in index order: every
// reduction is deterministic.
#include <cuda_runtime.h>
#include <math.h>

#include <cmath>

#include "appga_internal.h"

namespace appga {
namespace {

constexpr int THREADS = 256;  // setup / reduction kernels
constexpr int MAX_WARPS = 32;
constexpr int ROWS_PER_WARP = 8;  // projector rows per warp
constexpr int PW_WARPS = 2;       // warps per projector block
constexpr int PW_THREADS = PW_WARPS * 32;
constexpr int PW_ROWS = PW_WARPS * ROWS_PER_WARP;  // rows per projector block
#ifndef APPGA_PF
#define APPGA_PF 2
#endif
constexpr int PF = APPGA_PF;  // chunks of the nnz stream in flight per warp
constexpr int SLOT_W = 33;    // slot row stride: per-row sums read without bank conflicts

// Stencil tiles: ST_R x ST_C pixels, one pixel per thread of a projector block
constexpr int ST_R = 2;
constexpr int ST_C = 32;
static_assert(ST_R * ST_C == PW_THREADS, "stencil tile = one pixel per thread");
constexpr int TW = ST_C + 4;  // f tile width (halo 2)
constexpr int VW = ST_C + 2;  // v tile width (halo 1)

// ----------------------------------------------------------------- loads

// A and A^T are streamed once per iteration: bypass L1 and tag the lines
// evict-first in L2 (cache-policy operand) so the gathered vectors stay cached.
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
// A double-float is an unevaluated sum hi + lo of two floats (about 48
// significant bits).  Error-free transformations: Knuth's TwoSum and the
// FMA-based TwoProduct.  The _rn intrinsics keep the compiler from
// contracting or reassociating them.
struct df {
  float hi, lo;
};
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ df quick_renorm(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_add(df a, df b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return quick_renorm(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df df_add_f(df a, float b) {
  float s, e;
  two_sum(a.hi, b, s, e);
  return quick_renorm(s, __fadd_rn(e, a.lo));
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return quick_renorm(p, e);
}
__device__ __forceinline__ df df_mul_f(df a, float b) {
  const float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return quick_renorm(p, e);
}
__device__ __forceinline__ float df_to_f(df a) { return __fadd_rn(a.hi, a.lo); }

// (hi, lo) += a * x with the product and the sum error kept in lo (dot-product
// accumulator: the low parts are summed as plain floats).
__device__ __forceinline__ void acc_fma(float& hi, float& lo, float a, float x) {
  const float p = __fmul_rn(a, x);
  const float pe = __fmaf_rn(a, x, -p);
  float s, e;
  two_sum(hi, p, s, e);
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(e, pe));
}
__device__ __forceinline__ void acc_add(float& hi, float& lo, float h2, float l2) {
  float s, e;
  two_sum(hi, h2, s, e);
  hi = s;
  lo = __fadd_rn(__fadd_rn(lo, l2), e);
}

// Natural logarithm of a positive normal double-float x = hi + lo.
// Reduction: hi = 2^e m with m in [1, 2); c = 1 + j/64 the table point
// nearest m; r = (m + lo 2^-e - c)/c, |r| <= 1/128;
//   ln x = e ln 2 + ln c + ln(1 + r),
//   ln(1 + r) = r - r^2/2 + r^3/3 - r^4/4 + r^5/5 - r^6/6 + r^7/7 (+ O(r^8)),
// the first three terms in double-float, the rest in FP32 (below 2^-50 of
// the result).  ln c and ln 2 come as double-float constants computed on the
// host in extended precision.
__constant__ float c_logtab_hi[65];
__constant__ float c_logtab_lo[65];
__constant__ float c_ln2[2];
__constant__ float c_third[2];
__constant__ float c_kappa[2];  // the ratio guard factor kappa as a double-float

__device__ __forceinline__ df df_log(df x) {
  const int bits = __float_as_int(x.hi);
  const int e = ((bits >> 23) & 0xff) - 127;
  const float m = __int_as_float((bits & 0x007fffff) | 0x3f800000);
  const float ml = __fmul_rn(x.lo, __int_as_float((127 - e) << 23));  // lo * 2^-e, exact
  const int j = __float2int_rn(__fmul_rn(__fsub_rn(m, 1.f), 64.f));
  const float c = __fadd_rn(1.f, __fmul_rn((float)j, 0.015625f));
  const float d = __fsub_rn(m, c);  // exact: |m - c| <= 1/128 within [1, 2]
  float nh, nl;
  two_sum(d, ml, nh, nl);
  // r = (nh + nl) / c as a double-float
  const float qh = __fdiv_rn(nh, c);
  const float rem = __fmaf_rn(-qh, c, nh);
  const float ql = __fdiv_rn(__fadd_rn(rem, nl), c);
  const df r = quick_renorm(qh, ql);
  const df r2 = df_mul(r, r);
  const df r3 = df_mul(r2, r);
  const df third = {c_third[0], c_third[1]};
  // tail: -r^4/4 + r^5/5 - r^6/6 + r^7/7 from r^4 (hi only)
  const float rh = r.hi;
  const float r4 = __fmul_rn(r2.hi, r2.hi);
  float t = __fmaf_rn(rh, 1.f / 7.f, -1.f / 6.f);
  t = __fmaf_rn(rh, t, 0.2f);
  t = __fmaf_rn(rh, t, -0.25f);
  t = __fmul_rn(r4, t);
  df s = df_add(r, df_mul_f(r2, -0.5f));
  s = df_add(s, df_mul(r3, third));
  s = df_add_f(s, t);
  const df ln2 = {c_ln2[0], c_ln2[1]};
  const df lc = {c_logtab_hi[j], c_logtab_lo[j]};
  df out = df_add(df_mul_f(ln2, (float)e), lc);
  return df_add(out, s);
}

// ----------------------------------------------------------- reductions

__device__ __forceinline__ void warp_sum_acc(float& hi, float& lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    acc_add(hi, lo, h2, l2);
  }
}
__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// Deterministic block sum of a double-float accumulator (fixed tree); valid
// in warp 0.
__device__ df block_sum_acc(float hi, float lo) {
  __shared__ float red_hi[MAX_WARPS], red_lo[MAX_WARPS];
  warp_sum_acc(hi, lo);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) {
    red_hi[warp] = hi;
    red_lo[warp] = lo;
  }
  __syncthreads();
  float h = 0.f, l = 0.f;
  if (warp == 0) {
    if (lane < nw) {
      h = red_hi[lane];
      l = red_lo[lane];
    }
    warp_sum_acc(h, l);
  }
  return {h, l};
}
// Grid-wide deterministic reduction of one double-float per block, in two
// levels so that no single block sums thousands of partials serially: every
// block writes partial[b]; the last block to finish in each group of
// RED_GROUP blocks sums its group (in index order) into partial[nb + g]; the
// last group leader sums the group results.  Returns true in that final block
// only, with the total in *total (thread 0).  Group and final tickets are
// reset by their last user, so the counters start at zero for the next launch.
constexpr int RED_GROUP = 64;
__device__ bool grid_reduce(float2* partial, unsigned int* gtick, unsigned int* ftick, df mine,
                            double* total) {
  __shared__ int s_flag;
  const int nb = gridDim.x, b = blockIdx.x, g = b / RED_GROUP;
  const int ngroups = (nb + RED_GROUP - 1) / RED_GROUP;
  const int gsize = min(RED_GROUP, nb - g * RED_GROUP);
  if (threadIdx.x == 0) {
    partial[b] = make_float2(mine.hi, mine.lo);
    __threadfence();
    s_flag = (atomicAdd(&gtick[g], 1u) == (unsigned)(gsize - 1));
  }
  __syncthreads();
  if (!s_flag) return false;
  __threadfence();
  float h = 0.f, l = 0.f;
  for (int i = threadIdx.x; i < gsize; i += blockDim.x) {
    const float2 v = __ldcg(partial + g * RED_GROUP + i);
    acc_add(h, l, v.x, v.y);
  }
  const df gs = block_sum_acc(h, l);
  if (threadIdx.x == 0) {
    gtick[g] = 0;
    partial[nb + g] = make_float2(gs.hi, gs.lo);
    __threadfence();
    s_flag = (atomicAdd(ftick, 1u) == (unsigned)(ngroups - 1));
  }
  __syncthreads();
  if (!s_flag) return false;
  __threadfence();
  h = 0.f;
  l = 0.f;
  for (int i = threadIdx.x; i < ngroups; i += blockDim.x) {
    const float2 v = __ldcg(partial + nb + i);
    acc_add(h, l, v.x, v.y);
  }
  const df t = block_sum_acc(h, l);
  if (threadIdx.x == 0) {
    *ftick = 0;
    *total = (double)t.hi + (double)t.lo;
  }
  return true;
}
// Per-warp counters folded into a global counter without block barriers.
__device__ __forceinline__ void warp_count_add(unsigned long long* dst, int v) {
  v = warp_sum_i(v);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, (unsigned long long)v);
}
__device__ __forceinline__ void warp_flag_or(int* dst, int flag) {
  const unsigned any = __ballot_sync(0xffffffffu, flag != 0);
  if ((threadIdx.x & 31) == 0 && any) atomicOr(dst, flag ? flag : APPGA_FLAG_NONFINITE);
}

// ------------------------------------------------------------ projectors

// Row of entry p among rows q = 0..nrows-1 with starts bnd[0..nrows-1]
// (the last row starting at or before p; empty rows are skipped).
template <int R>
__device__ __forceinline__ int row_of(int p, const int (&bnd)[R + 1], int nrows) {
  int q = 0;
#pragma unroll
  for (int k = 1; k < R; ++k) q += (k < nrows && bnd[k] <= p) ? 1 : 0;
  return q;
}
// Row starts of rows row0 .. row0 + nrows (bnd[k] for k > nrows repeats the
// end); returns the end of the last row.
template <int R>
__device__ __forceinline__ int load_bounds(const DevCSR& M, int row0, int nrows, int lane,
                                           int (&bnd)[R + 1]) {
  const int b = lane <= nrows ? M.row_ptr[row0 + lane] : 0;
#pragma unroll
  for (int k = 0; k <= R; ++k) bnd[k] = __shfl_sync(0xffffffffu, b, k <= nrows ? k : nrows);
  return __shfl_sync(0xffffffffu, b, nrows);
}

// Rows [row0, row0 + nrows) of M times x; returns the sum of row `lane` in
// lanes 0..nrows-1: an accumulator pair if DF, else an FP32 value in out_hi.
// slot_hi / slot_lo: this warp's R*SLOT_W floats each of shared memory.
template <bool BF16, bool DF, int R>
__device__ __forceinline__ void warp_rows_dot(const DevCSR& M, int row0, int nrows,
                                              const float* __restrict__ x, int lane,
                                              float* slot_hi, float* slot_lo, float& out_hi,
                                              float& out_lo) {
  out_hi = 0.f;
  out_lo = 0.f;
  if (nrows <= 0) return;
  int bnd[R + 1];
  const int P1 = load_bounds<R>(M, row0, nrows, lane, bnd);
#pragma unroll
  for (int q = 0; q < R; ++q) {
    slot_hi[q * SLOT_W + lane] = 0.f;
    if (DF) slot_lo[q * SLOT_W + lane] = 0.f;
  }
  const uint64_t pol = evict_first_policy();
  const int P0 = bnd[0];
  const int nchunks = (P1 - P0 + 127) >> 7;
  int4 c[PF];
  float4 v[PF];
#pragma unroll
  for (int u = 0; u < PF; ++u) {
    const int p = P0 + (u << 7) + lane * 4;
    c[u] = make_int4(0, 0, 0, 0);
    v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (p < P1) {
      c[u] = ld_stream_i4(M.col + p, pol);
      v[u] = ld_vals<BF16>(M, p, pol);
    }
  }
  float hi = 0.f, lo = 0.f;
  int cur = -1;
  for (int t0 = 0; t0 < nchunks; t0 += PF) {
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int t = t0 + u;
      if (t < nchunks) {
        const int p = P0 + (t << 7) + lane * 4;
        const int4 cc = c[u];
        const float4 vv = v[u];
        const int pn = p + (PF << 7);
        if (pn < P1) {  // refill this slot with chunk t + PF before consuming chunk t
          c[u] = ld_stream_i4(M.col + pn, pol);
          v[u] = ld_vals<BF16>(M, pn, pol);
        }
        if (p < P1) {
          const int q = row_of<R>(p, bnd, nrows);
          if (q != cur) {
            if (cur >= 0) {
              slot_hi[cur * SLOT_W + lane] = hi;
              if (DF) slot_lo[cur * SLOT_W + lane] = lo;
            }
            cur = q;
            hi = 0.f;
            lo = 0.f;
          }
          const float x0 = __ldg(x + cc.x), x1 = __ldg(x + cc.y);
          const float x2 = __ldg(x + cc.z), x3 = __ldg(x + cc.w);
          if (DF) {
            acc_fma(hi, lo, vv.x, x0);
            acc_fma(hi, lo, vv.y, x1);
            acc_fma(hi, lo, vv.z, x2);
            acc_fma(hi, lo, vv.w, x3);
          } else {
            hi = fmaf(vv.x, x0, hi);
            hi = fmaf(vv.y, x1, hi);
            hi = fmaf(vv.z, x2, hi);
            hi = fmaf(vv.w, x3, hi);
          }
        }
      }
    }
  }
  if (cur >= 0) {
    slot_hi[cur * SLOT_W + lane] = hi;
    if (DF) slot_lo[cur * SLOT_W + lane] = lo;
  }
  __syncwarp();
  if (lane < nrows) {
    float h = 0.f, l = 0.f;
    if (DF) {
#pragma unroll 8
      for (int i = 0; i < 32; ++i) acc_add(h, l, slot_hi[lane * SLOT_W + i], slot_lo[lane * SLOT_W + i]);
    } else {
#pragma unroll 8
      for (int i = 0; i < 32; ++i) h += slot_hi[lane * SLOT_W + i];
    }
    out_hi = h;
    out_lo = l;
  }
  __syncwarp();
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

struct StencilSmem {
  float T[ST_R + 4][TW];     // f~ (or f) with halo 2
  float K[ST_R + 4][TW];     // f^k with halo 2
  float V[6][ST_R + 2][VW];  // grad phi~ fields with halo 1
};

// One stencil tile at (r0, c0): writes gR = B^T grad phi~(B f~) with
// f~ = fk + th (fk - fkm) for the tile pixels (if gR != nullptr) and returns
// this thread's term lam1 s_eps(pair) + lam2 s_eps(quad) of f^k (if want_reg).
__device__ float stencil_tile(StencilSmem& S, const float* __restrict__ fk,
                              const float* __restrict__ fkm, float th, int r0, int c0, int n,
                              float lam1, float lam2, float eps, float* __restrict__ gR,
                              bool want_reg) {
  for (int t = threadIdx.x; t < (ST_R + 4) * TW; t += blockDim.x) {
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
  // v = grad phi~(B f~) on the (ST_R+2) x (ST_C+2) points around the tile
  for (int t = threadIdx.x; t < (ST_R + 2) * VW; t += blockDim.x) {
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
  __syncthreads();
  float reg = 0.f;
  for (int t = threadIdx.x; t < ST_R * ST_C; t += blockDim.x) {
    const int ii = t / ST_C, jj = t % ST_C;
    const int r = r0 + ii, c = c0 + jj;
    if (r < n && c < n) {
      if (gR) {
        // B^T v at (r, c), located at (ii + 1, jj + 1) in V
        const int i = ii + 1, j = jj + 1;
        const bool r_lo = r >= 1, r_hi = r <= n - 2, c_lo = c >= 1, c_hi = c <= n - 2;
        float g = 0.f;
        if (c_lo) g += S.V[0][i][j];
        if (c_hi) g -= S.V[0][i][j + 1];
        if (r_lo) g += S.V[1][i][j];
        if (r_hi) g -= S.V[1][i + 1][j];
        g += form_u3<VW>(S.V[2], i, j, c_lo, c_hi);
        g += form_u6<VW>(S.V[3], i, j, r_lo, c_lo, c_hi);
        g += form_u5<VW>(S.V[4], i, j, r_lo, r_hi);
        g += form_u4<VW>(S.V[5], i, j, r_lo, r_hi, c_lo);
        gR[r * n + c] = g;
      }
      if (want_reg) {
        float u[6];
        diff_fields<TW>(S.K, ii + 2, jj + 2, r, c, n, u);
        const float n1 = u[0] * u[0] + u[1] * u[1];
        const float n2 = u[2] * u[2] + u[3] * u[3] + u[4] * u[4] + u[5] * u[5];
        reg += lam1 * s_eps_f(n1, eps) + lam2 * s_eps_f(n2, eps);
      }
    }
  }
  return reg;
}

__host__ __device__ __forceinline__ int st_tiles_x(int n) { return (n + ST_C - 1) / ST_C; }
__host__ __device__ __forceinline__ int st_tiles(int n) {
  return st_tiles_x(n) * ((n + ST_R - 1) / ST_R);
}
__host__ __device__ __forceinline__ int proj_blocks(int rows) {
  return (rows + PW_ROWS - 1) / PW_ROWS;
}

// Momentum scalar for index k (Eq. GNtheta) -- FP64 on the device.
__device__ double gn_t_dev(int k, double a, double b, double omega) {
  return a * pow((double)k, omega) + b;
}
__device__ void set_theta(SolverState* st, double theta) {
  st->theta = theta;
  const float h = (float)theta;
  st->theta_hi = h;
  st->theta_lo = (float)(theta - (double)h);
}

// ------------------------------------------------------------ k_forward

// Blocks [0, proj_blocks(m)) project rows; in the solver loop the blocks
// after them run the stencil tiles.
template <bool BF16>
__global__ void __launch_bounds__(PW_THREADS) k_forward(FwdArgs a) {
  __shared__ union {
    struct {
      float hi[PW_WARPS][ROWS_PER_WARP * SLOT_W];
      float lo[PW_WARPS][ROWS_PER_WARP * SLOT_W];
    } slot;
    StencilSmem st;
  } sm;
  SolverState* st = a.st;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (a.loop && st->done) return;  // uniform over the grid
  const int kk = a.loop ? st->k : 0;
  const int nproj = proj_blocks(a.A.rows);
  float acc_hi = 0.f, acc_lo = 0.f;  // this thread's share of the objective
  int hits = 0, bad = 0;
  if ((int)blockIdx.x < nproj) {
    const float* f = a.loop ? a.f[kk % 3] : a.f[0];
    const int m = a.A.rows;
    const int row0 = blockIdx.x * PW_ROWS + warp * ROWS_PER_WARP;
    const int nrows = max(0, min(ROWS_PER_WARP, m - row0));
    float hi, lo;
    warp_rows_dot<BF16, true, ROWS_PER_WARP>(a.A, row0, nrows, f, lane, sm.slot.hi[warp],
                                             sm.slot.lo[warp], hi, lo);
    if (lane < nrows) {
      const int row = row0 + lane;
      const df y = quick_renorm(hi, lo);
      const float gam = a.gamma[row], gg = a.g[row];
      if (a.loop) {
        a.y[kk & 1][row] = make_float2(y.hi, y.lo);
      } else {
        if (a.y[0]) a.y[0][row] = make_float2(y.hi, y.lo);
        if (a.y_out) a.y_out[row] = (double)y.hi + (double)y.lo;
      }
      if (a.w != nullptr) {
        df yt = y;
        if (a.loop) {
          // y~ = y + theta (y - y^{k-1}): the projection of f~ by linearity
          const float2 yp = a.y[(kk + 1) & 1][row];
          const df th = {st->theta_hi, st->theta_lo};
          const df dy = df_add(y, df_neg({yp.x, yp.y}));
          yt = df_add(y, df_mul(th, dy));
        }
        df den = df_add_f(yt, gam);
        const df floor_ = df_mul_f({c_kappa[0], c_kappa[1]}, gam);  // kappa * gamma
        if (df_add(den, df_neg(floor_)).hi < 0.f) {
          den = floor_;
          ++hits;
        }
        // w = 1 - g/den = (den - g)/den, numerator in double-float so the
        // weight keeps its relative accuracy when den ~ g
        const float wv = __fdiv_rn(df_to_f(df_add_f(den, -gg)), df_to_f(den));
        a.w[row] = wv;
        if (!isfinite(wv)) bad = 1;
      }
      if (!isfinite(y.hi)) bad = 1;
      if (a.want_data) {
        // data term y - g ln(y + gamma) (Eq. FidelityTerm), double-float
        const df term = df_add(y, df_neg(df_mul_f(df_log(df_add_f(y, gam)), gg)));
        acc_add(acc_hi, acc_lo, term.hi, term.lo);
      }
    }
  } else {
    // SHOITV gradient at f~^kk and the regulariser of Phi(f^kk)
    const int b = blockIdx.x - nproj;
    const int ntx = st_tiles_x(a.n);
    const float reg = stencil_tile(sm.st, a.f[kk % 3], a.f[(kk + 2) % 3], st->theta_hi,
                                   (b / ntx) * ST_R, (b % ntx) * ST_C, a.n, a.ip.lambda1,
                                   a.ip.lambda2, a.ip.eps, a.gR, a.want_data != 0);
    acc_hi = reg;
  }
  warp_count_add(&st->guard_hits, hits);
  warp_flag_or(&st->flags, bad ? APPGA_FLAG_NONFINITE : 0);
  if (!a.want_data) return;
  const df bsum = block_sum_acc(acc_hi, acc_lo);
  double tot = 0.0;
  if (grid_reduce(a.partial, a.gtick, &st->ticket_r, bsum, &tot)) {
    if (threadIdx.x == 0) {
      if (!a.loop) {
        if (a.data_out) *a.data_out = tot;
      } else {
        // Phi(f^kk) and the stopping test against Phi(f^{kk-1})
        const double prev = st->phi_cur;
        st->phi_prev = prev;
        st->phi_cur = tot;
        if (a.ip.rel_tol > 0.0 && kk > st->k0 && fabs(tot - prev) <= a.ip.rel_tol * fabs(prev)) {
          st->done = 1;
          st->result_k = kk;
          st->stopped_early = 1;
        }
      }
    }
  }
}

// -------------------------------------------------------------- k_pixel

template <bool BF16>
__global__ void __launch_bounds__(PW_THREADS) k_pixel(PixArgs a) {
  __shared__ float slot[PW_WARPS][ROWS_PER_WARP * SLOT_W];
  SolverState* st = a.st;
  if (st->done) return;  // uniform over the grid
  const int kk = st->k;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int d = a.At.rows;
  const int j0 = blockIdx.x * PW_ROWS + warp * ROWS_PER_WARP;
  const int np = max(0, min(ROWS_PER_WARP, d - j0));
  float bp, unused;
  warp_rows_dot<BF16, false, ROWS_PER_WARP>(a.At, j0, np, a.w, lane, slot[warp], nullptr, bp,
                                            unused);
  int bad = 0;
  if (lane < np) {
    const int j = j0 + lane;
    const float* fk = a.f[kk % 3];
    const float vk = fk[j];
    const float ft = fmaf(st->theta_hi, vk - a.f[(kk + 2) % 3][j], vk);
    float pk = vk;
    if (a.ip.freeze_iter >= 0) {
      if (kk == a.ip.freeze_iter) {
        a.pfreeze[j] = vk;
      } else if (kk > a.ip.freeze_iter) {
        pk = a.pfreeze[j];
      }
    }
    const float p = a.ip.beta * pk * a.inv_lambda[j];
    const float grad = bp + a.gR[j];
    const float xv = __fmaf_rn(-p, grad, ft);
    if (!isfinite(xv)) bad = 1;
    a.f[(kk + 1) % 3][j] = fmaxf(xv, 0.f);
  }
  warp_flag_or(&st->flags, bad ? APPGA_FLAG_NONFINITE : 0);
  // Finalise the iteration in the last block: the next index and momentum.
  double unused_total;
  if (grid_reduce(a.partial, a.gtick, &st->ticket_p, {0.f, 0.f}, &unused_total)) {
    if (threadIdx.x == 0) {
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
      set_theta(st, th_next);
    }
  }
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
  set_theta(st, theta);
  st->t_cur = t;
}

// Standalone back-projection (step a3): out = A^T w.
template <bool BF16>
__global__ void __launch_bounds__(PW_THREADS) k_backproject(DevCSR At, const float* __restrict__ w,
                                                            float* __restrict__ out) {
  __shared__ float slot[PW_WARPS][ROWS_PER_WARP * SLOT_W];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row0 = blockIdx.x * PW_ROWS + warp * ROWS_PER_WARP;
  const int nrows = max(0, min(ROWS_PER_WARP, At.rows - row0));
  float s, unused;
  warp_rows_dot<BF16, false, ROWS_PER_WARP>(At, row0, nrows, w, lane, slot[warp], nullptr, s,
                                            unused);
  if (lane < nrows) out[row0 + lane] = s;
}

// Stencil kernel: gR = B^T grad phi~(B f~) with f~ = f_cur + theta (f_cur - f_prev)
// (theta = 0, f_prev = f_cur: the plain SHOITV gradient, step a4).
__global__ void __launch_bounds__(PW_THREADS) k_stencil(int n, const float* __restrict__ f_cur,
                                                        const float* __restrict__ f_prev,
                                                        float theta, float lam1, float lam2,
                                                        float eps, float* __restrict__ out) {
  __shared__ StencilSmem S;
  const int ntx = st_tiles_x(n);
  stencil_tile(S, f_cur, f_prev, theta, (blockIdx.x / ntx) * ST_R, (blockIdx.x % ntx) * ST_C, n,
               lam1, lam2, eps, out, false);
}

// Regulariser term phi~(B f) (objective, step a6).
__global__ void __launch_bounds__(PW_THREADS) k_reg_term(int n, const float* __restrict__ f,
                                                         float lam1, float lam2, float eps,
                                                         float2* partial, unsigned int* gtick,
                                                         SolverState* st, double* out) {
  __shared__ StencilSmem S;
  const int ntx = st_tiles_x(n);
  const float reg = stencil_tile(S, f, f, 0.f, (blockIdx.x / ntx) * ST_R,
                                 (blockIdx.x % ntx) * ST_C, n, lam1, lam2, eps, nullptr, true);
  const df b = block_sum_acc(reg, 0.f);
  double tot = 0.0;
  if (grid_reduce(partial, gtick, &st->ticket_aux, b, &tot) && threadIdx.x == 0) *out = tot;
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
                                                  float2* partial, unsigned int* gtick,
                                                  SolverState* st, double* actc_out) {
  float h = 0.f, l = 0.f;
  for (int i = blockIdx.x * THREADS + threadIdx.x; i < m; i += gridDim.x * THREADS) {
    acc_add(h, l, g[i], 0.f);
    acc_add(h, l, -gamma[i], 0.f);
  }
  const df b = block_sum_acc(h, l);
  double tot = 0.0;
  if (grid_reduce(partial, gtick, &st->ticket_aux, b, &tot) && threadIdx.x == 0) *actc_out = tot;
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

// Double-float constants of df_log, computed once in extended precision.
struct LogTables {
  cudaError_t err = cudaSuccess;
  LogTables() {
    float th[65], tl[65], l2[2], t3[2], kp[2];
    for (int j = 0; j <= 64; ++j) {
      const long double v = logl(1.0L + (long double)j / 64.0L);
      th[j] = (float)v;
      tl[j] = (float)(v - (long double)th[j]);
    }
    const long double ln2 = logl(2.0L), third = 1.0L / 3.0L;
    l2[0] = (float)ln2;
    l2[1] = (float)(ln2 - (long double)l2[0]);
    t3[0] = (float)third;
    t3[1] = (float)(third - (long double)t3[0]);
    const long double kappa = (long double)KAPPA;
    kp[0] = (float)kappa;
    kp[1] = (float)(kappa - (long double)kp[0]);
    err = cudaMemcpyToSymbol(c_logtab_hi, th, sizeof th);
    if (err == cudaSuccess) err = cudaMemcpyToSymbol(c_logtab_lo, tl, sizeof tl);
    if (err == cudaSuccess) err = cudaMemcpyToSymbol(c_ln2, l2, sizeof l2);
    if (err == cudaSuccess) err = cudaMemcpyToSymbol(c_third, t3, sizeof t3);
    if (err == cudaSuccess) err = cudaMemcpyToSymbol(c_kappa, kp, sizeof kp);
  }
};
cudaError_t ensure_tables() {
  static LogTables t;
  return t.err;
}

}  // namespace

// ------------------------------------------------------------- launchers

int stencil_tiles(int n) { return st_tiles(n); }

int max_partials(int m, int n) {
  const int a = proj_blocks(m) + st_tiles(n);
  const int b = proj_blocks(n * n);
  const int nb = a > b ? a : b;
  return nb + nb / RED_GROUP + 1024;
}
int max_group_tickets(int m, int n) { return max_partials(m, n) / RED_GROUP + 1; }

cudaError_t launch_forward(const FwdArgs& a, cudaStream_t s) {
  cudaError_t e = ensure_tables();
  if (e != cudaSuccess) return e;
  const int grid = proj_blocks(a.A.rows) + (a.loop ? st_tiles(a.n) : 0);
  if (a.use_bf16)
    k_forward<true><<<grid, PW_THREADS, 0, s>>>(a);
  else
    k_forward<false><<<grid, PW_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_pixel(const PixArgs& a, cudaStream_t s) {
  const int grid = proj_blocks(a.At.rows);
  if (a.use_bf16)
    k_pixel<true><<<grid, PW_THREADS, 0, s>>>(a);
  else
    k_pixel<false><<<grid, PW_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_backproject(const DevCSR& At, const float* w, float* out, int use_bf16,
                               cudaStream_t s) {
  const int grid = proj_blocks(At.rows);
  if (use_bf16)
    k_backproject<true><<<grid, PW_THREADS, 0, s>>>(At, w, out);
  else
    k_backproject<false><<<grid, PW_THREADS, 0, s>>>(At, w, out);
  return cudaGetLastError();
}

cudaError_t launch_stencil(int n, const float* f_cur, const float* f_prev, float theta,
                           float lam1, float lam2, float eps, float* out, cudaStream_t s) {
  k_stencil<<<st_tiles(n), PW_THREADS, 0, s>>>(n, f_cur, f_prev, theta, lam1, lam2, eps, out);
  return cudaGetLastError();
}

cudaError_t launch_reg_term(int n, const float* f, float lam1, float lam2, float eps,
                            float2* partial, unsigned int* gtick, SolverState* st, double* out,
                            cudaStream_t s) {
  k_reg_term<<<st_tiles(n), PW_THREADS, 0, s>>>(n, f, lam1, lam2, eps, partial, gtick, st, out);
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
                                 long long npfov, float2* partial, unsigned int* gtick,
                                 SolverState* st, float* f_out, cudaStream_t s) {
  // the ACTc scalar is parked in the last partial slot (as raw bytes of a double)
  double* actc = reinterpret_cast<double*>(partial + max_partials(m, n) - 1);
  k_actc<<<256, THREADS, 0, s>>>(g, gamma, m, partial, gtick, st, actc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_fill_disk<<<(n * n + 255) / 256 < 1024 ? (n * n + 255) / 256 : 1024, 256, 0, s>>>(
      n, n_angles, (int)npfov, actc, f_out);
  return cudaGetLastError();
}

}  // namespace appga
