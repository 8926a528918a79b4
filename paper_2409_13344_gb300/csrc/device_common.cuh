// Device helpers shared by the single-slice and the batched kernels:
// streaming loads, double-float arithmetic (including a double-float natural
// logarithm), deterministic reductions and the SHOITV difference forms.
// Included by each CUDA translation unit (internal linkage: every unit keeps
// and initialises its own constant tables).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include <cmath>
#include <mutex>

#include "appga_internal.h"

namespace appga {
namespace {

constexpr int MAX_WARPS = 32;

// ----------------------------------------------------------------- loads

// A and A^T are streamed once per iteration: bypass L1 and tag the lines
// evict-first in L2 (cache-policy operand) so the gathered vectors stay cached.
// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialisation may start while its predecessor in the stream is still
// running: pdl_trigger lets this grid's successor launch once every block of
// this grid has started (or exited), and pdl_wait blocks until the
// predecessor grid has completed with its memory visible.  Before pdl_wait a
// kernel may read only data that no kernel of the stream writes.  Both are
// no-ops for kernels launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

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
__device__ __forceinline__ uint2 ld_stream_u2(const uint2* p, uint64_t pol) {
  uint2 r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u32 {%0,%1}, [%2], %3;"
      : "=r"(r.x), "=r"(r.y)
      : "l"(p), "l"(pol));
  return r;
}
// Columns of one packed 4-entry pack (layout at PACK_BASE_BITS): the base in
// bits 0-19, then three signed 14-bit offsets from it.
__device__ __forceinline__ int4 unpack_cols(uint2 u) {
  const int base = (int)(u.x & 0xfffffu);
  int4 c;
  c.x = base;
  c.y = base + (((int)(((u.x >> 20) | (u.y << 12)) << 18)) >> 18);
  c.z = base + (((int)(u.y << 16)) >> 18);
  c.w = base + (((int)(u.y << 2)) >> 18);
  return c;
}
__device__ __forceinline__ int ld_stream_i1(const int32_t* p, uint64_t pol) {
  int r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(r) : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ float ld_stream_f1(const float* p, uint64_t pol) {
  float r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(r) : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ float ld_stream_bf16_1(const uint16_t* p, uint64_t pol) {
  unsigned short u;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(u) : "l"(p), "l"(pol));
  return __uint_as_float((unsigned)u << 16);
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


// Set-up that a CUDA device needs once (constant tables, function
// attributes): run() calls init with the calling thread's current device and
// returns that device's result on every later call.  Each device of the
// process gets its own set-up.
constexpr int kMaxDevices = 64;
struct PerDeviceOnce {
  std::mutex mu;
  bool done[kMaxDevices] = {};
  cudaError_t err[kMaxDevices] = {};
  template <class F>
  cudaError_t run(F init) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!done[dev]) {
      err[dev] = init();
      done[dev] = true;
    }
    return err[dev];
  }
};

// Streaming multiprocessors of the current device (looked up once per device).
inline int current_sm_count() {
  static std::mutex mu;
  static int sms[kMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 1;
  std::lock_guard<std::mutex> lock(mu);
  if (sms[dev] == 0) {
    int s = 0;
    cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
    sms[dev] = s > 0 ? s : 1;
  }
  return sms[dev];
}

// Double-float constants of df_log, computed in extended precision and
// uploaded to the constant banks of the current device.
cudaError_t upload_log_tables() {
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
  cudaError_t err = cudaMemcpyToSymbol(c_logtab_hi, th, sizeof th);
  if (err == cudaSuccess) err = cudaMemcpyToSymbol(c_logtab_lo, tl, sizeof tl);
  if (err == cudaSuccess) err = cudaMemcpyToSymbol(c_ln2, l2, sizeof l2);
  if (err == cudaSuccess) err = cudaMemcpyToSymbol(c_third, t3, sizeof t3);
  if (err == cudaSuccess) err = cudaMemcpyToSymbol(c_kappa, kp, sizeof kp);
  return err;
}
// The tables of the current device, uploaded on its first use.
cudaError_t ensure_tables() {
  static PerDeviceOnce once;
  return once.run(upload_log_tables);
}


}  // namespace
}  // namespace appga
