// Single-slice CUDA kernels of the APPGA hot path (sm_103a).
//
//   k_forward  : y = A f^k, y~ = y + theta_k (y - y^{k-1}) (the projection of
//                f~^k by linearity), w = 1 - g / max(y~ + gamma, kappa gamma),
//                data term of the objective; in the solver loop the same launch
//                also runs the SHOITV stencil of f~^k = f^k + theta_k (f^k -
//                f^{k-1}) (B^T grad phi~(B f~^k)) and the regulariser term of
//                Phi(f^k), leaving per-block objective partials (steps a0, a1,
//                a2, a4, a6; Sec. 2.2, Eq. FidelityTerm, Eq. gradenvL2,
//                Eq. def:phi).  y is accumulated in FP32 in the solver loop and
//                in double-float by the stand-alone projection and objective.
//   k_pixel    : grad F = A^T w through the transposed CSR (no atomics) and the
//                EM-preconditioned projected update f^{k+1} = max(f~ - beta
//                (f^k / Lambda)(grad F + B^T grad phi~), 0) (steps a3, a5;
//                Eq. APPGAiter, Eq. EM)
//   k_finalize : one block: sums the forward phase's objective partials into
//                Phi(f^k) in a fixed order, runs the stopping test, advances
//                the iteration index and loads the next momentum scalar from
//                the FP64 table k_theta_table fills once per run (step a6;
//                Eq. GNtheta)
//
// Projector layouts.  The solver loop streams its matrices in the sliced
// layout (SellGroup): a warp owns a slice of SELL_ROWS rows, SELL_LANES lanes
// per row take the row's 4-entry packs in turn (packed 2-byte columns and
// value quads, PF steps in flight in registers, the next step's gathers
// issued while the current one accumulates), and a butterfly leaves each
// row's sum in all of its lanes.  When A has the quarter-turn symmetry the
// loop streams only its folded halves (FOLD): each stored entry serves two
// products, gathered as pairs (see fold_partner in appga_internal.h).  The
// stand-alone projections and objective stream the row-padded CSR
// (RowGroup): a warp owns R consecutive rows, whose entries form one
// contiguous range streamed in 128-entry chunks; lanes park per-row partials
// in shared-memory slots and lane q sums row q.  No block-wide barrier sits
// on either streaming path.
//
// The per-row epilogue runs on the FP32 pipe only: double-float (FP32 pair)
// arithmetic for y, y~, the guarded denominator, and a double-float natural
// logarithm for the data term -- this part's FP64 pipe is a small fraction of
// its FP32 rate, so FP64 is used only for a handful of scalars per launch.
//
// Kernels read the iteration index and theta from a device-resident
// SolverState, so a captured graph of (k_pixel, k_forward) pairs (the step
// finalisation runs in k_pixel's first blocks) replays without host
// involvement.  Block partials (double-float
// pairs) are combined in a fixed order (k_finalize, or a two-level ticketed
// reduction in the stand-alone calls), so every reduction is deterministic.
#include <cuda_runtime.h>
#include <math.h>

#include <cmath>

#include "appga_internal.h"
#include "device_common.cuh"

namespace appga {
namespace {

constexpr int THREADS = 256;  // setup / reduction kernels

// Projector launch shapes: warps per block (W), consecutive CSR rows per warp
// (R) and 128-entry chunks of the nnz stream in flight per warp (PF), for the
// forward projection (whose grid also runs the stencil tiles) and for the
// transposed one.  Chosen by timing on GB300 (256^2 workload): the forward
// with 4 rows and 2 chunks per warp fits in 56 registers (36 warps per SM),
// the transposed one with 8 rows and 3 chunks in 72 (28 warps per SM).
template <int W_, int R_, int PF_>
struct Shape {
  static constexpr int W = W_, R = R_, PF = PF_;
  static constexpr int THREADS = W_ * 32;
  static constexpr int ROWS = W_ * R_;  // rows per block
};
#ifndef APPGA_FW_W
#define APPGA_FW_W 4
#endif
#ifndef APPGA_FW_RPW
#define APPGA_FW_RPW 4
#endif
#ifndef APPGA_FW_PF
#define APPGA_FW_PF 2
#endif
#ifndef APPGA_PX_W
#define APPGA_PX_W 4
#endif
#ifndef APPGA_PX_RPW
#define APPGA_PX_RPW 8
#endif
#ifndef APPGA_PX_PF
#define APPGA_PX_PF 3
#endif
// the sliced layout's step loop runs whole groups of steps without per-step
// tests (1) or tests every step (0)
#ifndef APPGA_SELL_PEEL
#define APPGA_SELL_PEEL 1
#endif
// steps in flight per warp in the sliced layout's forward and pixel phases
#ifndef APPGA_SELL_FW_PF
#define APPGA_SELL_FW_PF 3
#endif
#ifndef APPGA_SELL_PX_PF
#define APPGA_SELL_PX_PF 4
#endif
// Slices each warp of the sliced projections streams in turn (the loads of
// the next slice are issued before the epilogue of the current one, which
// hides that epilogue's latency); the grids shrink by the same factor.
#ifndef APPGA_FW_SPW
#define APPGA_FW_SPW 1
#endif
#ifndef APPGA_PX_SPW
#define APPGA_PX_SPW 1
#endif
using FW = Shape<APPGA_FW_W, APPGA_FW_RPW, APPGA_FW_PF>;
using PX = Shape<APPGA_PX_W, APPGA_PX_RPW, APPGA_PX_PF>;
// Minimum resident blocks per SM asked of the compiler (a register budget);
// 0 leaves the choice to the compiler, which measured fastest.
#ifndef APPGA_FW_MINB
#define APPGA_FW_MINB 0
#endif
#ifndef APPGA_PX_MINB
#define APPGA_PX_MINB 0
#endif
#if APPGA_FW_MINB > 0
#define FW_BOUNDS __launch_bounds__(FW::THREADS, APPGA_FW_MINB)
#else
#define FW_BOUNDS __launch_bounds__(FW::THREADS)
#endif
#if APPGA_PX_MINB > 0
#define PX_BOUNDS __launch_bounds__(PX::THREADS, APPGA_PX_MINB)
#else
#define PX_BOUNDS __launch_bounds__(PX::THREADS)
#endif
#ifndef APPGA_GPIPE
#define APPGA_GPIPE 1
#endif
#ifndef APPGA_SFIRST
#define APPGA_SFIRST 0
#endif
// forward epilogue once per block (1) or once per warp (0)
#ifndef APPGA_FEPI
#define APPGA_FEPI 1
#endif
// a lane finds the row of its entry by advancing from its previous row (1)
// or by comparing against every row start of the group (0)
#ifndef APPGA_ROWINC
#define APPGA_ROWINC 1
#endif
// row starts of a warp's group kept in shared memory instead of registers
#ifndef APPGA_SBND
#define APPGA_SBND 1
#endif
// accumulation of y = A f in the solver loop: 0 = FP32 (as the back-projection),
// 1 = double-float per product
#ifndef APPGA_LOOP_DF
#define APPGA_LOOP_DF 0
#endif

constexpr int SLOT_W = 33;    // slot row stride: per-row sums read without bank conflicts

// Stencil tiles: ST_R x ST_C pixels, one pixel per thread of a projector block
constexpr int ST_R = FW::W;
constexpr int ST_C = 32;
static_assert(ST_R * ST_C == FW::THREADS, "stencil tile = one pixel per thread");
static_assert(FW::R <= 16 && PX::R <= 16, "row starts of a group: at most 16 in shared memory");
constexpr int TW = ST_C + 4;  // f tile width (halo 2)
constexpr int VW = ST_C + 2;  // v tile width (halo 1)

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
__device__ __forceinline__ float4 gather4(const float* __restrict__ x, int4 c) {
  return make_float4(__ldg(x + c.x), __ldg(x + c.y), __ldg(x + c.z), __ldg(x + c.w));
}

// Row starts of rows row0 .. row0 + nrows held one per lane (lane q <= nrows).
__device__ __forceinline__ int load_raw_bound(const DevCSR& M, int row0, int nrows, int lane) {
  return lane <= nrows ? M.row_ptr[row0 + lane] : 0;
}

// One group of R consecutive CSR rows of M streamed by one warp: the row
// starts, the group's entry range [P0, P1), and PF chunks of the stream in
// flight.  set_bounds + prologue issue the loads; stream() accumulates the
// products into per-lane row partials parked in the warp's shared-memory
// slots; slot_reduce() then sums row q in lane q.
template <bool BF16, bool DF, int R, int PF>
struct RowGroup {
#if APPGA_SBND
  int* sb;  // the warp's row starts in shared memory (INT_MAX past the last row)
#else
  int bnd[R + 1];
#endif
  int nrows, P0, P1;
  int4 c[PF];
  float4 v[PF];

  __device__ __forceinline__ void set_bounds(int braw, int nr) {
    nrows = nr;
#if APPGA_SBND
    const int lane = threadIdx.x & 31;
    if (lane < 4 * ((R + 3) / 4)) sb[lane] = lane < nr ? braw : 0x7fffffff;
    __syncwarp();
    P0 = __shfl_sync(0xffffffffu, braw, 0);
#else
#pragma unroll
    for (int k = 0; k <= R; ++k) bnd[k] = __shfl_sync(0xffffffffu, braw, k <= nr ? k : nr);
    P0 = bnd[0];
#endif
    P1 = __shfl_sync(0xffffffffu, braw, nr);
  }

  // first entry of row q of the group (q < nrows)
  __device__ __forceinline__ int row_start(int q) const {
#if APPGA_SBND
    return sb[q];
#else
    return bnd[q];
#endif
  }

  // row (within the group) of entry p
  __device__ __forceinline__ int row(int p) const {
#if APPGA_SBND
    int q = 0;
#pragma unroll
    for (int i = 0; i < (R + 3) / 4; ++i) {
      const int4 b = reinterpret_cast<const int4*>(sb)[i];
      if (i > 0 && 4 * i < R) q += b.x <= p;
      if (4 * i + 1 < R) q += b.y <= p;
      if (4 * i + 2 < R) q += b.z <= p;
      if (4 * i + 3 < R) q += b.w <= p;
    }
    return q;
#else
    return row_of<R>(p, bnd, nrows);
#endif
  }

  __device__ __forceinline__ void prologue(const DevCSR& M, int lane, uint64_t pol) {
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
  }

  // clears this lane's row slots (before a group is streamed into them)
  __device__ __forceinline__ static void clear_slots(int lane, float* slot_hi, float* slot_lo) {
#pragma unroll
    for (int q = 0; q < R; ++q) {
      slot_hi[q * SLOT_W + lane] = 0.f;
      if (DF) slot_lo[q * SLOT_W + lane] = 0.f;
    }
  }

  __device__ __forceinline__ void stream(const DevCSR& M, const float* __restrict__ x, int lane,
                                         uint64_t pol, float* slot_hi, float* slot_lo) {
    const int nchunks = (P1 - P0 + 127) >> 7;
    float hi = 0.f, lo = 0.f;
    int cur = -1;
#if APPGA_ROWINC
    // row of this lane's current entry (entries only move forward) and the
    // first entry of the row after it (INT_MAX past the last row)
    int q = 0;
    int nxt = nrows > 1 ? row_start(1) : 0x7fffffff;
#endif
#if APPGA_GPIPE
    // x values of the next chunk are gathered one chunk ahead, so the gather
    // latency overlaps the arithmetic of the current chunk
    float4 xg = make_float4(0.f, 0.f, 0.f, 0.f);
    if (P0 + lane * 4 < P1) xg = gather4(x, c[0]);
#endif
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
#if APPGA_GPIPE
          const float4 xx = xg;
          // chunk t + 1 sits in slot (u + 1) % PF (refilled above when PF = 1)
          if (p + 128 < P1) xg = gather4(x, c[(u + 1) % PF]);
#endif
          if (p < P1) {
#if APPGA_ROWINC
            while (p >= nxt) {
              ++q;
              nxt = q + 1 < nrows ? row_start(q + 1) : 0x7fffffff;
            }
#else
            const int q = row(p);
#endif
            if (q != cur) {
              if (cur >= 0) {
                slot_hi[cur * SLOT_W + lane] = hi;
                if (DF) slot_lo[cur * SLOT_W + lane] = lo;
              }
              cur = q;
              hi = 0.f;
              lo = 0.f;
            }
#if APPGA_GPIPE
            const float x0 = xx.x, x1 = xx.y, x2 = xx.z, x3 = xx.w;
            (void)cc;
#else
            const float x0 = __ldg(x + cc.x), x1 = __ldg(x + cc.y);
            const float x2 = __ldg(x + cc.z), x3 = __ldg(x + cc.w);
#endif
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
  }

};

// One slice of the sliced layout (DevSell) streamed by one warp: lane l
// works on row l / SELL_LANES of the slice and takes every SELL_LANES-th pack
// of it, so each step reads 32 consecutive packs (8-byte packed columns and
// 16 values bytes per lane) and no lane has to find the row of its entries.
// PF steps are kept in flight in registers and the gathers of the next step
// are issued while the current one accumulates (two FP32 accumulators per
// lane); the SELL_LANES partial sums of a row are combined by a butterfly,
// which leaves the same row sum in each of its lanes.
#if APPGA_SELL_PACK
using SellCols = uint2;  // one packed word per pack
__device__ __forceinline__ SellCols sell_cols_load(const DevSell& S, int pos, uint64_t pol) {
  return ld_stream_u2(S.cols + pos, pol);
}
__device__ __forceinline__ int4 sell_cols(SellCols c) { return unpack_cols(c); }
__device__ __forceinline__ SellCols sell_cols_zero() { return make_uint2(0u, 0u); }
#else
using SellCols = int4;  // four 32-bit columns per pack
__device__ __forceinline__ SellCols sell_cols_load(const DevSell& S, int pos, uint64_t pol) {
  return ld_stream_i4(reinterpret_cast<const int32_t*>(S.cols32 + pos), pol);
}
__device__ __forceinline__ int4 sell_cols(SellCols c) { return c; }
__device__ __forceinline__ SellCols sell_cols_zero() { return make_int4(0, 0, 0, 0); }
#endif

// The four gathered vector entries of a pack: one float each, or a pair
// (the quarter-turn folded loop gathers two vectors at once).
template <class V>
struct Quad {
  V x, y, z, w;
};
template <class V>
__device__ __forceinline__ Quad<V> gather_quad(const V* __restrict__ x, int4 c) {
  return {__ldg(x + c.x), __ldg(x + c.y), __ldg(x + c.z), __ldg(x + c.w)};
}
template <class V>
__device__ __forceinline__ Quad<V> zero_quad() {
  return {V{}, V{}, V{}, V{}};
}
// Entries 0, 2 of a pack into a0 and 1, 3 into a1.
__device__ __forceinline__ void fma_quad(float4 v, const Quad<float>& g, float& a0, float& a1) {
  a0 = fmaf(v.x, g.x, a0);
  a1 = fmaf(v.y, g.y, a1);
  a0 = fmaf(v.z, g.z, a0);
  a1 = fmaf(v.w, g.w, a1);
}
__device__ __forceinline__ void fma_quad(float4 v, const Quad<float2>& g, float2& a0,
                                         float2& a1) {
  a0.x = fmaf(v.x, g.x.x, a0.x);
  a0.y = fmaf(v.x, g.x.y, a0.y);
  a1.x = fmaf(v.y, g.y.x, a1.x);
  a1.y = fmaf(v.y, g.y.y, a1.y);
  a0.x = fmaf(v.z, g.z.x, a0.x);
  a0.y = fmaf(v.z, g.z.y, a0.y);
  a1.x = fmaf(v.w, g.w.x, a1.x);
  a1.y = fmaf(v.w, g.w.y, a1.y);
}
__device__ __forceinline__ float add_v(float a, float b) { return a + b; }
__device__ __forceinline__ float2 add_v(float2 a, float2 b) {
  return make_float2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ float shfl_xor_v(float a, int o) {
  return __shfl_xor_sync(0xffffffffu, a, o);
}
__device__ __forceinline__ float2 shfl_xor_v(float2 a, int o) {
  return make_float2(__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o));
}

template <bool BF16, int PF>
struct SellGroup {
  int q0, steps;
  SellCols c[PF];
  float4 v[PF];

  __device__ __forceinline__ static float4 vals(const DevSell& S, int pos, uint64_t pol) {
    if constexpr (BF16) {
      const uint2 u = ld_stream_u2(S.vals_bf16 + pos, pol);
      return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                         __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
    } else {
      return ld_stream_f4(reinterpret_cast<const float*>(S.vals + pos), pol);
    }
  }

  // before the kernel waits for its predecessor: the slice's first PF steps
  __device__ __forceinline__ void prologue(const DevSell& S, int slice, int lane, uint64_t pol) {
    q0 = S.off[slice] + lane;
    steps = (S.off[slice + 1] - S.off[slice]) >> 5;
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      c[u] = sell_cols_zero();
      v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (u < steps) {
        c[u] = sell_cols_load(S, q0 + (u << 5), pol);
        v[u] = vals(S, q0 + (u << 5), pol);
      }
    }
  }

  // Row sums of the slice times x (V = float), or times both halves of x
  // (V = float2), in every lane of the row.
  template <class V>
  __device__ __forceinline__ V stream(const DevSell& S, const V* __restrict__ x, uint64_t pol) {
    V a0{}, a1{};
    Quad<V> xg = zero_quad<V>();
    if (steps > 0) xg = gather_quad(x, sell_cols(c[0]));
    int t0 = 0;
#if APPGA_SELL_PEEL
    // whole groups of PF steps whose refills and next gathers all exist: no
    // per-step tests
    for (; t0 + 2 * PF <= steps; t0 += PF) {
#pragma unroll
      for (int u = 0; u < PF; ++u) {
        const int t = t0 + u;
        const float4 vv = v[u];
        c[u] = sell_cols_load(S, q0 + ((t + PF) << 5), pol);
        v[u] = vals(S, q0 + ((t + PF) << 5), pol);
        const Quad<V> xx = xg;
        xg = gather_quad(x, sell_cols(c[(u + 1) % PF]));
        fma_quad(vv, xx, a0, a1);
      }
    }
#endif
    for (; t0 < steps; t0 += PF) {
#pragma unroll
      for (int u = 0; u < PF; ++u) {
        const int t = t0 + u;
        if (t < steps) {
          const float4 vv = v[u];
          if (t + PF < steps) {  // refill this slot with step t + PF
            c[u] = sell_cols_load(S, q0 + ((t + PF) << 5), pol);
            v[u] = vals(S, q0 + ((t + PF) << 5), pol);
          }
          const Quad<V> xx = xg;
          // step t + 1 sits in slot (u + 1) % PF (refilled above when PF = 1)
          if (t + 1 < steps) xg = gather_quad(x, sell_cols(c[(u + 1) % PF]));
          fma_quad(vv, xx, a0, a1);
        }
      }
    }
    V r = add_v(a0, a1);
#pragma unroll
    for (int o = 1; o < SELL_LANES; o <<= 1) r = add_v(r, shfl_xor_v(r, o));
    return r;
  }
};

// Sum of row `lane` of a streamed group in lanes 0..nrows-1 from the warp's
// slots (an accumulator pair if DF).
template <bool DF>
__device__ __forceinline__ void slot_reduce(int lane, int nrows, const float* slot_hi,
                                            const float* slot_lo, float& out_hi, float& out_lo) {
  out_hi = 0.f;
  out_lo = 0.f;
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

// Rows [row0, row0 + nrows) of M times x; returns the sum of row `lane` in
// lanes 0..nrows-1: an accumulator pair if DF, else an FP32 value in out_hi.
// slot_hi / slot_lo: this warp's R*SLOT_W floats each of shared memory.
template <bool BF16, bool DF, int R, int PF>
__device__ __forceinline__ void warp_rows_dot(const DevCSR& M, int row0, int nrows,
                                              const float* __restrict__ x, int lane,
                                              float* slot_hi, float* slot_lo, float& out_hi,
                                              float& out_lo, int* sbnd) {
  out_hi = 0.f;
  out_lo = 0.f;
  if (nrows <= 0) return;
  RowGroup<BF16, DF, R, PF> rg;
#if APPGA_SBND
  rg.sb = sbnd;
#else
  (void)sbnd;
#endif
  rg.set_bounds(load_raw_bound(M, row0, nrows, lane), nrows);
  RowGroup<BF16, DF, R, PF>::clear_slots(lane, slot_hi, slot_lo);
  const uint64_t pol = evict_first_policy();
  rg.prologue(M, lane, pol);
  rg.stream(M, x, lane, pol, slot_hi, slot_lo);
  slot_reduce<DF>(lane, nrows, slot_hi, slot_lo, out_hi, out_lo);
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
template <class SH>
__host__ __device__ __forceinline__ int proj_blocks(int rows) {
  return (rows + SH::ROWS - 1) / SH::ROWS;
}

// Momentum scalar for index k (Eq. GNtheta) -- FP64 on the device.
__device__ double gn_t_dev(int k, double a, double b, double omega) {
  return a * pow((double)k, omega) + b;
}
__device__ __forceinline__ void put_theta(ThetaEntry* e, double theta) {
  e->v = theta;
  e->hi = (float)theta;
  e->lo = (float)(theta - (double)e->hi);
}
__device__ __forceinline__ void load_theta(SolverState* st, const ThetaEntry& e) {
  st->theta = e.v;
  st->theta_hi = e.hi;
  st->theta_lo = e.lo;
}

// ------------------------------------------------------------ k_forward

// Per-row epilogue of the forward phase (steps a1, a2, a6): stores y (and in
// the loop y~ by linearity), the guarded weight w = 1 - g/den (returned, and
// stored at w[row] if store_w), and adds the data term y - g ln(y + gamma) of
// the objective to (acc_hi, acc_lo).
__device__ __forceinline__ float forward_row(const FwdArgs& a, df th, int kk, int row, float hi,
                                             float lo, int& hits, int& bad, float& acc_hi,
                                             float& acc_lo, bool store_w = true) {
  float wv = 0.f;
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
    if (a.loop && !a.fresh_first) {
      // y~ = y + theta (y - y^{k-1}): the projection of f~ by linearity (the
      // first step of a fresh run has f^{k-1} = f^k, so there y~ = y)
      const float2 yp = a.y[(kk + 1) & 1][row];
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
    wv = __fdiv_rn(df_to_f(df_add_f(den, -gg)), df_to_f(den));
    if (store_w) a.w[row] = wv;
    if (!isfinite(wv)) bad = 1;
  }
  if (!isfinite(y.hi)) bad = 1;
  if (a.want_data) {
    // data term y - g ln(y + gamma) (Eq. FidelityTerm), double-float
    const df term = df_add(y, df_neg(df_mul_f(df_log(df_add_f(y, gam)), gg)));
    acc_add(acc_hi, acc_lo, term.hi, term.lo);
  }
  return wv;
}

// Rows per forward block: FW::W warps of FW::R CSR rows, or of one slice of
// SELL_ROWS rows in the sliced layout (per trip of the slice loop).
template <bool SL>
__host__ __device__ __forceinline__ constexpr int fw_block_rows() {
  return SL ? FW::W * SELL_ROWS : FW::ROWS;
}
// Projector blocks of the forward phase over `rows` rows: CSR row groups, or
// sliced with each warp taking APPGA_FW_SPW slices in turn.
__host__ __device__ __forceinline__ int fw_proj_blocks(int rows, bool sliced) {
  if (!sliced) return (rows + FW::ROWS - 1) / FW::ROWS;
  const int ns = (rows + SELL_ROWS - 1) / SELL_ROWS;
  return (ns + FW::W * APPGA_FW_SPW - 1) / (FW::W * APPGA_FW_SPW);
}
// Blocks of the pixel phase over d pixel rows (as fw_proj_blocks).
__host__ __device__ __forceinline__ int px_blocks(int d, bool sliced) {
  if (!sliced) return (d + PX::ROWS - 1) / PX::ROWS;
  const int ns = (d + SELL_ROWS - 1) / SELL_ROWS;
  return (ns + PX::W * APPGA_PX_SPW - 1) / (PX::W * APPGA_PX_SPW);
}

// Blocks [0, nproj) project rows (CSR row groups, or slices of the sliced
// layout when SL); in the solver loop the blocks after them run the stencil
// tiles.
//
// FOLD (quarter-turn folded loop, sliced): the slices hold A's first m/2
// rows; each stored row i gathers the pairs fpair and yields y_i and
// y_{fold_partner(i)}, so the block's 16 stored rows give 32 row epilogues,
// one per lane of warp 0, and w is stored as the pairs the folded
// back-projection gathers.
template <bool BF16, bool DFA, bool SL, bool FOLD>
__global__ void FW_BOUNDS k_forward(FwdArgs a) {
  __shared__ union {
    struct {
      float hi[FW::W][FW::R * SLOT_W];
      float lo[FW::W][FW::R * SLOT_W];
      int4 bnd[FW::W][4];
    } slot;
    StencilSmem st;
  } sm;
  static_assert(!(SL && DFA), "the sliced layout serves the FP32-accumulated projections");
  static_assert(!FOLD || SL, "the folded loop streams the sliced layout");
  pdl_trigger();
  SolverState* st = a.st;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // rows streamed (FOLD: the stored first half)
  const int m = SL ? a.S.rows : a.A.rows;
  constexpr int BROWS = fw_block_rows<SL>();
  const int nproj = fw_proj_blocks(m, SL);
  const int ns = SL ? a.S.slices : 0;
#if APPGA_SFIRST
  // stencil tiles take the first blocks, so the projector blocks end the grid
  const int pb = (int)blockIdx.x - ((int)gridDim.x - nproj);
  const int sb = blockIdx.x;
#else
  const int pb = blockIdx.x;
  const int sb = (int)blockIdx.x - nproj;
#endif
  const bool proj = pb >= 0 && pb < nproj;
  // CSR: this warp's rows; sliced: this warp's first slice
  const int row0 = SL ? (pb * FW::W + warp) * SELL_ROWS : pb * FW::ROWS + warp * FW::R;
  const int nrows = proj ? max(0, min(SL ? SELL_ROWS : FW::R, m - row0)) : 0;
  // The warp's row bounds and first chunks of A: no kernel writes them, so
  // they are fetched before waiting for the previous kernel of the stream.
  RowGroup<BF16, DFA, FW::R, FW::PF> rg;
  SellGroup<BF16, APPGA_SELL_FW_PF> sg;
  uint64_t pol = 0;
  if (proj) pol = evict_first_policy();
  if (nrows > 0) {
    if constexpr (SL) {
      sg.prologue(a.S, pb * FW::W + warp, lane, pol);
    } else {
#if APPGA_SBND
      rg.sb = reinterpret_cast<int*>(sm.slot.bnd[warp]);
#endif
      rg.set_bounds(load_raw_bound(a.A, row0, nrows, lane), nrows);
      decltype(rg)::clear_slots(lane, sm.slot.hi[warp], sm.slot.lo[warp]);
      rg.prologue(a.A, lane, pol);
    }
  }
  pdl_wait();
  int kk = 0;
  df th = {0.f, 0.f};
  if (a.loop) {
    // this step's index and status, handed over by the previous step's
    // finalisation; block 0 publishes them for the pixel phase.  done == 2:
    // the last pixel phase has run and this forward phase only evaluates the
    // objective of the result (uniform over the grid)
    const int dn = st->done_next;
    kk = st->k_next;
    const ThetaEntry te = a.theta_tab[kk - st->k0];
    th = {te.hi, te.lo};
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st->done = dn;
      st->k = kk;
      load_theta(st, te);
    }
    if (dn == 1) return;
  }
  float acc_hi = 0.f, acc_lo = 0.f;  // this thread's share of the objective
  int hits = 0, bad = 0;
  if (proj && SL) {
    // slices pb*W + warp + t*G, t = 0, 1, ...: the block's trip t covers
    // FW::W consecutive slices, whose row sums go to warp 0, so the
    // double-float epilogue (with the logarithm of the data term) runs once
    // per block trip; the next slice's loads are issued before it
    const float* f = a.ft ? a.ft : (a.loop ? a.f[kk % 3] : a.f[0]);
    const int G = nproj * FW::W;
    __shared__ float2 ysum[BROWS];
    for (int base = pb * FW::W; base < ns; base += G) {  // uniform over the block
      const int sl = base + warp;
      const int nr = sl < ns ? min(SELL_ROWS, m - sl * SELL_ROWS) : 0;
      float2 yy = make_float2(0.f, 0.f);  // (y, 0), or FOLD (y, y of the partner row)
      if (nr > 0) {
        if constexpr (FOLD) {
          yy = sg.stream(a.S, a.fpair, pol);
        } else {
          yy.x = sg.stream(a.S, f, pol);
        }
      }
      if (APPGA_FW_SPW > 1 && sl + G < ns) sg.prologue(a.S, sl + G, lane, pol);
      const int wrow = lane / SELL_LANES;
      if ((lane % SELL_LANES) == 0 && wrow < nr) ysum[warp * SELL_ROWS + wrow] = yy;
      __syncthreads();
      if (warp == 0) {
        const int brow0 = base * SELL_ROWS, bn = min(BROWS, m - brow0);
        if constexpr (FOLD) {
          static_assert(!FOLD || BROWS % 16 == 0, "folded row epilogues in passes of 16");
          // per pass, lanes 0-15 take 16 stored rows and lanes 16-31 their
          // partner rows
#pragma unroll
          for (int p0 = 0; p0 < BROWS; p0 += 16) {
            const int q = p0 + lane % 16;
            const bool partner = lane >= 16;
            float wv = 0.f;
            if (q < bn) {
              const float2 v = ysum[q];
              const int row =
                  partner ? fold_partner(brow0 + q, a.fold_half, a.fold_nb) : brow0 + q;
              wv = forward_row(a, th, kk, row, partner ? v.y : v.x, 0.f, hits, bad, acc_hi,
                               acc_lo, false);
            }
            const float wp = __shfl_down_sync(0xffffffffu, wv, 16);
            if (!partner && q < bn && a.w != nullptr)
              reinterpret_cast<float2*>(a.w)[brow0 + q] = make_float2(wv, wp);
          }
        } else {
          for (int q = lane; q < bn; q += 32) {
            const float2 v = ysum[q];
            forward_row(a, th, kk, brow0 + q, v.x, v.y, hits, bad, acc_hi, acc_lo);
          }
        }
      }
      if (APPGA_FW_SPW == 1) break;  // one trip: the grid covers every slice
      __syncthreads();  // ysum is refilled by the next trip
    }
  } else if (proj) {
    // the tiled copy when given (the solver's projections), else the image
    const float* f = a.ft ? a.ft : (a.loop ? a.f[kk % 3] : a.f[0]);
    float hi = 0.f, lo = 0.f;
    if (nrows > 0) {
      rg.stream(a.A, f, lane, pol, sm.slot.hi[warp], sm.slot.lo[warp]);
      slot_reduce<DFA>(lane, nrows, sm.slot.hi[warp], sm.slot.lo[warp], hi, lo);
    }
#if APPGA_FEPI
    // the block's row sums go to warp 0, so the double-float epilogue runs
    // once per block, not once per warp
    __shared__ float2 ysum_csr[BROWS];
    if (lane < nrows) ysum_csr[warp * FW::R + lane] = make_float2(hi, lo);
    __syncthreads();
    if (warp == 0) {
      const int brow0 = pb * BROWS, bn = min(BROWS, m - brow0);
      for (int q = lane; q < bn; q += 32) {
        const float2 v = ysum_csr[q];
        forward_row(a, th, kk, brow0 + q, v.x, v.y, hits, bad, acc_hi, acc_lo);
      }
    }
#else
    if (lane < nrows) forward_row(a, th, kk, row0 + lane, hi, lo, hits, bad, acc_hi, acc_lo);
#endif
  } else {
    // SHOITV gradient at f~^kk and the regulariser of Phi(f^kk)
    const int b = sb;
    const int ntx = st_tiles_x(a.n);
    const float reg = stencil_tile(sm.st, a.f[kk % 3], a.f[(kk + 2) % 3], th.hi,
                                   (b / ntx) * ST_R, (b % ntx) * ST_C, a.n, a.ip.lambda1,
                                   a.ip.lambda2, a.ip.eps, a.gR, a.want_data != 0);
    acc_hi = reg;
  }
  warp_count_add(&st->guard_hits, hits);
  warp_flag_or(&st->flags, bad ? APPGA_FLAG_NONFINITE : 0);
  if (!a.want_data) return;
  const df bsum = block_sum_acc(acc_hi, acc_lo);
  if (a.loop) {
    // the pixel phase of this step reduces the block partials and runs the
    // stopping test, so no grid-wide ordering is needed here
    if (threadIdx.x == 0) a.partial[blockIdx.x] = make_float2(bsum.hi, bsum.lo);
    return;
  }
  double tot = 0.0;
  if (grid_reduce(a.partial, a.gtick, &st->ticket_r, bsum, &tot)) {
    if (threadIdx.x == 0) {
      if (a.data_out) *a.data_out = tot;
    }
  }
}

// -------------------------------------------------------------- k_pixel

// EM-preconditioned projected update of pixel j (Eq. EM, Eq. cloformproiota)
// given the back-projection bp = (A^T w)_j; returns the preconditioner entry
// and leaves f_j^{k+1} in fn.
__device__ __forceinline__ float pixel_update(const PixArgs& a, int kk, int j, float bp,
                                              int& bad, float& fn_out) {
  const float* fk = a.f[kk % 3];
  const float vk = fk[j];
  const float ft = fmaf(a.st->theta_hi, vk - a.f[(kk + 2) % 3][j], vk);
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
  const float fn = fmaxf(xv, 0.f);
  a.f[(kk + 1) % 3][j] = fn;
  if (a.ft) a.ft[tiled_index(j / a.n, j % a.n, a.n)] = fn;  // the next forward's gathers
  fn_out = fn;
  return p;
}

// Step finalisation (step a6) after the forward phase of step kk, given
// Phi(f^kk) if tracked: stopping test, then the index and run status of the
// next forward phase (k_next, done_next).  One thread.
__device__ void finish_step(const PixArgs& a, SolverState* st, int kk, double phi) {
  if (a.ip.track) {
    const double prev = st->phi_cur;
    st->phi_prev = prev;
    st->phi_cur = phi;
    if (a.ip.rel_tol > 0.0 && kk > st->k0 && fabs(phi - prev) <= a.ip.rel_tol * fabs(prev)) {
      // f^kk is the result; the f^{kk+1} the pixel phase writes is not used
      st->done_next = 1;
      st->result_k = kk;
      st->stopped_early = 1;
      return;
    }
  }
  if (kk >= st->k_last) {
    // with the objective tracked, the forward phase of f^{kk+1} still runs
    // and a last finalisation turns its partials into Phi(f^{kk+1})
    st->done_next = a.ip.track ? 2 : 1;
    st->result_k = kk + 1;
  }
  st->k_next = kk + 1;
}

// The step finalisation inside the pixel phase (PixArgs::fuse_fin): the
// forward phase's block partials are summed in fixed groups of RED_GROUP by
// the pixel phase's first blocks (each group in index order), and the last
// of them to finish sums the group results in order and finalises the step.
// These blocks run first, so the reduction overlaps the rest of the phase
// instead of adding a serial tail or a launch.
__device__ void fused_finalize(const PixArgs& a, SolverState* st, int kk) {
  if (!a.ip.track) {
    if (blockIdx.x == 0 && threadIdx.x == 0) finish_step(a, st, kk, 0.0);
    return;
  }
  __shared__ int s_last;
  const int np = a.n_fwd_partial;
  const int ng = (np + RED_GROUP - 1) / RED_GROUP;
  for (int g = blockIdx.x; g < ng; g += gridDim.x) {  // uniform over the block
    float h = 0.f, l = 0.f;
    const int gsize = min(RED_GROUP, np - g * RED_GROUP);
    for (int i = threadIdx.x; i < gsize; i += blockDim.x) {
      const float2 v = __ldcg(a.fwd_partial + g * RED_GROUP + i);
      acc_add(h, l, v.x, v.y);
    }
    const df gs = block_sum_acc(h, l);
    if (threadIdx.x == 0) {
      a.partial[g] = make_float2(gs.hi, gs.lo);
      __threadfence();
      s_last = (atomicAdd(&st->ticket_p, 1u) == (unsigned)(ng - 1));
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      h = 0.f;
      l = 0.f;
      for (int i = threadIdx.x; i < ng; i += blockDim.x) {
        const float2 v = __ldcg(a.partial + i);
        acc_add(h, l, v.x, v.y);
      }
      const df t = block_sum_acc(h, l);
      if (threadIdx.x == 0) {
        st->ticket_p = 0u;
        finish_step(a, st, kk, (double)t.hi + (double)t.lo);
      }
    }
    __syncthreads();
  }
}


// FOLD (quarter-turn folded loop, sliced): warp o streams the folded A^T
// rows of orbit o's four pixels q_r = turn^r(q_0), one per SELL_LANES lanes,
// gathering the w pairs; (A^T w)_{q_r} = s1(q_r) + s2(q_{r-1}), the second
// term from the lanes of member r-1, and f^{k+1} at q_r goes out with its
// turned neighbour f^{k+1} at q_{r+1} as the next forward phase's pair.
template <bool BF16, bool SL, bool FOLD>
__global__ void PX_BOUNDS k_pixel(PixArgs a) {
  __shared__ float slot[PX::W][PX::R * SLOT_W];
  __shared__ int4 sbnd[PX::W][4];
  static_assert(!FOLD || (SL && SELL_ROWS % 4 == 0), "a folded slice is whole orbits of four");
  pdl_trigger();
  SolverState* st = a.st;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int d = a.At.rows;
  // CSR: this warp's pixel rows; sliced: this warp's slice
  const int j0 = SL ? (blockIdx.x * PX::W + warp) * SELL_ROWS : blockIdx.x * PX::ROWS + warp * PX::R;
  const int np = max(0, min(SL ? SELL_ROWS : PX::R, d - j0));
  // row bounds and first chunks of A^T before waiting (no kernel writes them)
  RowGroup<BF16, false, PX::R, PX::PF> rg;
  SellGroup<BF16, APPGA_SELL_PX_PF> sg;
  uint64_t pol = evict_first_policy();
  if (np > 0) {
    if constexpr (SL) {
      sg.prologue(a.S, blockIdx.x * PX::W + warp, lane, pol);
    } else {
#if APPGA_SBND
      rg.sb = reinterpret_cast<int*>(sbnd[warp]);
#endif
      rg.set_bounds(load_raw_bound(a.At, j0, np, lane), np);
      decltype(rg)::clear_slots(lane, slot[warp], nullptr);
      rg.prologue(a.At, lane, pol);
    }
  }
  pdl_wait();
  if (st->done) return;  // uniform over the grid
  const int kk = st->k;
  if (a.fuse_fin) fused_finalize(a, st, kk);
  int bad = 0;
  float pmax = 0.f;  // largest preconditioner entry this lane met
  if constexpr (SL) {
    // slices blockIdx.x * W + warp + t*G, t = 0, 1, ... (warp-uniform); the
    // next slice's loads are issued before this slice's pixel updates
    const int ns = a.S.slices, G = gridDim.x * PX::W;
    for (int sl = blockIdx.x * PX::W + warp; sl < ns; sl += G) {
      const int npr = min(SELL_ROWS, d - sl * SELL_ROWS);
      float bp;
      int j = -1;  // the pixel whose update this lane makes
      int jr = 0, jc = 0;
      if constexpr (FOLD) {
        const float2 sp = sg.stream(a.S, reinterpret_cast<const float2*>(a.w), pol);
        if (APPGA_PX_SPW > 1 && sl + G < ns) sg.prologue(a.S, sl + G, lane, pol);
        // row q of the slice is member q % 4 of orbit sl * SELL_ROWS / 4 + q / 4;
        // member q - 1 (mod 4) of its orbit sits in row qm (a last slice may
        // hold fewer orbits: npr rows)
        const int q = lane / SELL_LANES, sub = lane % SELL_LANES;
        const int qm = (q & ~3) | ((q + 3) & 3);
        const float s2 = __shfl_sync(0xffffffffu, sp.y, qm * SELL_LANES + sub);
        bp = sp.x + s2;
        if (sub == 0 && q < npr) {
          orbit_pixel(sl * (SELL_ROWS / 4) + q / 4, q & 3, a.n, &jr, &jc);
          j = jr * a.n + jc;
        }
      } else {
        bp = sg.stream(a.S, a.w, pol);
        if (APPGA_PX_SPW > 1 && sl + G < ns) sg.prologue(a.S, sl + G, lane, pol);
        if ((lane % SELL_LANES) == 0 && lane / SELL_LANES < npr)
          j = sl * SELL_ROWS + lane / SELL_LANES;
      }
      float fn = 0.f;
      if (j >= 0) pmax = fmaxf(pmax, pixel_update(a, kk, j, bp, bad, fn));
      if constexpr (FOLD) {
        // member q + 1 (mod 4) of the orbit: row qp
        const int qp = ((lane / SELL_LANES) & ~3) | ((lane / SELL_LANES + 1) & 3);
        const float fturn = __shfl_sync(0xffffffffu, fn, qp * SELL_LANES + lane % SELL_LANES);
        if (j >= 0) a.fpair[tiled_index(jr, jc, a.n)] = make_float2(fn, fturn);
      }
      if (APPGA_PX_SPW == 1) break;  // one trip: the grid covers every slice
    }
  } else {
    float bp = 0.f, unused = 0.f;
    if (np > 0) {
      rg.stream(a.At, a.w, lane, pol, slot[warp], nullptr);
      slot_reduce<false>(lane, np, slot[warp], nullptr, bp, unused);
    }
    float fn = 0.f;
    if (lane < np) pmax = fmaxf(pmax, pixel_update(a, kk, j0 + lane, bp, bad, fn));
  }
  if (a.want_pmax) {
    // largest preconditioner entry of this step (order-independent)
    const unsigned pm = __reduce_max_sync(0xffffffffu, __float_as_uint(pmax));
    if (lane == 0 && pm > 0u) atomicMax(&st->pmax_bits, pm);
  }
  warp_flag_or(&st->flags, bad ? APPGA_FLAG_NONFINITE : 0);
}

// Finalises a step after the pixel phase, in one block (so the pixel blocks
// end without a grid-wide ticket): Phi(f^kk) from the forward phase's block
// partials in a fixed order and the stopping test, the AFPPA dual step sizes,
// then the next index and its momentum scalar from the run's table.
constexpr int FIN_THREADS = 512;
#ifndef APPGA_FIN_BATCH
#define APPGA_FIN_BATCH 12
#endif
constexpr int FIN_BATCH = APPGA_FIN_BATCH;  // independent loads in flight per thread
__global__ void __launch_bounds__(FIN_THREADS) k_finalize(PixArgs a) {
  pdl_trigger();
  pdl_wait();
  SolverState* st = a.st;
  const int state = st->done;  // uniform over the block
  if (state == 1) return;
  const int kk = st->k;
  df phi = {0.f, 0.f};
  if (a.ip.track) {
    float h = 0.f, l = 0.f;
    for (int i0 = 0; i0 < a.n_fwd_partial; i0 += FIN_THREADS * FIN_BATCH) {
      float2 v[FIN_BATCH];
#pragma unroll
      for (int u = 0; u < FIN_BATCH; ++u) {
        const int i = i0 + u * FIN_THREADS + threadIdx.x;
        v[u] = i < a.n_fwd_partial ? a.fwd_partial[i] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < FIN_BATCH; ++u) acc_add(h, l, v[u].x, v[u].y);
    }
    phi = block_sum_acc(h, l);
  }
  if (threadIdx.x != 0) return;
  if (state == 2) {
    // after the run's last forward phase: Phi of the result, f^{result_k}
    st->phi_prev = st->phi_cur;
    st->phi_cur = (double)phi.hi + (double)phi.lo;
    st->done = 1;
    st->done_next = 1;
    return;
  }
  if (a.ip.track) {
    const double cur = (double)phi.hi + (double)phi.lo;
    const double prev = st->phi_cur;
    st->phi_prev = prev;
    st->phi_cur = cur;
    if (a.ip.rel_tol > 0.0 && kk > st->k0 && fabs(cur - prev) <= a.ip.rel_tol * fabs(prev)) {
      // f^kk is the result; the f^{kk+1} the pixel phase wrote is not used
      st->done = 1;
      st->done_next = 1;
      st->result_k = kk;
      st->stopped_early = 1;
      return;
    }
  }
  if (a.want_pmax) {
    // dual step sizes of this step: rho1 = 1/(2*8*p_max), rho2 = 1/(2*64*p_max)
    // (kept when every entry is zero: the all-zero iterate is absorbing)
    const float pm = __uint_as_float(st->pmax_bits);
    if (pm > 0.f) {
      st->rho1 = (float)(1.0 / (16.0 * (double)pm));
      st->rho2 = (float)(1.0 / (128.0 * (double)pm));
    }
    st->pmax_bits = 0u;
  }
  st->theta_prev = st->theta_hi;
  if (kk >= st->k_last) {
    // with the objective tracked, the forward phase of f^{kk+1} still runs
    // and a last finalisation turns its partials into Phi(f^{kk+1})
    st->done = a.ip.track ? 2 : 1;
    st->done_next = st->done;
    st->result_k = kk + 1;
  }
  st->k = kk + 1;
  st->k_next = kk + 1;
  load_theta(st, a.theta_tab[kk + 1 - st->k0]);  // kk + 1 <= k_last + 1
}

// Momentum scalars of a whole run, tab[i] = theta_{k0+i} for i <= n, in
// FP64: Eq. GNtheta with one thread per index, or Nesterov's recursion
// t_k = (1 + sqrt(1 + 4 t_{k-1}^2)) / 2 from t_0 = 1 in one thread; and
// theta_{k0} into the state.  Precomputed because an FP64 pow() in the
// per-step finalisation costs several microseconds on this part.  A resumed
// run computes the same values, so it replays an uninterrupted one bit for bit.
__global__ void k_theta_table(SolverState* st, ThetaEntry* tab, int k0, int n, int momentum,
                              double a, double b, double omega, SolverState init, int set_state) {
  pdl_wait();  // launched dependent: nothing is touched before the predecessor is done
  pdl_trigger();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && set_state) *st = init;
  if (momentum == APPGA_MOMENTUM_NESTEROV) {
    if (i != 0) return;
    double t = 1.0;
    for (int k = 1; k <= k0 + n; ++k) {
      const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
      if (k >= k0) put_theta(&tab[k - k0], (t - 1.0) / tn);
      t = tn;
    }
  } else if (i <= n) {
    const int k = k0 + i;
    put_theta(&tab[i], momentum == APPGA_MOMENTUM_GN
                           ? (gn_t_dev(k - 1, a, b, omega) - 1.0) / gn_t_dev(k, a, b, omega)
                           : 0.0);
  }
  if (i == 0) load_theta(st, tab[0]);
}

// Standalone back-projection (step a3): out = A^T w.
template <bool BF16>
__global__ void __launch_bounds__(PX::THREADS) k_backproject(DevCSR At, const float* __restrict__ w,
                                                            float* __restrict__ out) {
  __shared__ float slot[PX::W][PX::R * SLOT_W];
  __shared__ int4 sbnd[PX::W][4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row0 = blockIdx.x * PX::ROWS + warp * PX::R;
  const int nrows = max(0, min(PX::R, At.rows - row0));
  float s, unused;
  warp_rows_dot<BF16, false, PX::R, PX::PF>(At, row0, nrows, w, lane, slot[warp], nullptr, s,
                                            unused, reinterpret_cast<int*>(sbnd[warp]));
  if (lane < nrows) out[row0 + lane] = s;
}

// Stencil kernel: gR = B^T grad phi~(B f~) with f~ = f_cur + theta (f_cur - f_prev)
// (theta = 0, f_prev = f_cur: the plain SHOITV gradient, step a4).
__global__ void __launch_bounds__(FW::THREADS) k_stencil(int n, const float* __restrict__ f_cur,
                                                        const float* __restrict__ f_prev,
                                                        float theta, float lam1, float lam2,
                                                        float eps, float* __restrict__ out) {
  __shared__ StencilSmem S;
  const int ntx = st_tiles_x(n);
  stencil_tile(S, f_cur, f_prev, theta, (blockIdx.x / ntx) * ST_R, (blockIdx.x % ntx) * ST_C, n,
               lam1, lam2, eps, out, false);
}

// Regulariser term phi~(B f) (objective, step a6).
__global__ void __launch_bounds__(FW::THREADS) k_reg_term(int n, const float* __restrict__ f,
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

// Input check of a solver run: marks the run state with APPGA_FLAG_DOMAIN and
// ends the run (done = 1) if some g_i is negative or not finite, some gamma_i
// is not positive or not finite, or an entry of f_a / f_b (may be NULL) is
// negative or not finite.  No host round trip: the host reads the flag with
// the final state.
__device__ __forceinline__ bool bad_counts(float gi, float ci) {
  return !(isfinite(gi) && gi >= 0.f && isfinite(ci) && ci > 0.f);
}
__device__ __forceinline__ void mark_domain(SolverState* st) {
  atomicOr(&st->flags, APPGA_FLAG_DOMAIN);
  st->done = 1;
  st->done_next = 1;
}
__global__ void k_check_inputs(const float* __restrict__ g, const float* __restrict__ gamma,
                               int m, const float* __restrict__ fa,
                               const float* __restrict__ fb, int d, SolverState* st) {
  pdl_wait();
  pdl_trigger();
  int bad = 0;
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride)
    bad |= bad_counts(g[i], gamma[i]) ? 1 : 0;
  for (int q = 0; q < 2; ++q) {
    const float* f = q == 0 ? fa : fb;
    if (f == nullptr) continue;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += stride) {
      const float x = f[i];
      if (!(isfinite(x) && x >= 0.f)) bad = 1;
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) mark_domain(st);
}

// Initial image (Sec. 4.1): TMC * 1_disk, TMC = (sum g - sum gamma)/(NPFOV * NPA).
// With vst set, the same pass checks g and gamma for a solver run (as
// k_check_inputs does).
__global__ void __launch_bounds__(THREADS) k_actc(const float* __restrict__ g,
                                                  const float* __restrict__ gamma, int m,
                                                  float2* partial, unsigned int* gtick,
                                                  SolverState* st, double* actc_out,
                                                  SolverState* vst) {
  pdl_wait();
  pdl_trigger();
  float h = 0.f, l = 0.f;
  int bad = 0;
  for (int i = blockIdx.x * THREADS + threadIdx.x; i < m; i += gridDim.x * THREADS) {
    const float gi = g[i], ci = gamma[i];
    acc_add(h, l, gi, 0.f);
    acc_add(h, l, -ci, 0.f);
    bad |= bad_counts(gi, ci) ? 1 : 0;
  }
  if (vst != nullptr && __syncthreads_or(bad) && threadIdx.x == 0) mark_domain(vst);
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
// f_out (and f_out2, ft, fpair if not NULL; ft and fpair in the 8 x 8-tiled
// pixel order; the disk test is invariant under the quarter turn, so a
// folded pair holds the value twice)
__global__ void k_fill_disk(int n, int n_angles, int npfov, const double* actc, float* f_out,
                            float* f_out2, float* ft, float2* fpair) {
  pdl_wait();
  pdl_trigger();
  const double tmc = *actc / ((double)npfov * (double)n_angles);
  const float v = (float)tmc;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n * n; j += gridDim.x * blockDim.x) {
    const int r = j / n, c = j % n;
    const float x = in_disk(r, c, n) ? v : 0.f;
    f_out[j] = x;
    if (f_out2) f_out2[j] = x;
    if (ft) ft[tiled_index(r, c, n)] = x;
    if (fpair) fpair[tiled_index(r, c, n)] = make_float2(x, x);
  }
}

// Result of a solver run: out = f^{result_k} and out_prev = f^{result_k - 1}
// (may be NULL) from the iterate ring, unless the inputs failed the check.
__global__ void k_copy_result(const SolverState* st, const float* __restrict__ f0,
                              const float* __restrict__ f1, const float* __restrict__ f2,
                              float* __restrict__ out, float* __restrict__ out_prev, int d) {
  pdl_wait();
  pdl_trigger();
  if (st->flags & APPGA_FLAG_DOMAIN) return;
  const int rk = st->result_k;
  const float* ring[3] = {f0, f1, f2};
  const float* cur = ring[rk % 3];
  const float* prv = ring[(rk + 2) % 3];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d; j += gridDim.x * blockDim.x) {
    out[j] = cur[j];
    if (out_prev) out_prev[j] = prv[j];
  }
}

}  // namespace

__global__ void k_to_tiled(const float* __restrict__ f, float* __restrict__ ft, int n) {
  const int d = n * n;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d; j += gridDim.x * blockDim.x)
    ft[tiled_index(j / n, j % n, n)] = f[j];
}

__global__ void k_to_fold_pairs(const float* __restrict__ f, float2* __restrict__ fpair, int n) {
  const int d = n * n;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d; j += gridDim.x * blockDim.x)
    fpair[tiled_index(j / n, j % n, n)] = make_float2(f[j], f[quarter_turn(j, n)]);
}

// ------------------------------------------------------------- launchers

// The solver loop's forward projection gathers f^k from a copy in the 8 x 8-
// tiled pixel order (1): a ray crosses image rows, and tiles keep the pixels
// it meets close in memory; 0 gathers from the row-major iterate.
#ifndef APPGA_TILED_GATHER
#define APPGA_TILED_GATHER 1
#endif
bool tiled_gather_enabled() { return APPGA_TILED_GATHER != 0; }

cudaError_t launch_to_tiled(const float* f, float* ft, int n, cudaStream_t s) {
  const int d = n * n;
  const int grid = (d + 255) / 256 < 1024 ? (d + 255) / 256 : 1024;
  k_to_tiled<<<grid, 256, 0, s>>>(f, ft, n);
  return cudaGetLastError();
}

cudaError_t launch_to_fold_pairs(const float* f, float2* fpair, int n, cudaStream_t s) {
  const int d = n * n;
  const int grid = (d + 255) / 256 < 1024 ? (d + 255) / 256 : 1024;
  k_to_fold_pairs<<<grid, 256, 0, s>>>(f, fpair, n);
  return cudaGetLastError();
}

// The solver loop's kernels are launched with programmatic stream
// serialisation (1), so each may start while its predecessor drains; 0 gives
// plain stream order.
#ifndef APPGA_PDL
#define APPGA_PDL 1
#endif
// Preferred shared-memory carveout of the projector kernels in percent of the
// unified L1 / shared memory (-1: the driver's choice).  The projectors need
// little shared memory; the rest serves as L1 for the gathered vectors.
// Measured on GB300: 31 % for the forward kernel (the 100 KB configuration
// for its 9 resident blocks) is 2.3 us faster than the driver's choice; the
// back-projection is fastest with the driver's choice.
#ifndef APPGA_CARVEOUT_FW
#define APPGA_CARVEOUT_FW 31
#endif
#ifndef APPGA_CARVEOUT_PX
#define APPGA_CARVEOUT_PX -1
#endif
namespace {
template <class K>
cudaError_t set_carveout(K kern, int percent) {
  if (percent < 0) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, percent);
}
template <class... P, class... Args>
cudaError_t launch_dep(void (*kern)(P...), int grid, int block, cudaStream_t s, Args... args) {
#if APPGA_PDL
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr{};
  attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr.val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
#else
  kern<<<grid, block, 0, s>>>(args...);
  return cudaGetLastError();
#endif
}
}  // namespace

int stencil_tiles(int n) { return st_tiles(n); }
int forward_blocks_of(int m, int n, bool sliced, bool stencil) {
  return fw_proj_blocks(m, sliced) + (stencil ? st_tiles(n) : 0);
}
int forward_blocks(int m, int n, bool sliced) { return forward_blocks_of(m, n, sliced, true); }

int max_partials(int m, int n) {
  const int a = proj_blocks<FW>(m) + st_tiles(n);
  const int b = proj_blocks<PX>(n * n);
  const int nb = a > b ? a : b;
  return nb + nb / RED_GROUP + 1024;
}
int max_group_tickets(int m, int n) { return max_partials(m, n) / RED_GROUP + 1; }

cudaError_t launch_forward(const FwdArgs& a, cudaStream_t s) {
  cudaError_t e = ensure_tables();
  if (e != cudaSuccess) return e;
  const int grid = proj_blocks<FW>(a.A.rows) + (a.loop && !a.no_stencil ? st_tiles(a.n) : 0);
  // the solver (its loop and its projection of the previous iterate)
  // accumulates y in FP32; the stand-alone projection and objective calls
  // in double-float
  const bool dfa = (a.loop || a.solver_acc) ? APPGA_LOOP_DF != 0 : true;
  static PerDeviceOnce carve_once;
  const cudaError_t carve = carve_once.run([] {
    cudaError_t r = set_carveout(k_forward<true, true, false, false>, APPGA_CARVEOUT_FW);
    if (r == cudaSuccess) r = set_carveout(k_forward<true, false, false, false>, APPGA_CARVEOUT_FW);
    if (r == cudaSuccess) r = set_carveout(k_forward<false, true, false, false>, APPGA_CARVEOUT_FW);
    if (r == cudaSuccess) r = set_carveout(k_forward<false, false, false, false>, APPGA_CARVEOUT_FW);
    if (r == cudaSuccess) r = set_carveout(k_forward<true, false, true, false>, APPGA_CARVEOUT_FW);
    if (r == cudaSuccess) r = set_carveout(k_forward<false, false, true, false>, APPGA_CARVEOUT_FW);
    if (r == cudaSuccess) r = set_carveout(k_forward<true, false, true, true>, APPGA_CARVEOUT_FW);
    if (r == cudaSuccess) r = set_carveout(k_forward<false, false, true, true>, APPGA_CARVEOUT_FW);
    return r;
  });
  if (carve != cudaSuccess) return carve;
  // the sliced layout serves the solver's FP32-accumulated projections
  if (a.S.off != nullptr && !dfa) {
    const int sgrid = forward_blocks_of(a.S.rows, a.n, true, a.loop && !a.no_stencil);
    if (a.fpair != nullptr)
      return a.use_bf16 ? launch_dep(k_forward<true, false, true, true>, sgrid, FW::THREADS, s, a)
                        : launch_dep(k_forward<false, false, true, true>, sgrid, FW::THREADS, s, a);
    return a.use_bf16 ? launch_dep(k_forward<true, false, true, false>, sgrid, FW::THREADS, s, a)
                      : launch_dep(k_forward<false, false, true, false>, sgrid, FW::THREADS, s, a);
  }
  if (a.fpair != nullptr) return cudaErrorInvalidValue;  // the folded loop is sliced
  if (a.use_bf16)
    return dfa ? launch_dep(k_forward<true, true, false, false>, grid, FW::THREADS, s, a)
               : launch_dep(k_forward<true, false, false, false>, grid, FW::THREADS, s, a);
  return dfa ? launch_dep(k_forward<false, true, false, false>, grid, FW::THREADS, s, a)
             : launch_dep(k_forward<false, false, false, false>, grid, FW::THREADS, s, a);
}

cudaError_t launch_pixel(const PixArgs& a, cudaStream_t s) {
  static PerDeviceOnce carve_once;
  const cudaError_t carve = carve_once.run([] {
    cudaError_t r = set_carveout(k_pixel<true, false, false>, APPGA_CARVEOUT_PX);
    if (r == cudaSuccess) r = set_carveout(k_pixel<false, false, false>, APPGA_CARVEOUT_PX);
    if (r == cudaSuccess) r = set_carveout(k_pixel<true, true, false>, APPGA_CARVEOUT_PX);
    if (r == cudaSuccess) r = set_carveout(k_pixel<false, true, false>, APPGA_CARVEOUT_PX);
    if (r == cudaSuccess) r = set_carveout(k_pixel<true, true, true>, APPGA_CARVEOUT_PX);
    if (r == cudaSuccess) r = set_carveout(k_pixel<false, true, true>, APPGA_CARVEOUT_PX);
    return r;
  });
  if (carve != cudaSuccess) return carve;
  const bool sl = a.S.off != nullptr;
  const bool fold = a.fpair != nullptr;
  if (fold && (!sl || a.S.rows != a.At.rows || a.n % 2 != 0)) return cudaErrorInvalidValue;
  const int grid = px_blocks(a.At.rows, sl);
  cudaError_t e;
  if (fold)
    e = a.use_bf16 ? launch_dep(k_pixel<true, true, true>, grid, PX::THREADS, s, a)
                   : launch_dep(k_pixel<false, true, true>, grid, PX::THREADS, s, a);
  else if (a.use_bf16)
    e = sl ? launch_dep(k_pixel<true, true, false>, grid, PX::THREADS, s, a)
           : launch_dep(k_pixel<true, false, false>, grid, PX::THREADS, s, a);
  else
    e = sl ? launch_dep(k_pixel<false, true, false>, grid, PX::THREADS, s, a)
           : launch_dep(k_pixel<false, false, false>, grid, PX::THREADS, s, a);
  if (e != cudaSuccess || a.theta_tab == nullptr || a.fuse_fin) return e;
  return launch_dep(k_finalize, 1, FIN_THREADS, s, a);
}

cudaError_t launch_finalize(const PixArgs& a, cudaStream_t s) {
  return launch_dep(k_finalize, 1, FIN_THREADS, s, a);
}

cudaError_t launch_check_inputs(const float* g, const float* gamma, int m, const float* fa,
                                const float* fb, int d, SolverState* st, cudaStream_t s) {
  return launch_dep(k_check_inputs, 256, 256, s, g, gamma, m, fa, fb, d, st);
}

cudaError_t launch_copy_result(const SolverState* st, float* const f[3], float* out,
                               float* out_prev, int d, cudaStream_t s) {
  const int grid = (d + 255) / 256 < 1024 ? (d + 255) / 256 : 1024;
  return launch_dep(k_copy_result, grid, 256, s, st, (const float*)f[0], (const float*)f[1],
                    (const float*)f[2], out, out_prev, d);
}

cudaError_t launch_backproject(const DevCSR& At, const float* w, float* out, int use_bf16,
                               cudaStream_t s) {
  const int grid = proj_blocks<PX>(At.rows);
  if (use_bf16)
    k_backproject<true><<<grid, PX::THREADS, 0, s>>>(At, w, out);
  else
    k_backproject<false><<<grid, PX::THREADS, 0, s>>>(At, w, out);
  return cudaGetLastError();
}

cudaError_t launch_stencil(int n, const float* f_cur, const float* f_prev, float theta,
                           float lam1, float lam2, float eps, float* out, cudaStream_t s) {
  k_stencil<<<st_tiles(n), FW::THREADS, 0, s>>>(n, f_cur, f_prev, theta, lam1, lam2, eps, out);
  return cudaGetLastError();
}

cudaError_t launch_reg_term(int n, const float* f, float lam1, float lam2, float eps,
                            float2* partial, unsigned int* gtick, SolverState* st, double* out,
                            cudaStream_t s) {
  k_reg_term<<<st_tiles(n), FW::THREADS, 0, s>>>(n, f, lam1, lam2, eps, partial, gtick, st, out);
  return cudaGetLastError();
}

cudaError_t launch_validate_inputs(const float* g, const float* gamma, int m, const float* f,
                                   int d, int* flag, cudaStream_t s) {
  k_validate<<<256, 256, 0, s>>>(g, gamma, m, f, d, flag);
  return cudaGetLastError();
}

cudaError_t launch_theta_table(SolverState* st, ThetaEntry* tab, int k0, int n, int momentum,
                               double a, double b, double omega, cudaStream_t s,
                               const SolverState* init) {
  const int threads = 256, blocks = (n + 1 + threads - 1) / threads;
  SolverState z{};
  return launch_dep(k_theta_table, blocks, threads, s, st, tab, k0, n, momentum, a, b, omega,
                    init ? *init : z, init ? 1 : 0);
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
                                 SolverState* st, float* f_out, cudaStream_t s, float* f_out2,
                                 float* ft, SolverState* check_st, float2* fpair) {
  // the ACTc scalar is parked in the last partial slot (as raw bytes of a double)
  double* actc = reinterpret_cast<double*>(partial + max_partials(m, n) - 1);
  cudaError_t e = launch_dep(k_actc, 256, THREADS, s, g, gamma, m, partial, gtick, st,
                             actc, check_st);
  if (e != cudaSuccess) return e;
  return launch_dep(k_fill_disk, (n * n + 255) / 256 < 1024 ? (n * n + 255) / 256 : 1024, 256,
                    s, n, n_angles, (int)npfov, (const double*)actc, f_out, f_out2, ft, fpair);
}

}  // namespace appga
