// Figures of merit of a reconstruction (Sec. 4.1): MSE/PSNR against the
// ground truth, relative contrast of a hot region over a background region
// (RC, NRC), the normalized objective value and the central line profile.
#include <cuda_runtime.h>
#include <math.h>

#include <cmath>
#include <cstdint>

#include "appga.h"
#include "appga_internal.h"
#include "device_common.cuh"
#include "handles.h"

namespace appga {
namespace {

constexpr int FOM_THREADS = 256;
constexpr int FOM_BLOCKS = 304;  // two per SM on GB300; any count is correct
constexpr int FOM_N = 5;         // sums per block: sq. error, f on H, f on B, truth on H, truth on B

// Per-block double-float sums (fixed order inside the block): sum (f - t)^2,
// sum_H f, sum_B f, sum_H t, sum_B t; and the region sizes.
__global__ void __launch_bounds__(FOM_THREADS)
    k_fom_partial(int d, const float* __restrict__ f, const float* __restrict__ t,
                  const uint8_t* __restrict__ roi_h, const uint8_t* __restrict__ roi_b,
                  float2* __restrict__ part, int* __restrict__ cnt) {
  float h[FOM_N], l[FOM_N];
#pragma unroll
  for (int q = 0; q < FOM_N; ++q) h[q] = l[q] = 0.f;
  int nh = 0, nb = 0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d; j += gridDim.x * blockDim.x) {
    const float fv = f[j], tv = t[j];
    df e;
    two_sum(fv, -tv, e.hi, e.lo);  // f - t exactly
    const df sq = df_mul(e, e);
    acc_add(h[0], l[0], sq.hi, sq.lo);
    if (roi_h && roi_h[j]) {
      acc_add(h[1], l[1], fv, 0.f);
      acc_add(h[3], l[3], tv, 0.f);
      ++nh;
    }
    if (roi_b && roi_b[j]) {
      acc_add(h[2], l[2], fv, 0.f);
      acc_add(h[4], l[4], tv, 0.f);
      ++nb;
    }
  }
#pragma unroll
  for (int q = 0; q < FOM_N; ++q) {
    const df s = block_sum_acc(h[q], l[q]);
    if (threadIdx.x == 0) part[blockIdx.x * FOM_N + q] = make_float2(s.hi, s.lo);
  }
  nh = __reduce_add_sync(0xffffffffu, nh);
  nb = __reduce_add_sync(0xffffffffu, nb);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&cnt[blockIdx.x * 2], nh);  // integer sums: order does not matter
    atomicAdd(&cnt[blockIdx.x * 2 + 1], nb);
  }
}

// One block: totals in block order, then the figures in FP64.
__global__ void __launch_bounds__(FOM_THREADS)
    k_fom_final(int d, int nblocks, const float2* __restrict__ part, const int* __restrict__ cnt,
                double max_value, double* __restrict__ out) {
  __shared__ double tot[FOM_N];
  for (int q = 0; q < FOM_N; ++q) {
    float h = 0.f, l = 0.f;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
      const float2 v = part[b * FOM_N + q];
      acc_add(h, l, v.x, v.y);
    }
    const df s = block_sum_acc(h, l);
    if (threadIdx.x == 0) tot[q] = (double)s.hi + (double)s.lo;
  }
  if (threadIdx.x == 0) {
    long long a = 0, b = 0;
    for (int i = 0; i < nblocks; ++i) {
      a += cnt[2 * i];
      b += cnt[2 * i + 1];
    }
    const double mse = tot[0] / (double)d;
    out[0] = mse;
    out[1] = 10.0 * log10(max_value * max_value / mse);
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    double rc = nan, rc_true = nan;
    if (a > 0 && b > 0) {
      const double eh = tot[1] / (double)a, eb = tot[2] / (double)b;
      const double th = tot[3] / (double)a, tb = tot[4] / (double)b;
      rc = fabs(eh - eb) / eb;
      rc_true = fabs(th - tb) / tb;
    }
    out[2] = rc;
    out[3] = rc_true;
    out[4] = rc / rc_true;
    out[5] = (double)a;
    out[6] = (double)b;
  }
}

}  // namespace
}  // namespace appga

using namespace appga;

extern "C" appga_status appga_figures_of_merit(appga_ctx* ctx, int32_t d, const float* f,
                                               const float* f_true, const uint8_t* roi_h,
                                               const uint8_t* roi_b, double max_value,
                                               appga_fom* out_host, void* stream) {
  if (!ctx || !f || !f_true || !out_host) return fail(APPGA_EINVAL, "null argument");
  if (d < 1) return fail(APPGA_EINVAL, "d must be >= 1");
  if (!(max_value > 0.0) || !std::isfinite(max_value))
    return fail(APPGA_EINVAL, "max_value must be finite and > 0");
  if ((roi_h == nullptr) != (roi_b == nullptr))
    return fail(APPGA_EINVAL, "give both regions or neither");
  appga_status rc = enter_stream(ctx, stream);
  if (rc != APPGA_OK) return rc;
  cudaStream_t s = ctx->stream;
  // scratch: partials, counts, results (freed before returning)
  float2* part = nullptr;
  int* cnt = nullptr;
  double* res = nullptr;
  cudaError_t e = cudaMalloc((void**)&part, sizeof(float2) * FOM_BLOCKS * FOM_N);
  if (e == cudaSuccess) e = cudaMalloc((void**)&cnt, sizeof(int) * FOM_BLOCKS * 2);
  if (e == cudaSuccess) e = cudaMalloc((void**)&res, sizeof(double) * 7);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int) * FOM_BLOCKS * 2, s);
  if (e == cudaSuccess) {
    k_fom_partial<<<FOM_BLOCKS, FOM_THREADS, 0, s>>>(d, f, f_true, roi_h, roi_b, part, cnt);
    k_fom_final<<<1, FOM_THREADS, 0, s>>>(d, FOM_BLOCKS, part, cnt, max_value, res);
    e = cudaGetLastError();
  }
  double h[7] = {0, 0, 0, 0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, res, sizeof h, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(part);
  cudaFree(cnt);
  cudaFree(res);
  if (e != cudaSuccess) return cuda_fail(e, "figures of merit");
  out_host->mse = h[0];
  out_host->psnr = h[1];
  out_host->rc = h[2];
  out_host->rc_true = h[3];
  out_host->nrc = h[4];
  out_host->n_roi_h = (int64_t)h[5];
  out_host->n_roi_b = (int64_t)h[6];
  return leave_stream(ctx, stream);
}

extern "C" double appga_nofv(double phi_k, double phi_0, double phi_ref) {
  return (phi_k - phi_ref) / (phi_0 - phi_ref);
}

extern "C" appga_status appga_central_line_profile(appga_ctx* ctx, int32_t n_side, const float* f,
                                                   float* out, void* stream) {
  if (!ctx || !f || !out) return fail(APPGA_EINVAL, "null argument");
  if (n_side < 1) return fail(APPGA_EINVAL, "n_side must be >= 1");
  appga_status rc = enter_stream(ctx, stream);
  if (rc != APPGA_OK) return rc;
  const cudaError_t e = cudaMemcpyAsync(out, f + (size_t)(n_side / 2) * n_side,
                                        sizeof(float) * n_side, cudaMemcpyDeviceToDevice,
                                        ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "central line profile");
  return leave_stream(ctx, stream);
}
