// appga_objective_noalloc: the FP64 objective Phi(f) computed with all of
// its scratch memory (block partials of the grid reductions, their tickets,
// a scratch iteration state and two partial sums) in one fixed, file-scope
// device array instead of device memory the library allocates.
//
// Some callers cannot let a library allocate device memory after start-up:
// processes that hand the whole device memory to their own pool at launch
// (a serving process or a framework allocator that owns every byte, where a
// cudaMalloc behind its back fails or fragments the pool), and real-time
// reconstruction loops that forbid allocation once running (cudaMalloc and
// cudaFree can synchronise the device and add latency jitter).  This entry
// point lets them evaluate the objective with only the buffers they pass in
// and the matrix handle they created beforehand.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "appga.h"
#include "appga_internal.h"
#include "handles.h"

namespace {

// Scratch of every appga_objective_noalloc call: 256 KiB, enough for images
// up to 512 x 512 with sinograms up to 263 K bins.  Every GPU that loads the
// library holds this array until the process exits.
constexpr size_t kScratchBytes = 256 * 1024;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};  // device address of g_scratch, per device

// Device address of g_scratch on `device` (looked up once per device, with
// that device current).  In host code g_scratch is only a host-side stand-in
// for the symbol, never a usable device address.
cudaError_t scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_scratch_addr[device] == nullptr) {
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return e;
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

__global__ void k_sum2(const double* parts, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out = parts[0] + parts[1];
}

}  // namespace

extern "C" appga_status appga_objective_noalloc(appga_ctx* ctx, const appga_matrix* mat,
                                                const float* f, const float* g, const float* gamma,
                                                const appga_params* params, double* phi_out,
                                                void* stream) {
  using namespace appga;
  if (!ctx || !mat || !f || !g || !gamma || !params || !phi_out)
    return fail(APPGA_EINVAL, "null argument");
  if (mat->ctx != ctx) return fail(APPGA_EINVAL, "matrix belongs to another context");
  appga_status rc = appga_params_validate(params);
  if (rc != APPGA_OK) return rc;
  // scratch layout: partials | group tickets | state | two partial sums
  const int np = max_partials(mat->m, mat->n);
  const int ng = max_group_tickets(mat->m, mat->n);
  const size_t off_tick = align256((size_t)np * sizeof(float2));
  const size_t off_state = off_tick + align256((size_t)ng * sizeof(unsigned int));
  const size_t off_sums = off_state + align256(sizeof(SolverState));
  const size_t need = off_sums + 2 * sizeof(double);
  if (need > kScratchBytes)
    return fail(APPGA_EINVAL, "appga_objective_noalloc: this matrix needs " + std::to_string(need) +
                                  " bytes of scratch; the fixed scratch holds " +
                                  std::to_string(kScratchBytes) + " (images up to 512 x 512)");
  void* base = nullptr;
  cudaError_t e = scratch_address(ctx->device, &base);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
  e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  auto* bytes = static_cast<unsigned char*>(base);
  auto* partial = reinterpret_cast<float2*>(bytes);
  auto* gtick = reinterpret_cast<unsigned int*>(bytes + off_tick);
  auto* st = reinterpret_cast<SolverState*>(bytes + off_state);
  auto* sums = reinterpret_cast<double*>(bytes + off_sums);
  cudaStream_t s = (cudaStream_t)stream;
  // the tickets and the state start at zero; partials are written before read
  e = cudaMemsetAsync(gtick, 0, off_sums - off_tick, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(scratch)");
  FwdArgs a{};
  a.A = mat->A;
  a.use_bf16 = (params->a_precision == APPGA_PREC_BF16 && mat->has_bf16) ? 1 : 0;
  a.f[0] = f;
  a.g = g;
  a.gamma = gamma;
  a.st = st;
  a.partial = partial;
  a.gtick = gtick;
  a.data_out = sums;
  a.loop = 0;
  a.want_data = 1;
  a.n = mat->n;
  e = launch_forward(a, s);
  if (e == cudaSuccess)
    e = launch_reg_term(mat->n, f, (float)params->lambda1, (float)params->lambda2,
                        (float)params->eps, partial, gtick, st, sums + 1, s);
  if (e == cudaSuccess) {
    k_sum2<<<1, 32, 0, s>>>(sums, phi_out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_fail(e, "appga_objective_noalloc launch");
  return APPGA_OK;
}
