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
// Volumes are slice-major (voxel (z, r, c) at z n^2 + r n + c), so every
// plane of a tile is read and written with coalesced rows.  A block owns an
// 8 x 32 pixel tile and marches along z through a run of slices, keeping
// three planes of f~ and f^k (2-pixel in-plane halo) and three planes of the
// twelve gradient fields (1-pixel halo) in rings: each plane is loaded and
// each field plane computed once per run, so the z-direction costs no halo.
// Blocks are persistent over (tile, z-run) items and leave one row of
// per-slice regulariser sums (double-float pairs, fixed order) each.
//
// The solver keeps its iterates slot-minor ([d][Kp], one slot per slice) for
// the SpMM kernels; two transpose kernels move the current iterate to the
// slice-major ring and the gradient back.
#include <cuda_runtime.h>

#include "appga_internal.h"
#include "batched_internal.h"
#include "device_common.cuh"

namespace appga {
namespace {

constexpr int TR = 8, TC = 32;              // in-plane tile
constexpr int NT = TR * TC;                   // threads: one per tile pixel
constexpr int NWARP = NT / 32;
constexpr int HR = TR + 4, HC = TC + 4;       // f planes, halo 2
constexpr int WR = TR + 2, WC = TC + 2;       // gradient-field planes, halo 1
constexpr int NF = 12;                        // 3 + 9 components
constexpr int MAXZ = 128;                     // slices at most
#ifndef APPGA_VOL_ZRUN
#define APPGA_VOL_ZRUN 16
#endif
constexpr int ZRUN = APPGA_VOL_ZRUN;          // slices per item

// The field planes use the f planes' row stride (HC), so the in-plane index
// of a point is the same in both and neighbouring threads hit distinct banks.
struct Vol3Smem {
  float T[3][HR][HC];        // f~ ring
  float K[3][HR][HC];        // f^k ring (regulariser value)
  float W[3][NF][WR][HC];    // grad phi~ field ring (columns WC.. unused)
  float regv[NT];            // the regulariser of the current plane, one value per thread
  float reg_hi[MAXZ], reg_lo[MAXZ];  // per-slice sums of the block (double-float)
};

__device__ __forceinline__ int ring3(int p) { return (p + 6) % 3; }  // p >= -6

// Which neighbours of a voxel exist: D has a zero first row along each axis,
// so a difference towards a missing neighbour is zero.
struct Edges {
  bool c_lo, c_hi, r_lo, r_hi, z_lo, z_hi;
};

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

// The thirteen neighbours of a point that the twelve components read, loaded
// once into registers from three consecutive planes (m, 0, p) at in-plane
// offset o; X(dz, dr, dc) resolves at compile time.
struct Nbr {
  float v[27];
  __device__ __forceinline__ void load(const float* m, const float* z, const float* p, int o) {
    v[13] = z[o];
    v[12] = z[o - 1];
    v[14] = z[o + 1];
    v[10] = z[o - HC];
    v[16] = z[o + HC];
    v[15] = z[o + HC - 1];
    v[11] = z[o - HC + 1];
    v[4] = m[o];
    v[22] = p[o];
    v[21] = p[o - 1];
    v[5] = m[o + 1];
    v[19] = p[o - HC];
    v[7] = m[o + HC];
  }
  __device__ __forceinline__ float operator()(int dz, int dr, int dc) const {
    return v[(dz + 1) * 9 + (dr + 1) * 3 + (dc + 1)];
  }
};
// A field in three consecutive planes (m, 0, p) around in-plane offset o.
struct Planes3 {
  const float *m, *z, *p;
  int o;
  __device__ __forceinline__ float operator()(int dz, int dr, int dc) const {
    const float* b = dz < 0 ? m : (dz > 0 ? p : z);
    return b[o + dr * HC + dc];
  }
};

// What a thread knows of its points for a whole z-run (everything but z):
// its tile pixel, its two field points of a plane and its plane loads.
struct InPlane {
  bool c_lo, c_hi, r_lo, r_hi, ok;  // edges of the voxel's column and row; inside the image
};
__device__ __forceinline__ InPlane in_plane(int r, int c, int n) {
  return {c >= 1, c <= n - 2, r >= 1, r <= n - 2, r >= 0 && r < n && c >= 0 && c < n};
}
__device__ __forceinline__ Edges with_z(const InPlane& p, bool z_lo, bool z_hi) {
  return {p.c_lo, p.c_hi, p.r_lo, p.r_hi, z_lo, z_hi};
}
constexpr int NFP = WR * WC;               // field points of a plane
constexpr int FPT = (NFP + NT - 1) / NT;   // field points per thread
constexpr int LPT = (HR * HC + NT - 1) / NT;  // plane elements per thread

__global__ void __launch_bounds__(NT) k_stencil3d(Vol3Args a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Vol3Smem& S = *reinterpret_cast<Vol3Smem*>(smem_raw);
  if (a.bst != nullptr && a.bst->remaining == 0) return;  // uniform over the grid
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tr = tid / TC, tc = tid % TC;
  const int n = a.n, nz = a.nz;
  const long long d = (long long)n * n;
  const float *fk, *fkm;
  if (a.bst != nullptr) {
    const int G = a.bst->gstep;
    fk = a.f[G % 3];
    fkm = a.f[(G + 2) % 3];
  } else {
    fk = a.f[0];
    fkm = nullptr;
  }
  for (int s = tid; s < MAXZ; s += NT) {
    S.reg_hi[s] = 0.f;
    S.reg_lo[s] = 0.f;
  }
  const int ntx = (n + TC - 1) / TC, nty = (n + TR - 1) / TR, nzr = (nz + ZRUN - 1) / ZRUN;
  const int items = ntx * nty * nzr;
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    const int zr = it % nzr, txy = it / nzr;
    const int zb = zr * ZRUN, ze = min(nz, zb + ZRUN);
    const int r0 = (txy / ntx) * TR, c0 = (txy % ntx) * TC;
    const int r = r0 + tr, c = c0 + tc;
    // the run's invariants: this thread's voxel column, its field points and
    // its plane elements (2-D offset in the image, -1 outside)
    const InPlane vox = in_plane(r, c, n);
    const int vox_off = r * n + c;
    // field points row-aligned so a warp's 32 points are consecutive in a
    // plane row (no shared-memory bank conflicts): first pass, field rows
    // 0..7 at columns 0..31, one warp per row; second pass, rows 8 and 9 at
    // columns 0..31 and the 20 points of columns 32 and 33
    static_assert(TR == 8 && TC == 32 && NT == 256 && WR == 10 && WC == 34 && FPT == 2,
                  "the field-point passes are laid out for 8 x 32 tiles");
    InPlane fp[FPT];
    int fp_o[FPT];  // offset of the point in the f planes; -1: no point
#pragma unroll
    for (int u = 0; u < FPT; ++u) {
      int i = -1, j = 0;
      if (u == 0) {
        i = tid >> 5;
        j = tid & 31;
      } else if (tid < 64) {
        i = 8 + (tid >> 5);
        j = tid & 31;
      } else if (tid < 84) {
        i = (tid - 64) >> 1;
        j = 32 + ((tid - 64) & 1);
      }
      fp[u] = in_plane(r0 - 1 + i, c0 - 1 + j, n);
      fp_o[u] = i >= 0 ? (i + 1) * HC + (j + 1) : -1;
    }
    int ld_off[LPT];
#pragma unroll
    for (int u = 0; u < LPT; ++u) {
      const int t = tid + u * NT;
      const int i = t / HC, j = t % HC;
      const int rr = r0 - 2 + i, cc = c0 - 2 + j;
      ld_off[u] = (t < HR * HC && rr >= 0 && rr < n && cc >= 0 && cc < n) ? rr * n + cc : -1;
    }
    // plane loads are issued one step ahead into registers, so their latency
    // overlaps the field and gradient work of the current step
    float pk[LPT], pm[LPT];
    auto fetch = [&](int s) {
      const bool s_in = s >= 0 && s < nz;
      const float* fks = fk + (long long)(s_in ? s : 0) * d;
      const float* fms = fkm != nullptr ? fkm + (long long)(s_in ? s : 0) * d : nullptr;
#pragma unroll
      for (int u = 0; u < LPT; ++u) {
        pk[u] = 0.f;
        pm[u] = 0.f;
        if (s_in && ld_off[u] >= 0) {
          pk[u] = fks[ld_off[u]];
          if (fms != nullptr) pm[u] = fms[ld_off[u]];
        }
      }
    };
    fetch(zb - 2);
    // ring slots of planes s, s - 1 and s - 2 (plane s - 3 shares s's slot)
    int ra = ring3(zb - 2), rb = ring3(zb - 3), rc = ring3(zb - 4);
    for (int s = zb - 2; s <= ze + 1; ++s) {
      // plane s of f~ = f^k + theta_s (f^k - f^{k-1}) and of f^k (zero outside
      // the volume).  The ring slot it replaces (plane s - 3) was last read
      // before the previous step's second barrier.
      {
        const int ls = ra;
        const bool s_in = s >= 0 && s < nz;
        const float th = (s_in && fkm != nullptr) ? a.slots[s].theta_hi : 0.f;
#pragma unroll
        for (int u = 0; u < LPT; ++u) {
          const int t = tid + u * NT;
          if (t < HR * HC) {
            const float vk = pk[u];
            (&S.K[ls][0][0])[t] = vk;
            (&S.T[ls][0][0])[t] = fkm != nullptr ? fmaf(th, vk - pm[u], vk) : vk;
          }
        }
      }
      if (s + 1 <= ze + 1) fetch(s + 1);
      __syncthreads();
      // field plane P = s - 1 (needs f~ planes P - 1 .. P + 1)
      const int P = s - 1;
      if (P >= zb - 1 && P <= ze) {
        const bool inside = P >= 0 && P < nz;
        const bool z_lo = P >= 1, z_hi = P <= nz - 2;
        float lam1 = a.lam1, lam2 = a.lam2, eps = a.eps;
        if (inside && a.slots) {
          lam1 = a.slots[P].lambda1;
          lam2 = a.slots[P].lambda2;
          eps = a.slots[P].eps;
        }
        const float inv_eps = 1.f / eps;
        const float* Tm = &S.T[rc][0][0];
        const float* T0 = &S.T[rb][0][0];
        const float* Tp = &S.T[ra][0][0];
        float* Wo = &S.W[rb][0][0][0];
#pragma unroll
        for (int u = 0; u < FPT; ++u) {
          if (fp_o[u] < 0) continue;
          float v[NF];
#pragma unroll
          for (int q = 0; q < NF; ++q) v[q] = 0.f;
          if (inside && fp[u].ok) {
            const Edges e = with_z(fp[u], z_lo, z_hi);
            Nbr X;
            X.load(Tm, T0, Tp, fp_o[u]);
            all_comps(X, e, v);
            float n1, n2;
            norms(v, n1, n2);
            // lambda / max(||u||, eps) = lambda * min(rsqrt(||u||^2), 1/eps)
            const float s1 = lam1 * fminf(rsqrtf(n1), inv_eps);
            const float s2 = lam2 * fminf(rsqrtf(n2), inv_eps);
#pragma unroll
            for (int q = 0; q < 3; ++q) v[q] *= s1;
#pragma unroll
            for (int q = 3; q < NF; ++q) v[q] *= s2;
          }
          const int wo = fp_o[u] - HC - 1;  // the field planes' in-plane index
#pragma unroll
          for (int q = 0; q < NF; ++q) Wo[q * (WR * HC) + wo] = v[q];
        }
        // the regulariser at plane P from f^k (planes P - 1 .. P + 1): one
        // value per thread, summed by one warp after the barrier
        if (a.want_reg && P >= zb && P < ze) {
          float reg = 0.f;
          if (vox.ok) {
            const Edges e = with_z(vox, z_lo, z_hi);
            Nbr Xk;
            Xk.load(&S.K[rc][0][0], &S.K[rb][0][0], &S.K[ra][0][0], (tr + 2) * HC + (tc + 2));
            float uu[NF];
            all_comps(Xk, e, uu);
            float n1, n2;
            norms(uu, n1, n2);
            reg = lam1 * s_eps_f(n1, eps) + lam2 * s_eps_f(n2, eps);
          }
          S.regv[tid] = reg;
        }
      }
      __syncthreads();
      // the regulariser of plane P: warp P mod NWARP sums the block's values
      // in a fixed order (double-float)
      if (a.want_reg && P >= zb && P < ze && warp == (P & (NWARP - 1))) {
        float h = 0.f, l = 0.f;
#pragma unroll
        for (int k = 0; k < NT / 32; ++k) acc_add(h, l, S.regv[k * 32 + lane], 0.f);
        warp_sum_acc(h, l);
        if (lane == 0) acc_add(S.reg_hi[P], S.reg_lo[P], h, l);
      }
      // gradient at plane O = s - 2 (needs field planes O - 1 .. O + 1):
      // D^T for the first-order fields; each second-order block's transpose
      // is the block of the same form (symmetric ones) or of its partner
      // (4 <-> 6, 8 <-> 9, 10 <-> 11)
      const int O = s - 2;
      if (O >= zb && O < ze && vox.ok) {
        const Edges e = with_z(vox, O >= 1, O <= nz - 2);
        const float* Wm = &S.W[ra][0][0][0];  // plane O - 1 = s - 3
        const float* W0 = &S.W[rc][0][0][0];
        const float* Wp = &S.W[rb][0][0][0];
        const int o = (tr + 1) * HC + (tc + 1);
        constexpr int FS = WR * HC;  // field stride in a plane
        auto F = [&](int q) { return Planes3{Wm + q * FS, W0 + q * FS, Wp + q * FS, o}; };
        float g = 0.f;
        if (e.c_lo) g += W0[o];
        if (e.c_hi) g -= W0[o + 1];
        if (e.r_lo) g += W0[FS + o];
        if (e.r_hi) g -= W0[FS + o + HC];
        if (e.z_lo) g += W0[2 * FS + o];
        if (e.z_hi) g -= Wp[2 * FS + o];
        g += comp<3>(F(3), e);
        g += comp<6>(F(4), e);
        g += comp<5>(F(5), e);
        g += comp<4>(F(6), e);
        g += comp<7>(F(7), e);
        g += comp<9>(F(8), e);
        g += comp<8>(F(9), e);
        g += comp<11>(F(10), e);
        g += comp<10>(F(11), e);
        a.gR[(long long)O * d + vox_off] = g;
      }
      const int rn = rc;  // plane s + 1 takes the slot of plane s - 2
      rc = rb;
      rb = ra;
      ra = rn;
    }
  }
  if (!a.want_reg) return;
  __syncthreads();
  // the block's per-slice sums
  for (int s = tid; s < a.pstride; s += NT) {
    float h = 0.f, l = 0.f;
    if (s < MAXZ) {
      h = S.reg_hi[s];
      l = S.reg_lo[s];
    }
    a.partial[(long long)blockIdx.x * a.pstride + s] = make_float2(h, l);
  }
}

// slot-minor [d][Kp] -> slice-major [nz][d] of the ring entry of the current
// step (or every entry), 32 x 32 tiles through shared memory
__global__ void __launch_bounds__(256) k_slots_to_slices(const float* r0, const float* r1,
                                                         const float* r2, float* o0, float* o1,
                                                         float* o2, int d, int Kp, int nz,
                                                         const BatchState* bst, int all) {
  __shared__ float tile[32][33];
  if (bst != nullptr && bst->remaining == 0) return;
  const float* rin[3] = {r0, r1, r2};
  float* rout[3] = {o0, o1, o2};
  const int G = bst != nullptr ? bst->gstep : 0;
  const int j0 = blockIdx.x * 32, z0 = blockIdx.y * 32;
  for (int e = 0; e < 3; ++e) {
    if (!all && e != G % 3) continue;  // uniform over the block
    const float* in = rin[e];
    float* out = rout[e];
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
      const int j = j0 + k, z = z0 + threadIdx.x;
      tile[k][threadIdx.x] = (j < d && z < nz) ? in[(long long)j * Kp + z] : 0.f;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
      const int z = z0 + k, j = j0 + threadIdx.x;
      if (z < nz && j < d) out[(long long)z * d + j] = tile[threadIdx.x][k];
    }
  }
}

// slice-major [nz][d] -> slot-minor [d][Kp] (slots >= nz untouched)
__global__ void __launch_bounds__(256) k_slices_to_slots(const float* in, float* out, int d,
                                                         int Kp, int nz,
                                                         const BatchState* bst) {
  __shared__ float tile[32][33];
  if (bst != nullptr && bst->remaining == 0) return;
  const int j0 = blockIdx.x * 32, z0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int z = z0 + k, j = j0 + threadIdx.x;
    tile[k][threadIdx.x] = (z < nz && j < d) ? in[(long long)z * d + j] : 0.f;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int j = j0 + k, z = z0 + threadIdx.x;
    if (j < d && z < nz) out[(long long)j * Kp + z] = tile[threadIdx.x][k];
  }
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

int sm_count_vol() { return current_sm_count(); }

}  // namespace

int stencil3d_max_slices() { return MAXZ; }

int stencil3d_grid(int n, int nz) {
  const int items = ((n + TC - 1) / TC) * ((n + TR - 1) / TR) * ((nz + ZRUN - 1) / ZRUN);
  const int cap = 3 * sm_count_vol();
  return items < cap ? items : cap;
}

cudaError_t launch_stencil3d(const Vol3Args& a, cudaStream_t s) {
  if (a.nz < 1 || a.nz > MAXZ || a.n < 1) return cudaErrorInvalidValue;
  static PerDeviceOnce attr_once;
  const cudaError_t attr = attr_once.run([] {
    return cudaFuncSetAttribute(k_stencil3d, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(Vol3Smem));
  });
  if (attr != cudaSuccess) return attr;
  k_stencil3d<<<stencil3d_grid(a.n, a.nz), NT, sizeof(Vol3Smem), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sum_pairs(const float2* p, int rows, int cols, int pstride, double* out,
                             cudaStream_t s) {
  k_sum_pairs<<<1, 256, 0, s>>>(p, rows, cols, pstride, out);
  return cudaGetLastError();
}

cudaError_t launch_slots_to_slices(float* const* slot_ring, float* const* slice_ring, int d,
                                   int Kp, int nz, const BatchState* bst, int all,
                                   cudaStream_t s) {
  const dim3 grid((d + 31) / 32, (nz + 31) / 32), block(32, 8);
  k_slots_to_slices<<<grid, block, 0, s>>>(slot_ring[0], slot_ring[1], slot_ring[2],
                                           slice_ring[0], slice_ring[1], slice_ring[2], d, Kp,
                                           nz, bst, all);
  return cudaGetLastError();
}

cudaError_t launch_slices_to_slots(const float* in, float* out, int d, int Kp, int nz,
                                   const BatchState* bst, cudaStream_t s) {
  const dim3 grid((d + 31) / 32, (nz + 31) / 32), block(32, 8);
  k_slices_to_slots<<<grid, block, 0, s>>>(in, out, d, Kp, nz, bst);
  return cudaGetLastError();
}

}  // namespace appga
