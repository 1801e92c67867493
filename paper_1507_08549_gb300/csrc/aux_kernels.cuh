// aux_kernels.cuh -- small kernels around the stage kernel: packing a caller state into the padded
// working layout (with ghost images and the first stage's reductions), frozen-slot writes, and the
// FP64 conserved totals (Leung, Chu & Lin 2015: totals of mass and energy as in the Gresho test table
// of Sec. 5.2).
#pragma once
#include "stage_kernel.cuh"

namespace hydro {

// Grid-stride over the cells (a few blocks per SM); one block-level reduction and one atomic per slot
// and block at the end, so the global maxima see a few thousand atomics, not one per warp. Block `block`
// of `nblocks` takes cells block * 256 + threadIdx.x, step nblocks * 256.
template <typename real, int NF>
__device__ __forceinline__ void pack_range(const real* __restrict__ U, const GridParams<real>& g, real* out,
                                           real* alpha_slot, real* smax_slot, double* t_acc, double t0, int block,
                                           int nblocks) {
  __shared__ real sred[8][3];
  if (block == 0 && threadIdx.x == 0 && t_acc) *t_acc = t0;
  real amx = real(0), amy = real(0), smx = real(0);
  const long long n = static_cast<long long>(g.nx) * g.ny;
  const long long stride = static_cast<long long>(nblocks) * blockDim.x;
  for (long long k = static_cast<long long>(block) * blockDim.x + threadIdx.x; k < n; k += stride) {
    const int j = static_cast<int>(k / g.nx), i = static_cast<int>(k - static_cast<long long>(j) * g.nx);
    real val[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) val[f] = U[f * n + k];
    const long long off = static_cast<long long>(j + GY) * g.pitch + i + GX;
#pragma unroll
    for (int f = 0; f < NF; ++f) out[f * g.fstride + off] = val[f];
    if (i < 3 || i >= g.nx - 3 || j < 3 || j >= g.ny - 3)
      write_ghost_images<real, NF>(out, g.fstride, g.pitch, g.nx, g.ny, g.bc, i, j, val);
    real p, sx, sy, sm;
    Ar<real>::speeds(val[0], val[1], val[2], val[3], g.gamma, g.gm1, p, sx, sy, sm);
    bool ok = val[0] > real(0) && p > real(0) && RT<real>::finite(val[3]) && RT<real>::finite(val[1]) &&
              RT<real>::finite(val[2]) && RT<real>::finite(sm);
    if (NF == 5) ok = ok && RT<real>::finite(val[NF - 1]);
    if (!ok) atomicOr(g.err, ERR_NONPHYSICAL);
    amx = fmax(amx, sx);
    amy = fmax(amy, sy);
    smx = fmax(smx, sm);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    amx = fmax(amx, __shfl_xor_sync(0xffffffffu, amx, o));
    amy = fmax(amy, __shfl_xor_sync(0xffffffffu, amy, o));
    smx = fmax(smx, __shfl_xor_sync(0xffffffffu, smx, o));
  }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sred[warp][0] = amx;
    sred[warp][1] = amy;
    sred[warp][2] = smx;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    real m = real(0);
    for (int w = 0; w < 8; ++w) m = fmax(m, sred[w][threadIdx.x]);
    if (threadIdx.x == 0 && alpha_slot) RT<real>::atomic_max(&alpha_slot[0], m);
    if (threadIdx.x == 1 && alpha_slot) RT<real>::atomic_max(&alpha_slot[1], m);
    if (threadIdx.x == 2 && smax_slot) RT<real>::atomic_max(smax_slot, m);
  }
}

template <typename real, int NF>
__global__ void __launch_bounds__(256) pack_kernel(const real* __restrict__ U, GridParams<real> g,
                                                   real* alpha_slot, real* smax_slot, double* t_acc, double t0) {
  pack_range<real, NF>(U, g, g.out, alpha_slot, smax_slot, t_acc, t0, blockIdx.x, gridDim.x);
}

// Batched ensembles: member blockIdx.y, with its first-stage parameters P[m], packs its caller state U[m]
// into its buffer A (the stage's U^n) and reduces into its own slots; one launch for all members.
template <typename real, int NF>
__global__ void __launch_bounds__(256) batch_pack_kernel(const GridParams<real>* __restrict__ P,
                                                         const real* const* __restrict__ U,
                                                         const double* __restrict__ t0) {
  const int m = blockIdx.y;
  const GridParams<real>& g = P[m];
  pack_range<real, NF>(U[m], g, const_cast<real*>(g.un), const_cast<real*>(g.alpha_in), g.smax, g.t_acc, t0[m],
                       blockIdx.x, gridDim.x);
}

// ... and copies member blockIdx.y's buffer A back into its caller state U[m] (interior cells).
template <typename real, int NF>
__global__ void __launch_bounds__(256) batch_unpack_kernel(const GridParams<real>* __restrict__ P,
                                                           real* const* __restrict__ U) {
  const int m = blockIdx.y;
  const GridParams<real>& g = P[m];
  const long long n = static_cast<long long>(g.nx) * g.ny;
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  real* dst = U[m];
  for (long long k = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += stride) {
    const int j = static_cast<int>(k / g.nx), i = static_cast<int>(k - static_cast<long long>(j) * g.nx);
    const long long off = static_cast<long long>(j + GY) * g.pitch + i + GX;
#pragma unroll
    for (int f = 0; f < NF; ++f) dst[f * n + k] = g.un[f * g.fstride + off];
  }
}

// Copy the interior of a padded state to an unpadded one (to_padded = false) or back, every field in one
// launch: element k of the unpadded [nf][ny][nx] array is cell (k mod nx, (k / nx) mod ny) of field
// k / (nx ny).
template <typename real>
__global__ void __launch_bounds__(256) copy_state_kernel(real* __restrict__ dst, const real* __restrict__ src, int nx,
                                                         int ny, int nf, int pitch, long long fstride, bool to_padded) {
  const long long plane = static_cast<long long>(nx) * ny, n = plane * nf;
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  for (long long k = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += stride) {
    const int f = static_cast<int>(k / plane);
    const long long r = k - f * plane;
    const int j = static_cast<int>(r / nx), i = static_cast<int>(r - static_cast<long long>(j) * nx);
    const long long e = f * fstride + static_cast<long long>(j + GY) * pitch + i + GX;
    if (to_padded)
      dst[e] = src[k];
    else
      dst[k] = src[e];
  }
}

template <typename real>
__global__ void set_frozen_kernel(double* dt_slot, double dt, real* alpha_slots, double a0, double a1, double a2,
                                  double a3, double a4, double a5) {
  if (threadIdx.x == 0) {
    if (dt_slot) *dt_slot = dt;
    if (alpha_slots) {
      alpha_slots[0] = static_cast<real>(a0);
      alpha_slots[1] = static_cast<real>(a1);
      alpha_slots[2] = static_cast<real>(a2);
      alpha_slots[3] = static_cast<real>(a3);
      alpha_slots[4] = static_cast<real>(a4);
      alpha_slots[5] = static_cast<real>(a5);
    }
  }
}

// Per-thread FP64 sums over a grid-stride range, then a fixed-shape tree: the result depends only on
// the launch shape, which the host keeps fixed per device.
template <typename real, int NF>
__global__ void __launch_bounds__(256) totals_partial_kernel(const real* __restrict__ U, int nx, int ny, int geometry,
                                                             double x0, double dx, double dy,
                                                             double* __restrict__ partials) {
  const long long n = static_cast<long long>(nx) * ny;
  double acc[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) acc[f] = 0.0;
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  for (long long k = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += stride) {
    double dV = dx * dy;
    if (geometry == 1) {
      const int i = static_cast<int>(k % nx);
      dV = 6.283185307179586 * (x0 + (i + 0.5) * dx) * dx * dy;
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) acc[f] = fma(static_cast<double>(U[f * n + k]), dV, acc[f]);
  }
  __shared__ double sred[8][NF];
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[f] += __shfl_xor_sync(0xffffffffu, acc[f], o);
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int f = 0; f < NF; ++f) sred[warp][f] = acc[f];
  __syncthreads();
  if (threadIdx.x < NF) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += sred[w][threadIdx.x];
    partials[blockIdx.x * 5 + threadIdx.x] = s;
  }
}

static __global__ void totals_final_kernel(const double* __restrict__ partials, int nblocks, int nf, double* out) {
  const int f = threadIdx.x;
  if (f < 5) {
    double s = 0.0;
    if (f < nf)
      for (int b = 0; b < nblocks; ++b) s += partials[b * 5 + f];
    out[f] = s;
  }
}

}  // namespace hydro
