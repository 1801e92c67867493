// reinit_kernel.cuh -- level-set reinitialisation (Leung, Chu & Lin 2015, Sec. 2.2).
//
// front_kernel     one thread per cell: for the neighbour pairs (i,j)-(i+1,j) and (i,j)-(i,j+1) whose
//                  S values lie on opposite sides of zero (> 0 ash, <= 0 fuel) it appends the front
//                  point found by linear interpolation of S along the segment between the centres;
// distance_kernel  every cell's smallest distance to the front points (the points stream through
//                  shared memory in chunks; squared distances are compared, one square root at the
//                  end), then S_new = H(d) S_old + (1 - H(d)) d with the sign of S_old and
//                  H(d) = [1 - tanh((d - d0)/(Delta/3))] / [1 - tanh(-d0/(Delta/3))], d0 = 3 Delta.
// The point order depends on atomics; the minimum does not, so results are deterministic. FP64 uses
// the reference definition's operation order (true division, IEEE square root).
#pragma once
#include "stage_kernel.cuh"

namespace hydro {

template <typename real>
__global__ void __launch_bounds__(256) front_kernel(const real* __restrict__ phi, int nx, int ny, int pitch,
                                                    double x0, double y0, double dx, double dy,
                                                    real* __restrict__ front, int capacity, int* count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= nx) return;
  using A = Ar<real>;
  const real a = phi[static_cast<long long>(j) * pitch + i];
  // centre x0 + (i + 1/2) dx and the crossing x_a + dx (a / (a - b)), each operation rounded once
  const real xa = static_cast<real>(__dadd_rn(x0, __dmul_rn(i + 0.5, dx)));
  const real ya = static_cast<real>(__dadd_rn(y0, __dmul_rn(j + 0.5, dy)));
  const real rdx = static_cast<real>(dx), rdy = static_cast<real>(dy);
  if (i + 1 < nx) {
    const real b = phi[static_cast<long long>(j) * pitch + i + 1];
    if ((a > real(0)) != (b > real(0))) {
      const int k = atomicAdd(count, 1);
      if (k < capacity) {
        front[2 * k] = A::sum(xa, rdx * (a / (a - b)));
        front[2 * k + 1] = ya;
      }
    }
  }
  if (j + 1 < ny) {
    const real b = phi[static_cast<long long>(j + 1) * pitch + i];
    if ((a > real(0)) != (b > real(0))) {
      const int k = atomicAdd(count, 1);
      if (k < capacity) {
        front[2 * k] = xa;
        front[2 * k + 1] = A::sum(ya, rdy * (a / (a - b)));
      }
    }
  }
}

constexpr int REINIT_CHUNK = 1024;  // front points per shared-memory chunk

template <typename real>
__global__ void __launch_bounds__(256) distance_kernel(real* __restrict__ phi, int nx, int ny, int pitch,
                                                       double x0, double y0, double dx, double dy, double delta,
                                                       const real* __restrict__ front, int capacity,
                                                       const int* __restrict__ count, int* err) {
  __shared__ real sx[REINIT_CHUNK], sy[REINIT_CHUNK];
  __shared__ float2 sxy[sizeof(real) == 4 ? REINIT_CHUNK : 1];  // FP32: a point's x, y in one 8-byte load
  const int m = min(*count, capacity);
  if (*count > capacity) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, ERR_NONPHYSICAL);
    return;
  }
  if (m == 0) return;  // no front: S unchanged
  const long long n = static_cast<long long>(nx) * ny;
  const long long cell = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool active = cell < n;
  const int i = active ? static_cast<int>(cell % nx) : 0;
  const int j = active ? static_cast<int>(cell / nx) : 0;
  const real x = static_cast<real>(__dadd_rn(x0, __dmul_rn(i + 0.5, dx)));
  const real y = static_cast<real>(__dadd_rn(y0, __dmul_rn(j + 0.5, dy)));
  real best = real(INFINITY);
  for (int base = 0; base < m; base += REINIT_CHUNK) {
    const int len = min(REINIT_CHUNK, m - base);
    __syncthreads();
    for (int k = threadIdx.x; k < len; k += blockDim.x) {
      if constexpr (sizeof(real) == 4) {
        sxy[k] = make_float2(front[2 * (base + k)], front[2 * (base + k) + 1]);
      } else {
        sx[k] = front[2 * (base + k)];
        sy[k] = front[2 * (base + k) + 1];
      }
    }
    __syncthreads();
    if (active) {
      if constexpr (sizeof(real) == 8) {
        for (int k = 0; k < len; ++k) {
          const real ex = __dsub_rn(x, sx[k]), ey = __dsub_rn(y, sy[k]);
          const real d2 = __dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey));
          best = d2 < best ? d2 : best;
        }
      } else {
#pragma unroll 8
        for (int k = 0; k < len; ++k) {
          const float2 q = sxy[k];
          const real ex = x - q.x, ey = y - q.y;
          best = fminf(best, __fmaf_rn(ex, ex, ey * ey));
        }
      }
    }
  }
  if (!active) return;
  const long long g = static_cast<long long>(j) * pitch + i;
  const real s_old = phi[g];
  if constexpr (sizeof(real) == 4) {  // the blend in FP32 too (the FP64 pipe runs at 1/64 of the FP32 rate)
    const float d = sqrtf(best), df = static_cast<float>(delta);
    // (d - d0) / w with d0 = 3 delta, w = delta / 3; -d0 / w = -9
    const float H = (1.0f - tanhf((d - 3.0f * df) * (3.0f / df))) / (1.0f - tanhf(-9.0f));
    const float sd = s_old > 0.0f ? d : -d;
    phi[g] = H * s_old + (1.0f - H) * sd;
  } else {
    const double d = sqrt(static_cast<double>(best));
    const double d0 = 3.0 * delta, w = delta / 3.0;
    const double H = (1.0 - tanh((d - d0) / w)) / (1.0 - tanh(-d0 / w));
    const double sd = s_old > real(0) ? d : -d;
    phi[g] = static_cast<real>(H * static_cast<double>(s_old) + (1.0 - H) * sd);
  }
}

}  // namespace hydro
