// reinit_kernel.cuh -- level-set reinitialisation (Leung, Chu & Lin 2015, Sec. 2.2).
//
// front_kernel     one thread per cell: for the neighbour pairs (i,j)-(i+1,j) and (i,j)-(i,j+1) whose
//                  S values lie on opposite sides of zero (> 0 ash, <= 0 fuel) it appends the front
//                  point found by linear interpolation of S along the segment between the centres;
// distance_kernel  every cell's smallest distance to the front points (the points stream through
//                  shared memory in chunks; squared distances are compared, one square root at the
//                  end), then S_new = H(d) S_old + (1 - H(d)) d with the sign of S_old and
//                  H(d) = [1 - tanh((d - d0)/(Delta/3))] / [1 - tanh(-d0/(Delta/3))], d0 = 3 Delta.
//                  FP64 states, in the reference definition's operation order (true division, IEEE
//                  square root); FP32 states use distance_kernel_x2 (two cells per thread, packed FP32).
// The point order depends on atomics; the minimum does not, so results are deterministic.
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
  static_assert(sizeof(real) == 8, "FP32 states use distance_kernel_x2");
  __shared__ real sx[REINIT_CHUNK], sy[REINIT_CHUNK];
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
      sx[k] = front[2 * (base + k)];
      sy[k] = front[2 * (base + k) + 1];
    }
    __syncthreads();
    if (active) {
      for (int k = 0; k < len; ++k) {
        const real ex = __dsub_rn(x, sx[k]), ey = __dsub_rn(y, sy[k]);
        const real d2 = __dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey));
        best = d2 < best ? d2 : best;
      }
    }
  }
  if (!active) return;
  const long long g = static_cast<long long>(j) * pitch + i;
  const real s_old = phi[g];
  const double d = sqrt(static_cast<double>(best));
  const double d0 = 3.0 * delta, w = delta / 3.0;
  const double H = (1.0 - tanh((d - d0) / w)) / (1.0 - tanh(-d0 / w));
  const double sd = s_old > real(0) ? d : -d;
  phi[g] = static_cast<real>(H * static_cast<double>(s_old) + (1.0 - H) * sd);
}

// FP32: two cells per thread (cells b + t and b + 256 + t of a 512-cell block) in the two lanes of packed
// f32x2 arithmetic, each lane rounding exactly as the scalar kernel's operations (same distances, same
// minimum); the points are stored as (-x, -x, -y, -y) so one 16-byte load feeds both lanes.
template <typename real>  // float only (a template so that only the FP32 translation unit instantiates it)
__global__ void __launch_bounds__(256) distance_kernel_x2(real* __restrict__ phi, int nx, int ny, int pitch,
                                                          double x0, double y0, double dx, double dy, double delta,
                                                          const real* __restrict__ front, int capacity,
                                                          const int* __restrict__ count, int* err) {
  static_assert(sizeof(real) == 4, "packed FP32 distance kernel");
  __shared__ float4 sp[REINIT_CHUNK];
  const int m = min(*count, capacity);
  if (*count > capacity) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, ERR_NONPHYSICAL);
    return;
  }
  if (m == 0) return;  // no front: S unchanged
  const long long n = static_cast<long long>(nx) * ny;
  long long cell[2];
  bool active[2];
  float2 X, Y;
  float* xs = &X.x;
  float* ys = &Y.x;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    cell[h] = static_cast<long long>(blockIdx.x) * 512 + h * 256 + threadIdx.x;
    active[h] = cell[h] < n;
    const int i = active[h] ? static_cast<int>(cell[h] % nx) : 0;
    const int j = active[h] ? static_cast<int>(cell[h] / nx) : 0;
    xs[h] = static_cast<float>(__dadd_rn(x0, __dmul_rn(i + 0.5, dx)));
    ys[h] = static_cast<float>(__dadd_rn(y0, __dmul_rn(j + 0.5, dy)));
  }
  float best0 = INFINITY, best1 = INFINITY;
  for (int base = 0; base < m; base += REINIT_CHUNK) {
    const int len = min(REINIT_CHUNK, m - base);
    __syncthreads();
    for (int k = threadIdx.x; k < len; k += blockDim.x) {
      const float px = front[2 * (base + k)], py = front[2 * (base + k) + 1];
      sp[k] = make_float4(-px, -px, -py, -py);
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < len; ++k) {
      const float4 q = sp[k];
      const float2 ex = __fadd2_rn(X, make_float2(q.x, q.y));
      const float2 ey = __fadd2_rn(Y, make_float2(q.z, q.w));
      const float2 d2 = __ffma2_rn(ex, ex, __fmul2_rn(ey, ey));
      best0 = fminf(best0, d2.x);
      best1 = fminf(best1, d2.y);
    }
  }
  const float df = static_cast<float>(delta);
  const float norm = 1.0f / (1.0f - tanhf(-9.0f));
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (!active[h]) continue;
    const int i = static_cast<int>(cell[h] % nx), j = static_cast<int>(cell[h] / nx);
    const long long g = static_cast<long long>(j) * pitch + i;
    const float s_old = phi[g];
    const float d = sqrtf(h ? best1 : best0);
    // the blend of the scalar kernel: (d - d0) / w with d0 = 3 delta, w = delta / 3
    const float H = (1.0f - tanhf((d - 3.0f * df) * (3.0f / df))) * norm;
    const float sd = s_old > 0.0f ? d : -d;
    phi[g] = H * s_old + (1.0f - H) * sd;
  }
}

}  // namespace hydro
