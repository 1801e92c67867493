// totals_noalloc.cu -- conserved totals of a device state without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need the totals: code running
// inside a host callback or a custom allocator hook, a process whose memory pool is fixed at start-up,
// or an embedding framework that forbids cudaMalloc / cudaFree on its threads. hydro_init allocates
// (working states, reduction slots), so those callers cannot use conserved_totals. This entry point
// needs no context: its only scratch is the file-scope device array below, which every GPU that loads
// the library holds until the process exits.
//
// The reduction is a variant of the library's totals kernel: one FP64 partial per grid row (fixed
// order inside each row), then a fixed-order sum over rows, so a result is bitwise repeatable.
#include <cuda_runtime.h>

#include "../../include/hydro.h"

namespace {

constexpr int kMaxRows = 16384;  // ny limit: one 5-double partial per row

// per-row partials [kMaxRows][5] followed by the 5 totals
static __device__ __align__(256) double g_totals_scratch[kMaxRows * 5 + 5];

template <typename real, int NF>
__global__ void __launch_bounds__(256) row_partials_kernel(const real* __restrict__ U, int nx, int ny,
                                                           int geometry, double x0, double dx, double dy,
                                                           double* __restrict__ rows) {
  __shared__ double sred[8][NF];
  const long long n = static_cast<long long>(nx) * ny;
  for (int j = blockIdx.x; j < ny; j += gridDim.x) {
    double acc[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) acc[f] = 0.0;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const double dV = geometry == 1 ? 6.283185307179586 * (x0 + (i + 0.5) * dx) * dx * dy : dx * dy;
      const long long k = static_cast<long long>(j) * nx + i;
#pragma unroll
      for (int f = 0; f < NF; ++f) acc[f] = fma(static_cast<double>(U[f * n + k]), dV, acc[f]);
    }
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[f] += __shfl_xor_sync(0xffffffffu, acc[f], o);
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
#pragma unroll
      for (int f = 0; f < NF; ++f) sred[warp][f] = acc[f];
    __syncthreads();
    if (threadIdx.x < 5) {
      double s = 0.0;
      if (threadIdx.x < NF)
        for (int w = 0; w < 8; ++w) s += sred[w][threadIdx.x];
      rows[j * 5 + threadIdx.x] = s;  // every row entry is rewritten by every call
    }
    __syncthreads();
  }
}

__global__ void row_sum_kernel(const double* __restrict__ rows, int ny, double* __restrict__ out) {
  const int f = threadIdx.x;
  if (f < 5) {
    double s = 0.0;
    for (int j = 0; j < ny; ++j) s += rows[j * 5 + f];
    out[f] = s;
  }
}

// Device address of the scratch array in the current device's current context. Looked up on every
// call: the module (and with it the array) is placed anew when a context is recreated (after
// cudaDeviceReset, or under another driver-API context), so a cached address could be stale. After
// the module's first load the lookup allocates nothing.
int scratch_address(double** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_totals_scratch) != cudaSuccess || !p) return HYDRO_ECUDA;
  *out = static_cast<double*>(p);
  return HYDRO_OK;
}

template <typename real>
int run(const real* U, int nx, int ny, int nfields, int geometry, double x0, double dx, double dy,
        cudaStream_t s, double* rows, double out[5]) {
  const int blocks = ny < 4096 ? ny : 4096;
  if (nfields == 5)
    row_partials_kernel<real, 5><<<blocks, 256, 0, s>>>(U, nx, ny, geometry, x0, dx, dy, rows);
  else
    row_partials_kernel<real, 4><<<blocks, 256, 0, s>>>(U, nx, ny, geometry, x0, dx, dy, rows);
  if (cudaPeekAtLastError() != cudaSuccess) return HYDRO_ECUDA;
  double* res = rows + kMaxRows * 5;
  row_sum_kernel<<<1, 32, 0, s>>>(rows, ny, res);
  if (cudaPeekAtLastError() != cudaSuccess) return HYDRO_ECUDA;
  if (cudaMemcpyAsync(out, res, 5 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return HYDRO_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return HYDRO_ECUDA;
  return HYDRO_OK;
}

}  // namespace

int conserved_totals_noalloc(const void* U, int nx, int ny, int nfields, int dtype, int geometry, double x0,
                             double x1, double y0, double y1, void* stream, double out[5]) {
  if (!U || !out || nx < 1 || ny < 1 || (nfields != 4 && nfields != 5) || (dtype != HYDRO_F32 && dtype != HYDRO_F64) ||
      (geometry != 0 && geometry != 1) || !(x1 > x0) || !(y1 > y0))
    return HYDRO_EINVAL;
  if (ny > kMaxRows) return HYDRO_ESIZE;
  // an error left pending by the caller's own earlier work is not this call's: refuse without
  // launching and without consuming it, so the caller still sees it
  if (cudaPeekAtLastError() != cudaSuccess) return HYDRO_ECUDA;
  double* rows = nullptr;
  int rc = scratch_address(&rows);
  if (rc) return rc;
  const double dx = (x1 - x0) / nx, dy = (y1 - y0) / ny;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dtype == HYDRO_F64)
    return run<double>(static_cast<const double*>(U), nx, ny, nfields, geometry, x0, dx, dy, s, rows, out);
  return run<float>(static_cast<const float*>(U), nx, ny, nfields, geometry, x0, dx, dy, s, rows, out);
}
