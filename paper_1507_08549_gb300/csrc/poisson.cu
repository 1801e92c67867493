// poisson.cu -- launchers of the exact summation and the red-black SOR Poisson kernels (Sec. 2.1).
#include "poisson_kernel.cuh"

namespace hydro {

namespace {
unsigned blocks_for(long long n, int threads, int cap) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return static_cast<unsigned>(b < cap ? b : cap);
}

int sm_count() {
  static const int n = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
      (void)cudaGetLastError();
      return 152;
    }
    return v;
  }();
  return n;
}
}  // namespace

cudaError_t launch_exact_sum(const double* x, long long n, ExactAcc* acc, double* out, cudaStream_t s, int* launches) {
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(ExactAcc), s);
  if (e != cudaSuccess) return e;
  if (n > 0) {
    xs_array_kernel<<<blocks_for(n, 256, 4 * sm_count()), 256, 0, s>>>(x, n, acc);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (launches) ++*launches;
  }
  xs_round_kernel<<<1, 32, 0, s>>>(acc, out);
  if (launches) ++*launches;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_poisson_setup(PoissonParams* P_dev, ExactAcc* acc, long long n, int nx, int ny, cudaStream_t s,
                                 int* launches) {
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(ExactAcc), s);
  if (e != cudaSuccess) return e;
  poisson_mass_kernel<T><<<blocks_for(n, 256, 4 * sm_count()), 256, 0, s>>>(P_dev, acc);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int m = nx > ny ? nx : ny;
  poisson_setup_kernel<<<blocks_for(m, 256, 1024), 256, 0, s>>>(P_dev, acc);
  if (launches) *launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_sor_chunk(const PoissonParams* P_dev, SorCtl* ctl, int nx, int ny, cudaStream_t s, int* launches) {
  const int hx = (nx + 1) / 2;
  const dim3 grid((hx + SOR_BX - 1) / SOR_BX, (ny + SOR_BY - 1) / SOR_BY), block(SOR_BX, SOR_BY);
  for (int r = 0; r < SOR_CHUNK; ++r)
    for (int color = 0; color < 2; ++color) {
      sor_color_kernel<<<grid, block, 0, s>>>(P_dev, ctl, color, r);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  sor_advance_kernel<<<1, 32, 0, s>>>(ctl, SOR_CHUNK);
  if (launches) *launches += 2 * SOR_CHUNK + 1;
  return cudaGetLastError();
}

template cudaError_t launch_poisson_setup<float>(PoissonParams*, ExactAcc*, long long, int, int, cudaStream_t, int*);
template cudaError_t launch_poisson_setup<double>(PoissonParams*, ExactAcc*, long long, int, int, cudaStream_t, int*);

}  // namespace hydro
