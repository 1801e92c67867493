// peak_probe.cu -- measured fused multiply-add throughput of the GPU in FP32 and FP64, the cross-check of
// the arithmetic roofline (152 SMs x lanes x clock) that the benchmark reports against.
//
// Every thread runs 8 independent FMA chains for `iters` iterations (8 x iters FMAs per thread, no memory
// traffic in the loop); a grid of 8 CTAs of 256 threads per SM keeps every SM's FMA pipes busy. The result
// is FMAs per second (one FMA = 2 flops).
#include <cuda_runtime.h>

#include "hydro_internal.cuh"

namespace hydro {

namespace {
template <typename real>
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, real seed, real* sink) {
  real a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = seed + static_cast<real>(threadIdx.x + k);
  const real m = real(0.999999), c = real(1e-7);
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
  }
  real s = real(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == real(-1)) *sink = s;  // never true; keeps the chains live
}
}  // namespace

template <typename real>
cudaError_t run_fma_probe(int iters, cudaStream_t st, int num_sms, double* fma_per_s) {
  real* sink = nullptr;
  cudaError_t e = cudaMalloc(&sink, sizeof(real));
  if (e != cudaSuccess) return e;
  cudaEvent_t a = nullptr, b = nullptr;
  e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  const int blocks = 8 * num_sms, threads = 256;
  float ms = 0.f;
  if (e == cudaSuccess) {
    fma_probe_kernel<real><<<blocks, threads, 0, st>>>(iters / 8 + 1, real(1), sink);  // warm-up
    e = cudaEventRecord(a, st);
  }
  if (e == cudaSuccess) {
    fma_probe_kernel<real><<<blocks, threads, 0, st>>>(iters, real(1), sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (e == cudaSuccess) *fma_per_s = static_cast<double>(blocks) * threads * iters * 16.0 * 8.0 / (ms * 1e-3);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(sink);
  return e;
}

template cudaError_t run_fma_probe<float>(int, cudaStream_t, int, double*);
template cudaError_t run_fma_probe<double>(int, cudaStream_t, int, double*);

}  // namespace hydro
