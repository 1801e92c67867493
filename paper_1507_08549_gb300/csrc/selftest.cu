// selftest.cu -- self-test of the bounded device wait that guards the stage kernel's tile copies.
#include "stage_kernel.cuh"

namespace hydro {

namespace {
// One thread waits on an mbarrier that no arrival or copy completes, for `polls` polls, through the same
// bounded wait the stage kernel uses, and reports ERR_TIMEOUT as a lost tile copy would.
__global__ void wait_selftest_kernel(unsigned polls, int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    if (!mbar_wait_limit(&bar, 0u, polls)) atomicOr(err, ERR_TIMEOUT);
  }
}
}  // namespace

cudaError_t launch_wait_selftest(unsigned polls, int* err, cudaStream_t s) {
  wait_selftest_kernel<<<1, 32, 0, s>>>(polls, err);
  return cudaGetLastError();
}

}  // namespace hydro
