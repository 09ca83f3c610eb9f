// Self-test of the bounded mbarrier wait: the barrier's phase can never
// complete (16 transaction bytes announced, no copy issued), so every
// mbarrier.try_wait returns false after its own suspend limit and the loop
// gives up after `polls` attempts, exactly as the staged passes do after
// WZ_MBAR_SPIN_LIMIT polls.  Nothing is in flight when the block exits.
#include <cuda_runtime.h>

#include "wz.h"
#include "wz_probe.h"
#include "wz_tma.cuh"

namespace wz {
namespace {

__global__ void wait_timeout_probe(int polls, int* status, long long* cycles) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(&bar, 16u);
    const long long c0 = clock64();
    bool done = false;
    for (int i = 0; i < polls && !done; ++i) done = mbar_try_wait(&bar, 0);
    *cycles = clock64() - c0;
    *status = done ? WZ_OK : WZ_ETIMEOUT;
  }
}

}  // namespace
}  // namespace wz

extern "C" int wz_selftest_wait_timeout(int polls, int* status, long long* cycles) {
  if (!status || !cycles || polls < 1 || polls > 65536) return WZ_EINVAL;
  int* d = nullptr;
  if (cudaMalloc(&d, 16) != cudaSuccess) return WZ_ENOMEM;
  int* ds = d;
  long long* dc = reinterpret_cast<long long*>(d + 2);
  wz::count_launch();
  wz::wait_timeout_probe<<<1, 32>>>(polls, ds, dc);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(status, ds, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(cycles, dc, sizeof(long long), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? WZ_OK : WZ_ECUDA;
}
