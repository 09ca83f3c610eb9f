// Measurement helpers that are not part of the method: the bounded-wait
// self-test and an FMA throughput microkernel (the ALU peak the FP64 passes
// are reported against).
//
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

// FMA throughput: each thread runs 8 independent chains of `iters` fused
// multiply-adds (x <- a x + b, a fixed point of modulus < 1, so the values stay
// finite) and stores their sum, so no chain can be removed.
template <typename R>
__global__ void __launch_bounds__(256) fma_chains(R* out, int iters, R a, R b) {
  R acc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] = R(threadIdx.x & 7) + R(i);
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = fma(acc[i], a, b);
  }
  R s = R(0);
#pragma unroll
  for (int i = 0; i < 8; ++i) s += acc[i];
  out[(long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace wz

extern "C" int wz_fma_peak(int real_bytes, int iters, double* tflops, double* ms) {
  if (!tflops || !ms || (real_bytes != 4 && real_bytes != 8) || iters < 1 || iters > (1 << 24)) return WZ_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return WZ_ECUDA;
  const int threads = 256, blocks = sms * 8;  // 2048 threads per SM
  void* d = nullptr;
  if (cudaMalloc(&d, (size_t)blocks * threads * 8) != cudaSuccess) return WZ_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto launch = [&](int n) {
    wz::count_launch();
    if (real_bytes == 8)
      wz::fma_chains<double><<<blocks, threads>>>((double*)d, n, 0.999999, 1e-6);
    else
      wz::fma_chains<float><<<blocks, threads>>>((float*)d, n, 0.999f, 1e-3f);
  };
  launch(iters / 16 + 1);  // warm-up
  cudaEventRecord(e0);
  launch(iters);
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  if (e != cudaSuccess) return WZ_ECUDA;
  *ms = t;
  *tflops = 2.0 * 8.0 * (double)iters * blocks * threads / (t * 1e-3) / 1e12;
  return WZ_OK;
}

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
