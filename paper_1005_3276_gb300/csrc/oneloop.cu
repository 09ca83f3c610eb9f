// One-loop lattice sums of Sec. 5 on an N^4 momentum lattice (a = 1), FP64.
//
//   scalar     (1/N^4) sum_k [P(k+p).P(k) / (s(k) s(k+p)) - P^2(k) / s^2(k)] / (r(k) r(k+p))
//   fermion    (1/N^4) sum_k P_3(k+p) / (r(k) r(k+p) s(k+p))
//   auxiliary  (1/N^4) sum_k 1 / r(k)^2
//
// P_mu = sin k_mu, M = 1 - 2 sum sin^2(k_mu/2), s = sqrt(P^2 + M^2),
// r = 2 (1 - M/s) + (ma^2/2)(1 + M/s), p = (0, 0, 0, 2 pi / N), periodic k.
// The counterterms of Tables sse, fse, ase: Z_phi - 1 = scalar / sin^2(2 pi/N),
// Z_chi - 1 = -fermion / sin(2 pi/N), Z_F - 1 = auxiliary (each over |g|^2).
//
// The three directions transverse to p are equivalent under permutations and
// reflections n -> N - n, so the sum runs over sorted triples a <= b <= c of
// half-range indices (0..N/2) with their multiplicities, times the full range
// of the p direction: about N^4 / 48 terms.  One block per pair (a, b); its
// threads share the (c, n_3) range.  1 - M/s and 1 + M/s are evaluated in the
// form without cancellation (P^2 / (s (s + |M|)) for the small one).
#include <cmath>
#include <vector>

#include "../../include/wz.h"
#include "wz_cg.cuh"
#include "wz_probe.h"

namespace wz {
namespace {

struct LoopTabs {
  const double* sn;  // sin(2 pi n / N), n = 0..N
  const double* sh;  // 2 sin^2(pi n / N) = 1 - cos(2 pi n / N)
  int N, H;
  double ma2;
};

__device__ __forceinline__ void site_parts(double P2, double M, double ma2, double* s, double* r) {
  const double sv = sqrt(P2 + M * M);
  const double om = M >= 0.0 ? P2 / (sv * (sv + M)) : 1.0 - M / sv;  // 1 - M/s
  const double op = M >= 0.0 ? 1.0 + M / sv : P2 / (sv * (sv - M));  // 1 + M/s
  *s = sv;
  *r = 2.0 * om + 0.5 * ma2 * op;
}

// pairs (a, b), a <= b <= H, enumerated row by row: index of (a, b) = a (2H + 3 - a) / 2 + (b - a)
__device__ __forceinline__ void pair_of(long q, int H, int* a, int* b) {
  int aa = 0;
  long start = 0;
  while (true) {
    const long row = H + 1 - aa;  // pairs with this a
    if (q < start + row) break;
    start += row;
    ++aa;
  }
  *a = aa;
  *b = aa + (int)(q - start);
}

__device__ __forceinline__ double reflect_weight(int n, int H) { return (n == 0 || n == H) ? 1.0 : 2.0; }

__global__ void one_loop_sums(LoopTabs t, double* part) {
  __shared__ double red[33];
  int a, b;
  pair_of(blockIdx.x, t.H, &a, &b);
  const int N = t.N, H = t.H;
  const long units = (long)(H - b + 1) * N;  // (c, n3) with b <= c <= H
  double acc[3] = {0.0, 0.0, 0.0};
  for (long u = threadIdx.x; u < units; u += blockDim.x) {
    const int c = b + (int)(u / N), n3 = (int)(u % N);
    const double mult = (a == b && b == c) ? 1.0 : ((a == b || b == c) ? 3.0 : 6.0);
    const double w = mult * reflect_weight(a, H) * reflect_weight(b, H) * reflect_weight(c, H);
    const double sa = t.sn[a], sb = t.sn[b], sc = t.sn[c];
    const double S3 = sa * sa + sb * sb + sc * sc;
    const double W3 = t.sh[a] + t.sh[b] + t.sh[c];
    const double s3 = t.sn[n3], s3p = t.sn[n3 + 1];
    const double P2 = S3 + s3 * s3, P2p = S3 + s3p * s3p;
    const double M = 1.0 - W3 - t.sh[n3], Mp = 1.0 - W3 - t.sh[n3 + 1];
    double s, r, sp, rp;
    site_parts(P2, M, t.ma2, &s, &r);
    site_parts(P2p, Mp, t.ma2, &sp, &rp);
    const double dot = S3 + s3 * s3p;
    acc[0] += w * (dot / (s * sp) - P2 / (s * s)) / (r * rp);
    acc[1] += w * s3p / (r * rp * sp);
    acc[2] += w / (r * r);
  }
  for (int k = 0; k < 3; ++k) {
    const double v = block_sum(acc[k], red);
    __syncthreads();
    if (threadIdx.x == 0) part[(long)blockIdx.x * 3 + k] = v;
  }
}

// deterministic final sum over the block partials (one block)
__global__ void sum_partials3(const double* part, long n, double* out) {
  __shared__ double red[33];
  for (int k = 0; k < 3; ++k) {
    double v = 0.0;
    for (long i = threadIdx.x; i < n; i += blockDim.x) v += part[i * 3 + k];
    v = block_sum(v, red);
    __syncthreads();
    if (threadIdx.x == 0) out[k] = v;
  }
}

__global__ void loop_tables(double* sn, double* sh, int N) {
  for (int n = threadIdx.x + blockIdx.x * blockDim.x; n <= N; n += blockDim.x * gridDim.x) {
    sn[n] = sinpi(2.0 * n / N);
    const double h = sinpi((double)n / N);
    sh[n] = 2.0 * h * h;
  }
}

}  // namespace
}  // namespace wz

using namespace wz;

extern "C" int wz_one_loop(int N, double ma, double* z) {
  if (!z || N < 4 || N % 2 || N > 4096 || !(ma > 0.0)) return WZ_EINVAL;
  const int H = N / 2;
  const long npairs = (long)(H + 1) * (H + 2) / 2;
  double *sn = nullptr, *part = nullptr;
  if (cudaMalloc(&sn, sizeof(double) * (2 * (N + 1) + 3 * npairs + 3)) != cudaSuccess) return WZ_ENOMEM;
  double* sh = sn + (N + 1);
  part = sh + (N + 1);
  double* out = part + 3 * npairs;
  cudaError_t e;
  count_launch(3);
  loop_tables<<<(N + 256) / 256, 256>>>(sn, sh, N);
  LoopTabs t{sn, sh, N, H, ma * ma};
  one_loop_sums<<<(unsigned)npairs, 256>>>(t, part);
  sum_partials3<<<1, 256>>>(part, npairs, out);
  double h[3] = {0, 0, 0};
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(h, out, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(sn);
  if (e != cudaSuccess) return WZ_ECUDA;
  const double n4 = (double)N * N * (double)N * N;
  const double sp = std::sin(2.0 * 3.14159265358979323846 / N);
  z[0] = h[0] / n4 / (sp * sp);
  z[1] = -h[1] / n4 / sp;
  z[2] = h[2] / n4;
  return WZ_OK;
}
