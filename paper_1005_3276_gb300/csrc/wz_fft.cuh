// Register-resident mixed-radix FFT for one line of N complex values.
//
// Plain Cooley-Tukey decimation in time with radices 4, 2 and 3, written as a
// compile-time recursion so that every index and every twiddle is a constant
// after inlining: the line lives in registers and the twiddles are read from
// a constant-bank table (cos(2 pi k / 192), N must divide 192).
//
//   X[k] = sum_n x[n] exp(DIR * 2 pi i n k / N),  DIR = -1 forward, +1 inverse
//   (no 1/N normalisation; callers fold it into the momentum-space multiply).
#pragma once
#include <cuda_runtime.h>
#include "twiddles.h"

#define WZ_HD __host__ __device__ __forceinline__

namespace wz {

template <typename R> struct cplx { R x, y; };

template <typename R> WZ_HD cplx<R> mk(R a, R b) { return cplx<R>{a, b}; }
template <typename R> WZ_HD cplx<R> operator+(cplx<R> a, cplx<R> b) { return {a.x + b.x, a.y + b.y}; }
template <typename R> WZ_HD cplx<R> operator-(cplx<R> a, cplx<R> b) { return {a.x - b.x, a.y - b.y}; }
// FP32 complex add / subtract as one packed f32x2 instruction on sm_100 and
// later (the two components are independent lanes; round to nearest as the
// scalar forms)
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
__device__ __forceinline__ unsigned long long f2_pack(cplx<float> a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ cplx<float> f2_unpack(unsigned long long r) {
  cplx<float> a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
#endif
WZ_HD cplx<float> operator+(cplx<float> a, cplx<float> b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(d);
#else
  return {a.x + b.x, a.y + b.y};
#endif
}
WZ_HD cplx<float> operator-(cplx<float> a, cplx<float> b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(d);
#else
  return {a.x - b.x, a.y - b.y};
#endif
}
template <typename R> WZ_HD cplx<R> operator*(cplx<R> a, cplx<R> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename R> WZ_HD cplx<R> operator*(R s, cplx<R> a) { return {s * a.x, s * a.y}; }
template <typename R> WZ_HD cplx<R> conj(cplx<R> a) { return {a.x, -a.y}; }
// multiply by +i or -i
template <typename R> WZ_HD cplx<R> mul_i(cplx<R> a) { return {-a.y, a.x}; }
template <typename R> WZ_HD cplx<R> mul_mi(cplx<R> a) { return {a.y, -a.x}; }
// a * conj(b) summed real part helpers
template <typename R> WZ_HD R re_conj_mul(cplx<R> a, cplx<R> b) { return a.x * b.x + a.y * b.y; }

static __constant__ double c_tw64[WZ_TW_N] = {WZ_TW_TABLE};
static __constant__ float c_tw32[WZ_TW_N] = {WZ_TW_TABLE};
// host copies so that the same templates can be exercised on the CPU
static const double h_tw64[WZ_TW_N] = {WZ_TW_TABLE};

template <typename R> struct Tw;
template <> struct Tw<double> {
  static WZ_HD double cosk(int k) {
#ifdef __CUDA_ARCH__
    return c_tw64[k];
#else
    return h_tw64[k];
#endif
  }
};
template <> struct Tw<float> {
  static WZ_HD float cosk(int k) {
#ifdef __CUDA_ARCH__
    return c_tw32[k];
#else
    return float(h_tw64[k]);
#endif
  }
};

// exp(DIR * 2 pi i j / N) * a, with the trivial angles done exactly.
template <int N, int DIR, typename R>
WZ_HD cplx<R> twiddle(cplx<R> a, int j) {
  j = ((j % N) + N) % N;
  if (j == 0) return a;
  if (4 * j == N) return DIR < 0 ? mul_mi(a) : mul_i(a);
  if (2 * j == N) return cplx<R>{-a.x, -a.y};
  if (4 * j == 3 * N) return DIR < 0 ? mul_i(a) : mul_mi(a);
  constexpr int S = WZ_TW_N / N;
  const int k = j * S;
  const R c = Tw<R>::cosk(k);
  const R s = Tw<R>::cosk((k + 3 * WZ_TW_N / 4) % WZ_TW_N);  // sin(theta) = cos(theta - pi/2)
  const R sd = DIR < 0 ? -s : s;
  return cplx<R>{a.x * c - a.y * sd, a.x * sd + a.y * c};
}

template <int R_, int DIR, typename R> struct Butterfly;
template <int DIR, typename R> struct Butterfly<2, DIR, R> {
  static WZ_HD void run(cplx<R>* t) {
    cplx<R> a = t[0], b = t[1];
    t[0] = a + b;
    t[1] = a - b;
  }
};
template <int DIR, typename R> struct Butterfly<4, DIR, R> {
  static WZ_HD void run(cplx<R>* t) {
    cplx<R> t0 = t[0] + t[2], t1 = t[0] - t[2], t2 = t[1] + t[3], d = t[1] - t[3];
    cplx<R> t3 = DIR < 0 ? mul_mi(d) : mul_i(d);
    t[0] = t0 + t2;
    t[2] = t0 - t2;
    t[1] = t1 + t3;
    t[3] = t1 - t3;
  }
};
template <int DIR, typename R> struct Butterfly<3, DIR, R> {
  static WZ_HD void run(cplx<R>* t) {
    const R h = R(0.86602540378443864676);  // sqrt(3)/2
    cplx<R> s = t[1] + t[2], d = t[1] - t[2];
    cplx<R> a = t[0] - R(0.5) * s;
    cplx<R> b = (DIR < 0 ? -h : h) * mul_i(d);
    t[0] = t[0] + s;
    t[1] = a + b;
    t[2] = a - b;
  }
};

template <int N> struct FirstRadix {
  static constexpr int value = (N % 4 == 0 && N != 8 && N != 4) ? 4 : (N == 4 ? 4 : (N % 2 == 0 ? 2 : 3));
};

// out[k], k = 0..N-1 (contiguous) = DFT of in[IS * n], n = 0..N-1.
template <int N, int DIR, typename R> struct Fft {
  template <int IS>
  static WZ_HD void run(const cplx<R>* in, cplx<R>* out) {
    constexpr int RX = FirstRadix<N>::value;
    constexpr int M = N / RX;
    static_assert(RX * M == N, "unsupported FFT length");
    cplx<R> sub[N];
#pragma unroll
    for (int r = 0; r < RX; ++r) Fft<M, DIR, R>::template run<IS * RX>(in + r * IS, sub + r * M);
#pragma unroll
    for (int k = 0; k < M; ++k) {
      cplx<R> t[RX];
#pragma unroll
      for (int r = 0; r < RX; ++r) t[r] = twiddle<N, DIR, R>(sub[r * M + k], r * k);
      Butterfly<RX, DIR, R>::run(t);
#pragma unroll
      for (int q = 0; q < RX; ++q) out[k + M * q] = t[q];
    }
  }
};
template <int DIR, typename R> struct Fft<1, DIR, R> {
  template <int IS>
  static WZ_HD void run(const cplx<R>* in, cplx<R>* out) { out[0] = in[0]; }
};

// In-place convenience wrapper.
template <int N, int DIR, typename R>
WZ_HD void fft_line(cplx<R> (&v)[N]) {
  cplx<R> out[N];
  Fft<N, DIR, R>::template run<1>(v, out);
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = out[i];
}

// Same, on the first N entries of a longer register array.
template <int N, int DIR, typename R>
WZ_HD void fft_ptr(cplx<R>* v) {
  cplx<R> out[N];
  Fft<N, DIR, R>::template run<1>(v, out);
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = out[i];
}

}  // namespace wz
