// Host-side launch interface: per-extent launchers are explicit template
// instantiations in their own translation units (kern_L*.cu, zt_*.cu), so the
// host code here only dispatches on the run-time extent.
#pragma once
#include <utility>

#include "wz_ctx.h"
#include "wz_hmc.cuh"
#include "wz_probe.h"

// extents with compiled kernels; the xy pass needs X == Y, the zt pass a (Z, T) pair
#define WZ_FOR_EXTENTS(F) F(4) F(6) F(8) F(12) F(16) F(32)
#define WZ_FOR_ZT_PAIRS(F) F(4, 4) F(6, 6) F(8, 8) F(12, 12) F(16, 16) F(32, 32) F(8, 16) F(16, 32) F(8, 32) F(32, 64)

namespace wz {

enum { FK_FORCE = 0, FK_BOSON_FWD = 1, FK_BOSON_INV = 2 };

// Launch k on st, with programmatic stream serialization when pdl is set (the
// kernel may then be scheduled while its predecessor on st finishes; it waits
// for it in pdl_wait before touching memory).
template <typename... KArgs, typename... Args>
static cudaError_t launch_k(bool pdl, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                            Args&&... args) {
  if (!pdl) {
    k<<<grid, block, smem, st>>>(std::forward<Args>(args)...);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

template <typename Kern>
static cudaError_t set_smem(Kern k, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Blocks of a persistent kernel that are resident at once on the current
// device: SMs x blocks per SM (occupancy at the launch's threads and dynamic
// shared memory), looked up once per device.
struct ResidentBlocks {
  int n[64] = {};
  template <typename Kern>
  cudaError_t get(Kern k, int threads, size_t smem, int* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && n[dev] > 0) {
      *out = n[dev];
      return cudaSuccess;
    }
    int sms = 0, per = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, threads, smem)) != cudaSuccess) return e;
    const int r = (per > 0 ? per : 1) * sms;
    if (dev >= 0 && dev < 64) n[dev] = r;
    *out = r;
    return cudaSuccess;
  }
};

// The dynamic shared-memory attribute is a property of a kernel on one device:
// a process that drives several devices sets it once on each of them.
#define WZ_MAX_DEVICES 64
struct SmemAttrDone {
  bool done[WZ_MAX_DEVICES] = {};
};
template <typename Kern>
static cudaError_t set_smem_once(Kern k, size_t bytes, SmemAttrDone& d) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= WZ_MAX_DEVICES) return set_smem(k, bytes);  // beyond the table: every launch
  if (d.done[dev]) return cudaSuccess;
  e = set_smem(k, bytes);
  if (e == cudaSuccess) d.done[dev] = true;
  return e;
}

template <typename R, int L> cudaError_t launch_xy_L(int mode, const XYArgs<R>& a, cudaStream_t st);
template <typename R, typename LO, int L>
cudaError_t launch_cg_L(bool pc, int mode, const CGArgs<R, LO>& a, int nrhs, cudaStream_t st);
template <int L> cudaError_t launch_fk_L(int which, const ForceArgs<double>& a, dim3 grid, cudaStream_t st);
template <typename R, int NZ, int NT> cudaError_t launch_zt_p(int mul, const ZTArgs<R>& a, int nrhs, cudaStream_t st);

#define WZ_DECL_L(n)                                                                                        \
  extern template cudaError_t launch_xy_L<float, n>(int, const XYArgs<float>&, cudaStream_t);              \
  extern template cudaError_t launch_xy_L<double, n>(int, const XYArgs<double>&, cudaStream_t);            \
  extern template cudaError_t launch_cg_L<float, float, n>(bool, int, const CGArgs<float, float>&, int,     \
                                                           cudaStream_t);                                   \
  extern template cudaError_t launch_cg_L<double, double, n>(bool, int, const CGArgs<double, double>&, int, \
                                                             cudaStream_t);                                 \
  extern template cudaError_t launch_cg_L<double, float, n>(bool, int, const CGArgs<double, float>&, int,   \
                                                            cudaStream_t);                                  \
  extern template cudaError_t launch_fk_L<n>(int, const ForceArgs<double>&, dim3, cudaStream_t);
WZ_FOR_EXTENTS(WZ_DECL_L)
#undef WZ_DECL_L
#define WZ_DECL_ZT(z, t)                                                                            \
  extern template cudaError_t launch_zt_p<float, z, t>(int, const ZTArgs<float>&, int, cudaStream_t); \
  extern template cudaError_t launch_zt_p<double, z, t>(int, const ZTArgs<double>&, int, cudaStream_t);
WZ_FOR_ZT_PAIRS(WZ_DECL_ZT)
#undef WZ_DECL_ZT

template <typename R>
inline cudaError_t launch_xy(int L, int mode, const XYArgs<R>& a, cudaStream_t st) {
  switch (L) {
#define WZ_CASE(n) \
  case n: return launch_xy_L<R, n>(mode, a, st);
    WZ_FOR_EXTENTS(WZ_CASE)
#undef WZ_CASE
  }
  return cudaErrorInvalidValue;
}

template <typename R>
inline cudaError_t launch_zt(int nz, int nt, int mul, const ZTArgs<R>& a, int nrhs, cudaStream_t st) {
#define WZ_CASE(z, t) \
  if (nz == z && nt == t) return launch_zt_p<R, z, t>(mul, a, nrhs, st);
  WZ_FOR_ZT_PAIRS(WZ_CASE)
#undef WZ_CASE
  return cudaErrorInvalidValue;
}

template <typename R, typename LO>
inline cudaError_t launch_cg(int L, bool pc, int mode, const CGArgs<R, LO>& a, int nrhs, cudaStream_t st) {
  switch (L) {
#define WZ_CASE(n) \
  case n: return launch_cg_L<R, LO, n>(pc, mode, a, nrhs, st);
    WZ_FOR_EXTENTS(WZ_CASE)
#undef WZ_CASE
  }
  return cudaErrorInvalidValue;
}

inline cudaError_t launch_fk(int L, int which, const ForceArgs<double>& a, dim3 grid, cudaStream_t st) {
  switch (L) {
#define WZ_CASE(n) \
  case n: return launch_fk_L<n>(which, a, grid, st);
    WZ_FOR_EXTENTS(WZ_CASE)
#undef WZ_CASE
  }
  return cudaErrorInvalidValue;
}

// blocks of an xy pass over the T*Z planes of one field
inline int xy_nblk(int L, int TZ) {
  switch (L) {
#define WZ_CASE(n) \
  case n: return (TZ + XYShape<n>::PPC - 1) / XYShape<n>::PPC;
    WZ_FOR_EXTENTS(WZ_CASE)
#undef WZ_CASE
  }
  return 0;
}

}  // namespace wz
