// wz_apply_mdagm_noalloc: the fused (M^dagger M + shift) apply without any
// device allocation at call time.
//
// wz_apply keeps its pass intermediates (the momentum-space field A and the
// position-space M psi) in a context workspace that grows with cudaMalloc on
// demand.  Some callers cannot allow that: a caller that has handed all device
// memory to its own pool, a latency-critical loop in which cudaMalloc (which
// may synchronise the device) is not acceptable, or code that must not fail
// half-way through on an out-of-memory error.  This variant runs the same
// five pass kernels with the intermediates in a file-scope device array of a
// fixed size instead.
//
// The array is part of this library's device image: every GPU that loads the
// library holds it (WZ_NOALLOC_SCRATCH_BYTES) until the process exits.  Host
// code cannot use the array's name as a device address (in host code it is a
// host-side stand-in); its device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on
// that device.  That first call may load the library's device code on the
// device, so make it during set-up, before any stream capture.
//
// All calls share the array and it keeps the contents of the last call.
// Nothing in it has to start at zero: every byte a call reads was written
// earlier in the same call.  Calls that overlap on the GPU (different streams,
// or different threads) race on the array and must be serialised by the caller.
#include <mutex>

#include "apply_impl.cuh"
#include "wz_ctx.h"

#define WZ_NOALLOC_SCRATCH_BYTES (32u << 20)
#define WZ_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_noalloc_scratch[WZ_NOALLOC_SCRATCH_BYTES];

namespace wz {
extern template int apply_op<float>(wz_ctx*, int, const cplx<float>*, cplx<float>*, int, float, cplx<float>*);
extern template int apply_op<double>(wz_ctx*, int, const cplx<double>*, cplx<double>*, int, double, cplx<double>*);
extern template size_t apply_ws_bytes<float>(const wz_ctx*, int, int);
extern template size_t apply_ws_bytes<double>(const wz_ctx*, int, int);
}  // namespace wz

namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_addr[WZ_NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on device dev (which must be current).
int noalloc_scratch(wz_ctx* c, int dev, void** out) {
  if (dev < 0 || dev >= WZ_NOALLOC_MAX_DEVICES) return wz::set_error(c, WZ_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return wz::cuda_error(c, e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return WZ_OK;
}

}  // namespace

extern "C" int wz_apply_mdagm_noalloc(wz_ctx* c, int dtype, const void* in, void* out, int nrhs, double shift) {
  using namespace wz;
  if (!c) return WZ_EINVAL;
  if (!in || !out || nrhs < 0) return set_error(c, WZ_EINVAL, "wz_apply_mdagm_noalloc: bad argument");
  if (dtype != WZ_C64 && dtype != WZ_C128) return set_error(c, WZ_EINVAL, "wz_apply_mdagm_noalloc: unknown dtype");
  if (nrhs == 0) return WZ_OK;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(c, e, "cudaGetDevice");
  if (dev != c->device)
    return set_error(c, WZ_EINVAL, "wz_apply_mdagm_noalloc: make the context's device current first");
  if (!is_device_pointer(in) || !is_device_pointer(out))
    return set_error(c, WZ_EINVAL, "wz_apply_mdagm_noalloc: in and out must be device pointers");
  const size_t need = dtype == WZ_C128 ? apply_ws_bytes<double>(c, WZ_OP_MDAGM, nrhs)
                                       : apply_ws_bytes<float>(c, WZ_OP_MDAGM, nrhs);
  if (need > WZ_NOALLOC_SCRATCH_BYTES)
    return set_error(c, WZ_EINVAL,
                     "wz_apply_mdagm_noalloc: this call needs " + std::to_string(need) +
                         " bytes of scratch but the static scratch holds " +
                         std::to_string((size_t)WZ_NOALLOC_SCRATCH_BYTES) + " bytes; use fewer right-hand sides or wz_apply");
  void* scratch = nullptr;
  int rc = noalloc_scratch(c, dev, &scratch);
  if (rc) return rc;
  if (dtype == WZ_C128)
    return apply_op<double>(c, WZ_OP_MDAGM, (const cplx<double>*)in, (cplx<double>*)out, nrhs, shift,
                            (cplx<double>*)scratch);
  return apply_op<float>(c, WZ_OP_MDAGM, (const cplx<float>*)in, (cplx<float>*)out, nrhs, (float)shift,
                         (cplx<float>*)scratch);
}
