// FP32 instantiation of the pass sequencing (inner solver precision).
#include "apply_impl.cuh"
namespace wz {
template int apply_op<float>(wz_ctx*, int, const cplx<float>*, cplx<float>*, int, float, cplx<float>*);
template size_t apply_ws_bytes<float>(const wz_ctx*, int, int);
}  // namespace wz
