// FP64 instantiation of the pass sequencing.
#include "apply_impl.cuh"
namespace wz {
template int apply_op<double>(wz_ctx*, int, const cplx<double>*, cplx<double>*, int, double, cplx<double>*);
template size_t apply_ws_bytes<double>(const wz_ctx*, int, int);
}  // namespace wz
