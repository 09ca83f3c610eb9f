// zt passes of (Z, T) = (4, 4) in both precisions.
#include "launch_impl.cuh"
namespace wz {
template cudaError_t launch_zt_p<float, 4, 4>(int, const ZTArgs<float>&, int, cudaStream_t);
template cudaError_t launch_zt_p<double, 4, 4>(int, const ZTArgs<double>&, int, cudaStream_t);
}  // namespace wz
