// zt passes of (Z, T) = (32, 64) in both precisions.
#include "launch_impl.cuh"
namespace wz {
template cudaError_t launch_zt_p<float, 32, 64>(int, const ZTArgs<float>&, int, cudaStream_t);
template cudaError_t launch_zt_p<double, 32, 64>(int, const ZTArgs<double>&, int, cudaStream_t);
}  // namespace wz
