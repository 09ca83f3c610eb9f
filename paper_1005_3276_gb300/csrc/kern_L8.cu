// Kernels of extent 8: every xy pass (apply, CG, force) in both precisions.
#include "launch_impl.cuh"
namespace wz {
template cudaError_t launch_xy_L<float, 8>(int, const XYArgs<float>&, cudaStream_t);
template cudaError_t launch_xy_L<double, 8>(int, const XYArgs<double>&, cudaStream_t);
template cudaError_t launch_cg_L<float, float, 8>(bool, int, const CGArgs<float, float>&, int, cudaStream_t);
template cudaError_t launch_cg_L<double, double, 8>(bool, int, const CGArgs<double, double>&, int, cudaStream_t);
template cudaError_t launch_cg_L<double, float, 8>(bool, int, const CGArgs<double, float>&, int, cudaStream_t);
template cudaError_t launch_fk_L<8>(int, const ForceArgs<double>&, dim3, cudaStream_t);
}  // namespace wz
