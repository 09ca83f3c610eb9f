// Kernels of extent 6: every xy pass (apply, CG, force) in both precisions.
#include "launch_impl.cuh"
namespace wz {
template cudaError_t launch_xy_L<float, 6>(int, const XYArgs<float>&, cudaStream_t);
template cudaError_t launch_xy_L<double, 6>(int, const XYArgs<double>&, cudaStream_t);
template cudaError_t launch_cg_L<float, float, 6>(bool, int, const CGArgs<float, float>&, int, cudaStream_t);
template cudaError_t launch_cg_L<double, double, 6>(bool, int, const CGArgs<double, double>&, int, cudaStream_t);
template cudaError_t launch_cg_L<double, float, 6>(bool, int, const CGArgs<double, float>&, int, cudaStream_t);
template cudaError_t launch_fk_L<6>(int, const ForceArgs<double>&, dim3, cudaStream_t);
}  // namespace wz
