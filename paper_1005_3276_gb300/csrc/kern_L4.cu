// Kernels of extent 4: every xy pass (apply, CG, force) in both precisions.
#include "launch_impl.cuh"
namespace wz {
template cudaError_t launch_xy_L<float, 4>(int, const XYArgs<float>&, cudaStream_t);
template cudaError_t launch_xy_L<double, 4>(int, const XYArgs<double>&, cudaStream_t);
template cudaError_t launch_cg_L<float, float, 4>(bool, int, const CGArgs<float, float>&, int, cudaStream_t);
template cudaError_t launch_cg_L<double, double, 4>(bool, int, const CGArgs<double, double>&, int, cudaStream_t);
template cudaError_t launch_cg_L<double, float, 4>(bool, int, const CGArgs<double, float>&, int, cudaStream_t);
template cudaError_t launch_fk_L<4>(int, const ForceArgs<double>&, dim3, cudaStream_t);
}  // namespace wz
