// Mixed-precision solver: FP32 iteration, FP64 reliable updates.
#include "solver_impl.cuh"
namespace wz {
template int solve_impl<float>(wz_ctx*, const cplx<double>*, cplx<double>*, int, const ShiftSpec&, double, int,
                               bool, double, SolveOut*, bool);
}  // namespace wz
