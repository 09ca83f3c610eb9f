// FP64 solver: FP64 iteration with a final FP64 true-residual check.
#include "solver_impl.cuh"
namespace wz {
template int solve_impl<double>(wz_ctx*, const cplx<double>*, cplx<double>*, int, const ShiftSpec&, double, int,
                               bool, double, SolveOut*, bool);
}  // namespace wz
