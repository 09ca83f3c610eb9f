// Solver entry shared between the C ABI and the solver translation units.
#pragma once
#include "wz_ctx.h"

namespace wz {

struct SolveOut {
  int iterations = 0, total_iterations = 0, reliable_updates = 0, converged = 0;
  double max_true_residual = 0.0;
};

// b, x: FP64 device fields.  RI = float: FP32 iteration with FP64 reliable
// updates every time |r| drops by delta; RI = double: FP64 iteration.
// inline_capture: the caller is capturing the context stream into a larger
// graph; the solve is added to it as a WHILE conditional node (no stats).
template <typename RI>
int solve_impl(wz_ctx* c, const cplx<double>* b, cplx<double>* x, int nrhs, double shift, double tol, int maxiter,
               bool pc, double delta, SolveOut* out, bool inline_capture = false);
extern template int solve_impl<float>(wz_ctx*, const cplx<double>*, cplx<double>*, int, double, double, int, bool,
                                      double, SolveOut*, bool);
extern template int solve_impl<double>(wz_ctx*, const cplx<double>*, cplx<double>*, int, double, double, int, bool,
                                       double, SolveOut*, bool);

// FP64 true relative residuals of (M^dag M + shift) x = b for nrhs device
// fields; uses the apply workspace and synchronises the context stream.
int true_residuals(wz_ctx* c, const cplx<double>* b, const cplx<double>* x, int nrhs, double shift,
                   double* rel_out);

}  // namespace wz
