// Solver entry shared between the C ABI and the solver translation units.
#pragma once
#include "wz_ctx.h"
#include "wz_cg.cuh"

namespace wz {

struct SolveOut {
  int iterations = 0, total_iterations = 0, reliable_updates = 0, converged = 0;
  double max_true_residual = 0.0;
};

// b, x: FP64 device fields.  RI = float: FP32 iteration with FP64 reliable
// updates every time |r| drops by delta; RI = double: FP64 iteration.
// inline_capture: the caller is capturing the context stream into a larger
// graph; the solve is added to it as a WHILE conditional node (no stats).
// nrhs systems; system q solves (M^dag M + sh.of(q)) x_q = b[sh.src(q)] (x has
// nrhs fields, b as many as sh.src addresses).  Preconditioned shifted systems
// are solved in the form M~^dag M~ + sigma M0^-1^dag M0^-1 (Sec. 7.4).
template <typename RI>
int solve_impl(wz_ctx* c, const cplx<double>* b, cplx<double>* x, int nrhs, const ShiftSpec& sh, double tol,
               int maxiter, bool pc, double delta, SolveOut* out, bool inline_capture = false);
extern template int solve_impl<float>(wz_ctx*, const cplx<double>*, cplx<double>*, int, const ShiftSpec&, double,
                                      int, bool, double, SolveOut*, bool);
extern template int solve_impl<double>(wz_ctx*, const cplx<double>*, cplx<double>*, int, const ShiftSpec&, double,
                                       int, bool, double, SolveOut*, bool);

// the same shift for every system
inline ShiftSpec single_shift(double shift) {
  ShiftSpec s;
  s.beta[0] = shift;
  return s;
}

// FP64 true relative residuals of (M^dag M + shift) x = b for nrhs device
// fields; uses the apply workspace and synchronises the context stream.
// b[sh.src(q)] is the right-hand side of system q.
int true_residuals(wz_ctx* c, const cplx<double>* b, const cplx<double>* x, int nrhs, const ShiftSpec& sh,
                   double* rel_out);

}  // namespace wz
