// Force and trajectory entries shared by the single-lattice and batch APIs.
#pragma once
#include "solver.h"

namespace wz {

// Forces and actions of every member at the context's phi; eta: [nm][npf]
// device fields.  ra: rational action (RHMC) or null for the single pole.
int force_impl(wz_ctx* c, const cplx<double>* eta, int npf, double tol, unsigned parts, cplx<double>* grad,
               double* S_B, double* S_pf, SolveOut* so, const wz_rational* ra = nullptr);

// One trajectory of every member; st: nm entries (may be null).  ra and rh:
// rational action and heatbath (RHMC), both or neither.
int trajectory_impl(wz_ctx* c, const wz_hmc_params* h, wz_traj_stats* st, const wz_rational* ra = nullptr,
                    const wz_rational* rh = nullptr);

}  // namespace wz
