// r(M^dag M) applied through shifted solves (Eq. jkjk, Eq. yuier, Sec. 7.4).
//
//   out = a0 in + sum_i alpha_i X_i,   (M^dag M + beta_i) X_i = in
//
// All d shifted systems of all right-hand sides run as one batched CG (one
// right-hand side per system, each stopping on its own residual); with the
// preconditioning flag the poles up to the cut-off are solved in the M0^-1
// preconditioned form of Sec. 7.4 and the rest without, as two solves.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "solver.h"
#include "wz_hmc.cuh"
#include "wz_probe.h"

using namespace wz;

extern "C" int wz_rational_apply(wz_ctx* c, const wz_rational* r, const void* in, void* out, int nrhs, double tol,
                                 int maxiter, unsigned flags, double pc_cutoff, wz_solve_stats* stats) {
  if (!c) return WZ_EINVAL;
  if (!r || !in || !out || in == out || nrhs < 0 || tol <= 0.0 || maxiter < 1 || r->d < 0 || r->d > WZ_RATIONAL_MAX ||
      !std::isfinite(r->a0))
    return set_error(c, WZ_EINVAL, "wz_rational_apply: bad argument");
  for (int i = 0; i < r->d; ++i)
    if (!(r->beta[i] >= 0.0) || !std::isfinite(r->alpha[i]))
      return set_error(c, WZ_EINVAL, "wz_rational_apply: shifts must be >= 0 and residues finite");
  if (c->nm > 1 && nrhs % c->nm) return set_error(c, WZ_EINVAL, "wz_rational_apply: nrhs must be a multiple of the members");
  const bool pc = (flags & WZ_SOLVE_PC) != 0;
  if (pc && (c->nm > 1 || !c->same_mass))
    return set_error(c, WZ_EINVAL, "wz_rational_apply: preconditioned poles need a single-lattice context");
  const auto t0 = std::chrono::steady_clock::now();
  if (stats) *stats = wz_solve_stats{};
  if (nrhs == 0) return WZ_OK;

  const long n4 = 4L * c->V;
  const size_t f1 = sizeof(cplx<double>) * (size_t)n4, fb = f1 * nrhs;
  const bool din = is_device_pointer(in), dout = is_device_pointer(out);
  const cplx<double>* pin = (const cplx<double>*)in;
  cplx<double>* pout = (cplx<double>*)out;
  if (!din || !dout) {
    WZ_CUDA_TRY(c, c->ws_stage.reserve(2 * fb));
    cplx<double>* sb = (cplx<double>*)c->ws_stage.ptr;
    if (!din) {
      WZ_CUDA_TRY(c, cudaMemcpyAsync(sb, in, fb, cudaMemcpyHostToDevice, c->stream));
      pin = sb;
    }
    if (!dout) pout = sb + n4 * nrhs;
  }
  const int d = r->d;
  const int inner = c->nm > 1 ? nrhs / c->nm : nrhs;
  // pole order: ascending shift, the preconditioned ones (beta <= cut-off) first
  std::vector<int> ord(d);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return r->beta[a] < r->beta[b]; });
  int npc = 0;
  if (pc)
    while (npc < d && r->beta[ord[npc]] <= pc_cutoff) ++npc;
  PoleSum ps;
  ps.d = d;
  ps.inner = inner;
  ps.a0 = r->a0;
  for (int q = 0; q < d; ++q) ps.alpha[q] = r->alpha[ord[q]];

  SolveOut acc;
  int status = WZ_OK;
  cplx<double>* X = nullptr;
  if (d > 0) {
    WZ_CUDA_TRY(c, c->ws_rat.reserve(fb * d));
    X = (cplx<double>*)c->ws_rat.ptr;
    // systems [pole][rhs] for one lattice ([member][pole][rhs] in general: one solve)
    auto run = [&](int p0, int np, bool with_pc) -> int {
      ShiftSpec sh;
      sh.d = np;
      sh.inner = inner;
      for (int q = 0; q < np; ++q) sh.beta[q] = r->beta[ord[p0 + q]];
      SolveOut o;
      cplx<double>* xs = X + (long)p0 * inner * n4;
      int rc = (flags & WZ_SOLVE_MIXED)
                   ? solve_impl<float>(c, pin, xs, np * nrhs, sh, tol, maxiter, with_pc, 0.1, &o)
                   : solve_impl<double>(c, pin, xs, np * nrhs, sh, tol, maxiter, with_pc, 0.0, &o);
      acc.total_iterations += o.total_iterations;
      acc.reliable_updates += o.reliable_updates;
      acc.converged += o.converged;
      acc.iterations = std::max(acc.iterations, o.iterations);
      acc.max_true_residual = std::max(acc.max_true_residual, o.max_true_residual);
      return rc;
    };
    int rc = WZ_OK;
    if (npc > 0) rc = run(0, npc, true);
    if ((rc == WZ_OK || rc == WZ_NOT_CONVERGED) && npc < d) {
      const int rc2 = run(npc, d - npc, false);
      rc = rc == WZ_OK ? rc2 : rc;
    }
    if (rc != WZ_OK && rc != WZ_NOT_CONVERGED) return rc;
    status = rc;
  }
  count_launch();
  pole_combine<<<dim3(64, nrhs), 256, 0, c->stream>>>(pin, X ? X : pout, pout, n4, ps);
  WZ_CUDA_TRY(c, cudaGetLastError());
  if (!dout) WZ_CUDA_TRY(c, cudaMemcpyAsync(out, pout, fb, cudaMemcpyDeviceToHost, c->stream));
  WZ_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (stats) {
    stats->iterations = acc.iterations;
    stats->total_iterations = acc.total_iterations;
    stats->reliable_updates = acc.reliable_updates;
    stats->converged = acc.converged;
    stats->max_true_residual = acc.max_true_residual;
    stats->site_applies = (double)(acc.total_iterations + acc.reliable_updates) * (double)c->V;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (status == WZ_NOT_CONVERGED) set_error(c, status, "wz_rational_apply: a shifted solve reached maxiter");
  return status;
}
