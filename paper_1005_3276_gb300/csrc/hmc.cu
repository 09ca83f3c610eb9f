// Forces, actions, molecular dynamics and HMC trajectories (host sequencing).
//
// force(phi):  X_k = (M^dag M)^-1 eta_k   (one batched CG over the npf pseudofermions)
//              G_k = site contraction of Z_k = M X_k with X_k         (xy_force)
//              G   = G_B(phi) + sum_k G_k, S_B partials                (xy_boson_inv)
// The leapfrog / Omelyan integrators and the Metropolis step follow Sec. 7.2;
// the state (phi, pi) stays in FP64 on the device throughout.
#include <chrono>
#include <cstring>
#include <vector>

#include "apply_impl.cuh"
#include "solver.h"
#include "wz_hmc.cuh"

namespace wz {

enum { FK_FORCE = 0, FK_BOSON_FWD = 1, FK_BOSON_INV = 2 };

template <int L>
static cudaError_t launch_fk_L(int which, const ForceArgs<double>& a, dim3 grid, cudaStream_t st) {
  using S = XYShape<L>;
  const size_t smem = sizeof(cplx<double>) * S::PLANE * S::PPC + 33 * sizeof(double);
  static bool done[3] = {false, false, false};
  cudaError_t e = cudaSuccess;
  if (!done[which]) {
    if (which == FK_FORCE) e = set_smem(xy_force<L>, smem);
    if (which == FK_BOSON_FWD) e = set_smem(xy_boson_fwd<L>, smem);
    if (which == FK_BOSON_INV) e = set_smem(xy_boson_inv<L>, smem);
    if (e != cudaSuccess) return e;
    done[which] = true;
  }
  ++g_launches;
  if (which == FK_FORCE) xy_force<L><<<grid, S::THREADS, smem, st>>>(a);
  if (which == FK_BOSON_FWD) xy_boson_fwd<L><<<grid, S::THREADS, smem, st>>>(a);
  if (which == FK_BOSON_INV) xy_boson_inv<L><<<grid, S::THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_fk(int L, int which, const ForceArgs<double>& a, dim3 grid, cudaStream_t st) {
  switch (L) {
#define WZ_CASE(n) \
  case n: return launch_fk_L<n>(which, a, grid, st);
    WZ_FOR_EXTENTS(WZ_CASE)
#undef WZ_CASE
  }
  return cudaErrorInvalidValue;
}

static int xy_blocks(int L, int TZ) {
  switch (L) {
#define WZ_CASE(n) \
  case n: return (TZ + XYShape<n>::PPC - 1) / XYShape<n>::PPC;
    WZ_FOR_EXTENTS(WZ_CASE)
#undef WZ_CASE
  }
  return 0;
}

static unsigned grid1d(long n) {
  long b = (n + 255) / 256;
  return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

// Workspace of the force / MD code (FP64), carved from ctx->ws_force.
struct ForceWS {
  cplx<double>* X;     // [npf][V][4] solutions
  cplx<double>* A;     // [npf][V][4] momentum intermediate
  cplx<double>* Gk;    // [npf][V] per-pseudofermion forces
  cplx<double>* Bk;    // [V][4] packed scalar field / its transform
  cplx<double>* G;     // [V] total force
  cplx<double>* pi;    // [V] momenta
  cplx<double>* phi0;  // [V] phi at the start of the trajectory
  cplx<double>* R;     // [npf][V][4] heatbath sources
  cplx<double>* eta;   // [npf][V][4] pseudofermions
  double* sb0;         // S_B partials at the start
  double* sb1;         // S_B partials of the latest force evaluation
  double* kin0;        // |pi|^2 partials at the start
  double* kin1;
  double* spf0;        // |R|^2 partials
  double* spf1;        // Re eta^dag X partials
  double* res;         // metropolis result [H0, H1, dH, u, accept]
  int nb;              // xy blocks for one field
};

static const int NPART = 4096;  // partial arrays are sized for the largest grid used

static int force_ws(wz_ctx* c, int npf, ForceWS* w) {
  const size_t f4 = sizeof(cplx<double>) * 4 * (size_t)c->V;
  const size_t f1 = sizeof(cplx<double>) * (size_t)c->V;
  size_t off = 0;
  auto take = [&](size_t n) {
    size_t r = off;
    off += (n + 255) & ~size_t(255);
    return r;
  };
  const size_t oX = take(f4 * npf), oA = take(f4 * npf), oGk = take(f1 * npf), oB = take(f4), oG = take(f1),
               oPi = take(f1), oP0 = take(f1), oR = take(f4 * npf), oE = take(f4 * npf),
               oParts = take(sizeof(double) * (6 * NPART + 8));
  WZ_CUDA_TRY(c, c->ws_force.reserve(off));
  char* b = (char*)c->ws_force.ptr;
  w->X = (cplx<double>*)(b + oX);
  w->A = (cplx<double>*)(b + oA);
  w->Gk = (cplx<double>*)(b + oGk);
  w->Bk = (cplx<double>*)(b + oB);
  w->G = (cplx<double>*)(b + oG);
  w->pi = (cplx<double>*)(b + oPi);
  w->phi0 = (cplx<double>*)(b + oP0);
  w->R = (cplx<double>*)(b + oR);
  w->eta = (cplx<double>*)(b + oE);
  double* p = (double*)(b + oParts);
  w->sb0 = p;
  w->sb1 = p + NPART;
  w->kin0 = p + 2 * NPART;
  w->kin1 = p + 3 * NPART;
  w->spf0 = p + 4 * NPART;
  w->spf1 = p + 5 * NPART;
  w->res = p + 6 * NPART;
  w->nb = xy_blocks(c->X, c->T * c->Z);
  if (w->nb > NPART) return set_error(c, WZ_EINVAL, "lattice too large for the force partials");
  return WZ_OK;
}

struct ForceOpts {
  double tol = 1e-10;
  int maxiter = 100000;
  bool mixed = true;
  bool fermion = true;
  bool boson = true;
};

// G = dS/dphi for the current phi; S_B partials into sb_part (nb values).
// On return X holds (M^dag M)^-1 eta.
static int force_eval(wz_ctx* c, const ForceWS& w, const cplx<double>* eta, int npf, const ForceOpts& o,
                      double* sb_part, SolveOut* so) {
  cudaStream_t s = c->stream;
  const int L = c->X;
  const int TZ = c->T * c->Z;
  cudaError_t e;
  int npf_eff = o.fermion ? npf : 0;
  if (npf_eff > 0) {
    int rc = o.mixed ? solve_impl<float>(c, eta, w.X, npf, 0.0, o.tol, o.maxiter, false, 0.1, so)
                     : solve_impl<double>(c, eta, w.X, npf, 0.0, o.tol, o.maxiter, false, 0.0, so);
    if (rc) return rc;
    // Z = M X without the site term: forward xy, +Dslash; the site term and the
    // contraction are fused into xy_force
    XYArgs<double> xa{};
    xa.phi = c->phi64;
    xa.k = site_coef_of<double>(c);
    xa.nplanes = npf * TZ;
    xa.TZ = TZ;
    xa.psi = w.X;
    xa.A_out = w.A;
    e = launch_xy<double>(L, XY_FWD, xa, s);
    if (e != cudaSuccess) return cuda_error(c, e, "force: xy forward");
    ZTArgs<double> za = zt_args<double>(c, 1.0);
    za.A = w.A;
    e = launch_zt<double>(c->Z, c->T, ZT_DSLASH, za, npf, s);
    if (e != cudaSuccess) return cuda_error(c, e, "force: zt");
    ForceArgs<double> fa{};
    fa.A = w.A;
    fa.X = w.X;
    fa.Gk = w.Gk;
    fa.phi = c->phi64;
    fa.k = site_coef_of<double>(c);
    fa.TZ = TZ;
    fa.V = c->V;
    e = launch_fk(L, FK_FORCE, fa, dim3(w.nb, npf), s);
    if (e != cudaSuccess) return cuda_error(c, e, "force: xy_force");
  }
  // bosonic part (+ the sum of the fermion forces)
  ForceArgs<double> ba{};
  ba.phi = c->phi64;
  ba.k = site_coef_of<double>(c);  // the boson kernels use k.m; W' uses g itself
  ba.g_re = c->p.g_re;
  ba.g_im = c->p.g_im;
  ba.TZ = TZ;
  ba.V = c->V;
  ba.A_out = w.Bk;
  ba.A = w.Bk;
  ba.Gk_in = w.Gk;
  ba.npf = npf_eff;
  ba.G = w.G;
  ba.part = sb_part;
  if (o.boson) {
    e = launch_fk(L, FK_BOSON_FWD, ba, dim3(w.nb), s);
    if (e != cudaSuccess) return cuda_error(c, e, "force: boson forward");
    ZTArgs<double> za = zt_args<double>(c, 1.0);
    za.A = w.Bk;
    e = launch_zt<double>(c->Z, c->T, ZT_SCALAR, za, 1, s);
    if (e != cudaSuccess) return cuda_error(c, e, "force: boson zt");
  } else {
    // zero scalar transform: the inverse pass then only sums the fermion forces
    e = cudaMemsetAsync(w.Bk, 0, sizeof(cplx<double>) * 4 * c->V, s);
    if (e != cudaSuccess) return cuda_error(c, e, "force: memset");
  }
  e = launch_fk(L, FK_BOSON_INV, ba, dim3(w.nb), s);
  if (e != cudaSuccess) return cuda_error(c, e, "force: boson inverse");
  return WZ_OK;
}

static double host_sum(wz_ctx* c, const double* dev, int n, double* pinned) {
  cudaMemcpyAsync(pinned, dev, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream);
  cudaStreamSynchronize(c->stream);
  double t = 0.0;
  for (int i = 0; i < n; ++i) t += pinned[i];
  return t;
}

static void add_solve(SolveOut& acc, const SolveOut& s) {
  acc.total_iterations += s.total_iterations;
  acc.reliable_updates += s.reliable_updates;
  acc.iterations = acc.iterations > s.iterations ? acc.iterations : s.iterations;
  acc.converged += s.converged;
  acc.max_true_residual = acc.max_true_residual > s.max_true_residual ? acc.max_true_residual : s.max_true_residual;
}

// Molecular dynamics: phi (context) and w.pi evolve in place.  On return w.G,
// w.X and w.sb1 belong to the final phi.  nforce counts force evaluations.
static int md_integrate(wz_ctx* c, ForceWS& w, const cplx<double>* eta, int npf, double tau, int nsteps,
                        int integrator, const ForceOpts& o, SolveOut* acc, int* nforce, bool first_into_sb0) {
  cudaStream_t s = c->stream;
  const long V = c->V;
  const double eps = tau / nsteps;
  const unsigned g = grid1d(V);
  SolveOut so;
  int rc;
  auto F = [&](bool first) {
    SolveOut one;
    int r = force_eval(c, w, eta, npf, o, (first && first_into_sb0) ? w.sb0 : w.sb1, &one);
    add_solve(*acc, one);
    ++*nforce;
    if (r == WZ_NOT_CONVERGED) return set_error(c, r, "force: solver did not converge");
    return r;
  };
  auto P = [&](double h) {
    g_launches++;
    update_pi<<<g, 256, 0, s>>>(w.pi, w.G, h, V);
    return cudaGetLastError();
  };
  auto Q = [&](double h) {
    g_launches++;
    update_phi<<<g, 256, 0, s>>>(c->phi64, c->phi32, w.pi, h, V);
    return cudaGetLastError();
  };
  if (integrator == 0) {  // leapfrog
    if ((rc = F(true))) return rc;
    WZ_CUDA_TRY(c, P(0.5 * eps));
    for (int k = 0; k < nsteps; ++k) {
      WZ_CUDA_TRY(c, Q(eps));
      if ((rc = F(false))) return rc;
      WZ_CUDA_TRY(c, P(k < nsteps - 1 ? eps : 0.5 * eps));
    }
  } else {  // Omelyan 2MN: P(l e) Q(e/2) P((1-2l) e) Q(e/2) P(l e); the last force is reused
    const double lam = 0.1931833275037836;
    if ((rc = F(true))) return rc;
    for (int k = 0; k < nsteps; ++k) {
      WZ_CUDA_TRY(c, P(k == 0 ? lam * eps : 2.0 * lam * eps));
      WZ_CUDA_TRY(c, Q(0.5 * eps));
      if ((rc = F(false))) return rc;
      WZ_CUDA_TRY(c, P((1.0 - 2.0 * lam) * eps));
      WZ_CUDA_TRY(c, Q(0.5 * eps));
      if ((rc = F(false))) return rc;
    }
    WZ_CUDA_TRY(c, P(lam * eps));
  }
  (void)so;
  return WZ_OK;
}

}  // namespace wz

using namespace wz;

extern "C" {

int wz_get_phi(wz_ctx* c, void* phi) {
  if (!c || !phi) return set_error(c, WZ_EINVAL, "wz_get_phi: null pointer");
  WZ_CUDA_TRY(c, cudaMemcpyAsync(phi, c->phi64, sizeof(cplx<double>) * c->V, cudaMemcpyDefault, c->stream));
  WZ_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return WZ_OK;
}

int wz_force(wz_ctx* c, const void* eta, int npf, double tol, unsigned parts, void* grad, double* S_B,
             double* S_pf, wz_solve_stats* stats) {
  if (!c) return WZ_EINVAL;
  if (!grad || npf < 0 || (npf > 0 && !eta) || tol <= 0.0) return set_error(c, WZ_EINVAL, "wz_force: bad argument");
  const auto t0 = std::chrono::steady_clock::now();
  ForceWS w;
  int rc = force_ws(c, npf > 0 ? npf : 1, &w);
  if (rc) return rc;
  const size_t f4 = sizeof(cplx<double>) * 4 * (size_t)c->V;
  const cplx<double>* e = (const cplx<double>*)eta;
  if (npf > 0 && !is_device_pointer(eta)) {
    WZ_CUDA_TRY(c, cudaMemcpyAsync(w.eta, eta, f4 * npf, cudaMemcpyHostToDevice, c->stream));
    e = w.eta;
  }
  ForceOpts o;
  o.tol = tol;
  o.fermion = (parts & 1) != 0 && npf > 0;
  o.boson = (parts & 2) != 0;
  SolveOut so;
  rc = force_eval(c, w, e, npf, o, w.sb1, &so);
  if (rc && rc != WZ_NOT_CONVERGED) return rc;
  WZ_CUDA_TRY(c, cudaMemcpyAsync(grad, w.G, sizeof(cplx<double>) * c->V, cudaMemcpyDefault, c->stream));
  double* pin = (double*)((char*)c->host_pinned + WZ_PINNED_SCRATCH_OFFSET);
  if (S_B) *S_B = o.boson ? host_sum(c, w.sb1, w.nb, pin) : 0.0;
  if (S_pf) {
    if (o.fermion) {
      ++g_launches;
      dot_re_partials<<<256, 256, 0, c->stream>>>(e, w.X, 4L * c->V * npf, w.spf1);
      WZ_CUDA_TRY(c, cudaGetLastError());
      *S_pf = host_sum(c, w.spf1, 256, pin);
    } else {
      *S_pf = 0.0;
    }
  }
  WZ_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (stats) {
    stats->iterations = so.iterations;
    stats->total_iterations = so.total_iterations;
    stats->reliable_updates = so.reliable_updates;
    stats->converged = so.converged;
    stats->max_true_residual = so.max_true_residual;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return rc;
}

int wz_md_integrate(wz_ctx* c, void* pi, const void* eta, int npf, const wz_hmc_params* h, wz_traj_stats* st) {
  if (!c) return WZ_EINVAL;
  if (!pi || !h || npf < 0 || (npf > 0 && !eta) || h->nsteps < 1 || h->tol <= 0.0)
    return set_error(c, WZ_EINVAL, "wz_md_integrate: bad argument");
  const auto t0 = std::chrono::steady_clock::now();
  ForceWS w;
  int rc = force_ws(c, npf > 0 ? npf : 1, &w);
  if (rc) return rc;
  const size_t f1 = sizeof(cplx<double>) * (size_t)c->V, f4 = 4 * f1;
  WZ_CUDA_TRY(c, cudaMemcpyAsync(w.pi, pi, f1, cudaMemcpyDefault, c->stream));
  if (npf > 0) WZ_CUDA_TRY(c, cudaMemcpyAsync(w.eta, eta, f4 * npf, cudaMemcpyDefault, c->stream));
  ForceOpts o;
  o.tol = h->tol;
  o.maxiter = h->maxiter > 0 ? h->maxiter : 100000;
  o.mixed = (h->flags & WZ_HMC_FP64_SOLVES) == 0;
  SolveOut acc;
  int nf = 0;
  rc = md_integrate(c, w, w.eta, npf, h->tau, h->nsteps, h->integrator, o, &acc, &nf, false);
  if (rc) return rc;
  WZ_CUDA_TRY(c, cudaMemcpyAsync(pi, w.pi, f1, cudaMemcpyDefault, c->stream));
  WZ_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (st) {
    memset(st, 0, sizeof(*st));
    st->force_evals = nf;
    st->cg_iterations = acc.total_iterations;
    st->reliable_updates = acc.reliable_updates;
    st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return WZ_OK;
}

int wz_trajectory(wz_ctx* c, const wz_hmc_params* h, wz_traj_stats* st) {
  if (!c) return WZ_EINVAL;
  if (!h || h->npf < 0 || h->nsteps < 1 || h->tol <= 0.0 || h->tau <= 0.0)
    return set_error(c, WZ_EINVAL, "wz_trajectory: bad argument");
  const auto t0 = std::chrono::steady_clock::now();
  const int npf = h->npf;
  ForceWS w;
  int rc = force_ws(c, npf > 0 ? npf : 1, &w);
  if (rc) return rc;
  cudaStream_t s = c->stream;
  const long V = c->V;
  const unsigned g = grid1d(V);
  // heatbath: pi ~ N(0,1), R ~ exp(-|R|^2), eta = M^dag R
  g_launches += 2;
  draw_momenta<<<g, 256, 0, s>>>(w.pi, V, h->seed, h->traj_index);
  WZ_CUDA_TRY(c, cudaGetLastError());
  if (npf > 0) {
    draw_sources<<<grid1d(4 * V * npf), 256, 0, s>>>(w.R, npf, V, h->seed, h->traj_index);
    WZ_CUDA_TRY(c, cudaGetLastError());
    WZ_CUDA_TRY(c, c->ws_apply.reserve(apply_ws_bytes<double>(c, WZ_OP_MDAG, npf)));
    rc = apply_op<double>(c, WZ_OP_MDAG, w.R, w.eta, npf, 0.0, (cplx<double>*)c->ws_apply.ptr);
    if (rc) return rc;
  }
  WZ_CUDA_TRY(c, cudaMemcpyAsync(w.phi0, c->phi64, sizeof(cplx<double>) * V, cudaMemcpyDeviceToDevice, s));
  g_launches += 2;
  dot_re_partials<<<256, 256, 0, s>>>(w.pi, w.pi, V, w.kin0);
  if (npf > 0) dot_re_partials<<<256, 256, 0, s>>>(w.R, w.R, 4L * V * npf, w.spf0);
  else WZ_CUDA_TRY(c, cudaMemsetAsync(w.spf0, 0, 256 * sizeof(double), s));
  WZ_CUDA_TRY(c, cudaGetLastError());
  ForceOpts o;
  o.tol = h->tol;
  o.maxiter = h->maxiter > 0 ? h->maxiter : 100000;
  o.mixed = (h->flags & WZ_HMC_FP64_SOLVES) == 0;
  SolveOut acc;
  int nf = 0;
  rc = md_integrate(c, w, w.eta, npf, h->tau, h->nsteps, h->integrator, o, &acc, &nf, true);
  if (rc) return rc;
  g_launches += 2;
  dot_re_partials<<<256, 256, 0, s>>>(w.pi, w.pi, V, w.kin1);
  if (npf > 0) dot_re_partials<<<256, 256, 0, s>>>(w.eta, w.X, 4L * V * npf, w.spf1);
  else WZ_CUDA_TRY(c, cudaMemsetAsync(w.spf1, 0, 256 * sizeof(double), s));
  HParts hp{w.kin0, 256, w.sb0, w.nb, w.spf0, 256, w.kin1, 256, w.sb1, w.nb, w.spf1, 256};
  g_launches += 2;
  metropolis<<<1, 32, 0, s>>>(hp, w.res, h->seed, h->traj_index);
  WZ_CUDA_TRY(c, cudaGetLastError());
  if (!(h->flags & WZ_HMC_NO_METROPOLIS)) {
    restore_phi<<<g, 256, 0, s>>>(c->phi64, c->phi32, w.phi0, w.res, V);
    WZ_CUDA_TRY(c, cudaGetLastError());
  }
  double* pin = (double*)((char*)c->host_pinned + WZ_PINNED_SCRATCH_OFFSET);
  WZ_CUDA_TRY(c, cudaMemcpyAsync(pin, w.res, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
  WZ_CUDA_TRY(c, cudaStreamSynchronize(s));
  if (st) {
    st->H0 = pin[0];
    st->H1 = pin[1];
    st->dH = pin[2];
    st->u = pin[3];
    st->accept = (h->flags & WZ_HMC_NO_METROPOLIS) ? 1 : (pin[4] != 0.0);
    st->force_evals = nf;
    st->cg_iterations = acc.total_iterations;
    st->reliable_updates = acc.reliable_updates;
    st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return WZ_OK;
}

}  // extern "C"
