// Forces, actions, molecular dynamics and HMC trajectories (host sequencing).
//
// force(phi):  X_k = (M^dag M)^-1 eta_k   (one batched CG over the npf pseudofermions)
//              G_k = site contraction of Z_k = M X_k with X_k         (xy_force)
//              G   = G_B(phi) + sum_k G_k, S_B partials                (xy_boson_inv)
// With a rational action (RHMC, Eq. jkjk) the solve holds d shifted systems
// per pseudofermion, X_ik = (M^dag M + beta_i)^-1 eta_k, laid out
// [member][pole][pseudofermion], and G_ik carries the weight alpha_i.
// The leapfrog / Omelyan integrators and the Metropolis step follow Sec. 7.2;
// the state (phi, pi) stays in FP64 on the device throughout.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "hmc.h"
#include "solver_impl.cuh"
#include "wz_hmc.cuh"

namespace wz {

static unsigned grid1d(long n) {
  long b = (n + 255) / 256;
  return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

// Workspace of the force / MD code (FP64), carved from ctx->ws_force.  Every
// field carries the member index outermost; npf pseudofermions per member.
struct ForceWS {
  cplx<double>* X;     // [nm][d][npf][V][4] solutions (d poles; 1 without a rational action)
  cplx<double>* A;     // [nm][d][npf][V][4] momentum intermediate
  cplx<double>* Gk;    // [nm][d][npf][V] per-system forces
  cplx<double>* Y;     // [nm][npf][V][4] r(M^dag M) eta (rational action)
  cplx<double>* Bk;    // [nm][V][4] packed scalar field / its transform
  cplx<double>* G;     // [nm][V] total force
  cplx<double>* pi;    // [nm][V] momenta
  cplx<double>* phi0;  // [nm][V] phi at the start of the trajectory
  cplx<double>* R;     // [nm][npf][V][4] heatbath sources
  cplx<double>* eta;   // [nm][npf][V][4] pseudofermions
  double* sb0;         // [nm][nb] S_B partials at the start
  double* sb1;         // [nm][nb] S_B partials of the latest force evaluation
  double* kin0;        // [nm][ND] |pi|^2 partials at the start
  double* kin1;
  double* spf0;        // [nm][ND] |R|^2 partials
  double* spf1;        // [nm][ND] Re eta^dag X partials
  double* res;         // [nm][5] metropolis results [H0, H1, dH, u, accept]
  int nb;              // xy blocks for one field
};

static const int ND = 128;  // blocks of the dot-product partials per member

// npf pseudofermions; ds solutions per pseudofermion held at once (the larger
// of the action's and the heatbath's pole counts), df of them in the force.
static int force_ws(wz_ctx* c, int npf, ForceWS* w, int ds = 1, int df = 1) {
  const long nm = c->nm;
  const size_t f4 = sizeof(cplx<double>) * 4 * (size_t)c->V;
  const size_t f1 = sizeof(cplx<double>) * (size_t)c->V;
  w->nb = xy_nblk(c->X, c->T * c->Z);
  const size_t npart = (size_t)nm * (w->nb > ND ? w->nb : ND);
  size_t off = 0;
  auto take = [&](size_t n) {
    size_t r = off;
    off += (n + 255) & ~size_t(255);
    return r;
  };
  const size_t oX = take(f4 * npf * nm * ds), oA = take(f4 * npf * nm * df), oGk = take(f1 * npf * nm * df),
               oY = take(f4 * npf * nm), oB = take(f4 * nm),
               oG = take(f1 * nm), oPi = take(f1 * nm), oP0 = take(f1 * nm), oR = take(f4 * npf * nm),
               oE = take(f4 * npf * nm), oParts = take(sizeof(double) * (6 * npart + 5 * nm + 8));
  WZ_CUDA_TRY(c, c->ws_force.reserve(off));
  char* b = (char*)c->ws_force.ptr;
  w->X = (cplx<double>*)(b + oX);
  w->A = (cplx<double>*)(b + oA);
  w->Gk = (cplx<double>*)(b + oGk);
  w->Y = (cplx<double>*)(b + oY);
  w->Bk = (cplx<double>*)(b + oB);
  w->G = (cplx<double>*)(b + oG);
  w->pi = (cplx<double>*)(b + oPi);
  w->phi0 = (cplx<double>*)(b + oP0);
  w->R = (cplx<double>*)(b + oR);
  w->eta = (cplx<double>*)(b + oE);
  double* p = (double*)(b + oParts);
  w->sb0 = p;
  w->sb1 = p + npart;
  w->kin0 = p + 2 * npart;
  w->kin1 = p + 3 * npart;
  w->spf0 = p + 4 * npart;
  w->spf1 = p + 5 * npart;
  w->res = p + 6 * npart;
  return WZ_OK;
}

// A rational function on the device: pole shifts for the solver, residues for
// the force weights and the combination; inner = pseudofermions per member.
struct RatPoles {
  ShiftSpec sh;
  PoleSum ps;
};

static RatPoles make_poles(const wz_rational* r, int inner) {
  RatPoles q;
  q.sh.d = q.ps.d = r->d;
  q.sh.inner = q.ps.inner = inner;
  q.ps.a0 = r->a0;
  for (int i = 0; i < r->d; ++i) {
    q.sh.beta[i] = r->beta[i];
    q.ps.alpha[i] = r->alpha[i];
  }
  return q;
}

struct ForceOpts {
  const RatPoles* ra = nullptr;  // rational action (null: single pole, beta = 0)
  double tol = 1e-10;
  int maxiter = 100000;
  bool mixed = true;
  bool fermion = true;
  bool boson = true;
  bool inline_capture = false;  // solves become conditional nodes of an ongoing capture
};

// G = dS/dphi for the current phi of every member; S_B partials into
// sb_part ([nm][nb]).  On return X holds (M^dag M)^-1 eta.
static int force_eval(wz_ctx* c, const ForceWS& w, const cplx<double>* eta, int npf, const ForceOpts& o,
                      double* sb_part, SolveOut* so) {
  cudaStream_t s = c->stream;
  const int L = c->X;
  const int TZ = c->T * c->Z;
  const int nm = c->nm;
  cudaError_t e;
  int npf_eff = o.fermion ? npf : 0;
  const int dpol = o.ra ? o.ra->ps.d : 1;  // systems per pseudofermion
  if (npf_eff > 0) {
    const int nr = nm * npf * dpol;  // right-hand sides of the batched solve
    const ShiftSpec sh = o.ra ? o.ra->sh : single_shift(0.0);
    int rc = o.mixed ? solve_impl<float>(c, eta, w.X, nr, sh, o.tol, o.maxiter, false, 0.1, so, o.inline_capture)
                     : solve_impl<double>(c, eta, w.X, nr, sh, o.tol, o.maxiter, false, 0.0, so, o.inline_capture);
    if (rc) return rc;
    // Z = M X without the site term: forward xy, +Dslash; the site term and the
    // contraction are fused into xy_force
    XYArgs<double> xa = xy_args<double>(c, nr);
    xa.psi = w.X;
    xa.A_out = w.A;
    e = launch_xy<double>(L, XY_FWD, xa, s);
    if (e != cudaSuccess) return cuda_error(c, e, "force: xy forward");
    ZTArgs<double> za = zt_args<double>(c, 1.0);
    za.A = w.A;
    e = launch_zt<double>(c->Z, c->T, ZT_DSLASH, za, nr, s);
    if (e != cudaSuccess) return cuda_error(c, e, "force: zt");
    ForceArgs<double> fa{};
    fa.A = w.A;
    fa.X = w.X;
    fa.Gk = w.Gk;
    fa.phi = c->phi64;
    fa.kArr = c->k64;
    fa.rpm = npf * dpol;
    if (o.ra) fa.pw = o.ra->ps;
    fa.Z = c->Z;
    fa.twc = c->t64.twc;
    fa.tws = c->t64.tws;
    fa.TZ = TZ;
    fa.V = c->V;
    e = launch_fk(L, FK_FORCE, fa, dim3(w.nb, nr), s);
    if (e != cudaSuccess) return cuda_error(c, e, "force: xy_force");
  }
  // bosonic part (+ the sum of the fermion forces of each member)
  ForceArgs<double> ba{};
  ba.phi = c->phi64;
  ba.kArr = c->k64;
  ba.rpm = 1;
  ba.TZ = TZ;
  ba.V = c->V;
  ba.nblk = w.nb;
  ba.A_out = w.Bk;
  ba.A = w.Bk;
  ba.Gk_in = w.Gk;
  ba.npf = npf_eff * dpol;
  ba.G = w.G;
  ba.part = sb_part;
  if (o.boson) {
    e = launch_fk(L, FK_BOSON_FWD, ba, dim3(w.nb, nm), s);
    if (e != cudaSuccess) return cuda_error(c, e, "force: boson forward");
    ZTArgs<double> za = zt_args<double>(c, 1.0);
    za.A = w.Bk;
    e = launch_zt<double>(c->Z, c->T, ZT_SCALAR, za, nm, s);
    if (e != cudaSuccess) return cuda_error(c, e, "force: boson zt");
  } else {
    // zero scalar transform: the inverse pass then only sums the fermion forces
    e = cudaMemsetAsync(w.Bk, 0, sizeof(cplx<double>) * 4 * c->V * nm, s);
    if (e != cudaSuccess) return cuda_error(c, e, "force: memset");
  }
  e = launch_fk(L, FK_BOSON_INV, ba, dim3(w.nb, nm), s);
  if (e != cudaSuccess) return cuda_error(c, e, "force: boson inverse");
  return WZ_OK;
}

// partials [nm][ND] of the pseudofermion action from the solutions in w.X:
// Re eta^dag X (single pole) or Re eta^dag (a0 eta + sum_i alpha_i X_i).
static int pf_action_partials(wz_ctx* c, const ForceWS& w, const cplx<double>* eta, int npf, const RatPoles* ra,
                              double* part) {
  const long n4 = 4L * c->V;
  const cplx<double>* y = w.X;
  if (ra) {
    count_launch();
    pole_combine<<<dim3(64, c->nm * npf), 256, 0, c->stream>>>(eta, w.X, w.Y, n4, ra->ps);
    WZ_CUDA_TRY(c, cudaGetLastError());
    y = w.Y;
  }
  count_launch();
  dot_re_partials<<<dim3(ND, c->nm), 256, 0, c->stream>>>(eta, y, n4 * npf, part);
  WZ_CUDA_TRY(c, cudaGetLastError());
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
// spf_first (may be null): pseudofermion-action partials from the first force
// evaluation (the action at the starting phi).
static int md_integrate(wz_ctx* c, ForceWS& w, const cplx<double>* eta, int npf, double tau, int nsteps,
                        int integrator, const ForceOpts& o, SolveOut* acc, int* nforce, bool first_into_sb0,
                        double* spf_first = nullptr) {
  cudaStream_t s = c->stream;
  const long V = c->V * c->nm;  // all members' fields update together
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
    if (!r && first && spf_first && npf > 0) r = pf_action_partials(c, w, eta, npf, o.ra, spf_first);
    return r;
  };
  auto P = [&](double h) {
    count_launch();
    update_pi<<<g, 256, 0, s>>>(w.pi, w.G, h, V);
    return cudaGetLastError();
  };
  auto Q = [&](double h) {
    count_launch();
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

// sum of the per-member partial slices [nm][n] -> out[nm] (synchronises)
static int host_member_sums(wz_ctx* c, const double* dev, int n, std::vector<double>& out) {
  const int nm = c->nm;
  double* pin = (double*)((char*)c->host_pinned + WZ_PINNED_SCRATCH_OFFSET);
  if (sizeof(double) * (size_t)n * nm > WZ_PINNED_BYTES - WZ_PINNED_SCRATCH_OFFSET)
    return set_error(c, WZ_EINVAL, "too many members for the pinned read-back");
  WZ_CUDA_TRY(c, cudaMemcpyAsync(pin, dev, sizeof(double) * n * nm, cudaMemcpyDeviceToHost, c->stream));
  WZ_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  out.assign(nm, 0.0);
  for (int j = 0; j < nm; ++j)
    for (int i = 0; i < n; ++i) out[j] += pin[(long)j * n + i];
  return WZ_OK;
}

// Forces and actions of every member.  eta: [nm][npf] fields (device).
int force_impl(wz_ctx* c, const cplx<double>* eta, int npf, double tol, unsigned parts, cplx<double>* grad,
               double* S_B, double* S_pf, SolveOut* so, const wz_rational* ra) {
  ForceWS w;
  const int dpol = ra ? ra->d : 1;
  int rc = force_ws(c, npf > 0 ? npf : 1, &w, dpol, dpol);
  if (rc) return rc;
  RatPoles rp;
  ForceOpts o;
  if (ra) {
    rp = make_poles(ra, npf);
    o.ra = &rp;
  }
  o.tol = tol;
  o.fermion = (parts & 1) != 0 && npf > 0;
  o.boson = (parts & 2) != 0;
  rc = force_eval(c, w, eta, npf, o, w.sb1, so);
  if (rc && rc != WZ_NOT_CONVERGED) return rc;
  WZ_CUDA_TRY(c, cudaMemcpyAsync(grad, w.G, sizeof(cplx<double>) * c->V * c->nm, cudaMemcpyDefault, c->stream));
  std::vector<double> v;
  if (S_B) {
    if (o.boson) {
      int r2 = host_member_sums(c, w.sb1, w.nb, v);
      if (r2) return r2;
      for (int j = 0; j < c->nm; ++j) S_B[j] = v[j];
    } else {
      for (int j = 0; j < c->nm; ++j) S_B[j] = 0.0;
    }
  }
  if (S_pf) {
    if (o.fermion) {
      int r2 = pf_action_partials(c, w, eta, npf, o.ra, w.spf1);
      if (r2) return r2;
      r2 = host_member_sums(c, w.spf1, ND, v);
      if (r2) return r2;
      for (int j = 0; j < c->nm; ++j) S_pf[j] = v[j];
    } else {
      for (int j = 0; j < c->nm; ++j) S_pf[j] = 0.0;
    }
  }
  WZ_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return rc;
}

// Enqueue one trajectory of every member (Sec. 7.2) on c->stream without any
// host interaction in graph mode; the trajectory number is read on the device
// from c->counters[3].  nf: force evaluations.
// rh: heatbath rational function (RHMC; with o.ra) or null (eta = M^dag R).
// body_h (may be null): kernels per trip of the captured heatbath solver loop.
static int enqueue_trajectory(wz_ctx* c, ForceWS& w, const wz_hmc_params* h, const ForceOpts& o, SolveOut* acc,
                              int* nf, const RatPoles* rh = nullptr, unsigned long long* body_h = nullptr) {
  const int npf = h->npf;
  const int nm = c->nm;
  cudaStream_t s = c->stream;
  const long V = c->V, VN = c->V * nm;
  const unsigned g = grid1d(VN);
  const unsigned long long* trajp = c->counters + 3;
  int rc;
  // heatbath: pi ~ N(0,1), R ~ exp(-|R|^2), eta = M^dag R (one pole) or
  // eta = r_h(M^dag M) R (RHMC, Eq. hbeq)
  count_launch();
  draw_momenta<<<g, 256, 0, s>>>(w.pi, V, nm, c->mid, h->seed, trajp);
  WZ_CUDA_TRY(c, cudaGetLastError());
  if (npf > 0) {
    count_launch();
    draw_sources<<<grid1d(4 * VN * npf), 256, 0, s>>>(w.R, npf, V, nm, c->mid, h->seed, trajp);
    WZ_CUDA_TRY(c, cudaGetLastError());
    if (rh) {
      SolveOut one;
      c->trip_slot = 4;
      rc = o.mixed ? solve_impl<float>(c, w.R, w.X, nm * npf * rh->sh.d, rh->sh, o.tol, o.maxiter, false, 0.1, &one,
                                       o.inline_capture)
                   : solve_impl<double>(c, w.R, w.X, nm * npf * rh->sh.d, rh->sh, o.tol, o.maxiter, false, 0.0, &one,
                                        o.inline_capture);
      c->trip_slot = 2;
      if (body_h) *body_h = c->inline_body_launches;
      add_solve(*acc, one);
      if (rc == WZ_NOT_CONVERGED) return set_error(c, rc, "heatbath: solver did not converge");
      if (rc) return rc;
      count_launch();
      pole_combine<<<dim3(64, nm * npf), 256, 0, s>>>(w.R, w.X, w.eta, 4L * V, rh->ps);
      WZ_CUDA_TRY(c, cudaGetLastError());
    } else {
      rc = apply_op<double>(c, WZ_OP_MDAG, w.R, w.eta, npf * nm, 0.0, (cplx<double>*)c->ws_apply.ptr);
      if (rc) return rc;
    }
  }
  WZ_CUDA_TRY(c, cudaMemcpyAsync(w.phi0, c->phi64, sizeof(cplx<double>) * VN, cudaMemcpyDeviceToDevice, s));
  count_launch();
  dot_re_partials<<<dim3(ND, nm), 256, 0, s>>>(w.pi, w.pi, V, w.kin0);
  if (npf > 0 && !o.ra) {  // eta^dag (M^dag M)^-1 eta = |R|^2 exactly
    count_launch();
    dot_re_partials<<<dim3(ND, nm), 256, 0, s>>>(w.R, w.R, 4L * V * npf, w.spf0);
  } else if (npf == 0) {
    WZ_CUDA_TRY(c, cudaMemsetAsync(w.spf0, 0, ND * nm * sizeof(double), s));
  }
  WZ_CUDA_TRY(c, cudaGetLastError());
  // RHMC: S_pf at the start from the solves of the first force evaluation
  rc = md_integrate(c, w, w.eta, npf, h->tau, h->nsteps, h->integrator, o, acc, nf, true,
                    (npf > 0 && o.ra) ? w.spf0 : nullptr);
  if (rc) return rc;
  count_launch();
  dot_re_partials<<<dim3(ND, nm), 256, 0, s>>>(w.pi, w.pi, V, w.kin1);
  if (npf > 0) {
    rc = pf_action_partials(c, w, w.eta, npf, o.ra, w.spf1);
    if (rc) return rc;
  } else {
    WZ_CUDA_TRY(c, cudaMemsetAsync(w.spf1, 0, ND * nm * sizeof(double), s));
  }
  HParts hp{w.kin0, ND, w.sb0, w.nb, w.spf0, ND, w.kin1, ND, w.sb1, w.nb, w.spf1, ND};
  count_launch(2);
  metropolis<<<(nm + 31) / 32, 32, 0, s>>>(hp, w.res, nm, c->mid, h->seed, trajp);
  WZ_CUDA_TRY(c, cudaGetLastError());
  if (!(h->flags & WZ_HMC_NO_METROPOLIS)) {
    restore_phi<<<g, 256, 0, s>>>(c->phi64, c->phi32, w.phi0, w.res, V, nm);
    WZ_CUDA_TRY(c, cudaGetLastError());
  }
  return WZ_OK;
}

// One trajectory of every member; st: nm entries (may be null).  In graph mode
// the whole trajectory -- draws, heatbath, every force evaluation with its
// solver loop as a WHILE conditional node, the updates, H and the Metropolis
// decisions -- is one CUDA graph, captured once per parameter set and then
// replayed (the trajectory number is written to the device before a replay).
// FNV-1a over the coefficients of the rational action and heatbath (graph key)
static unsigned long long rational_hash(const wz_rational* ra, const wz_rational* rh) {
  unsigned long long hsh = 1469598103934665603ULL;
  auto mix = [&](const void* p, size_t n) {
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) hsh = (hsh ^ b[i]) * 1099511628211ULL;
  };
  for (const wz_rational* r : {ra, rh}) {
    if (!r) {
      mix("-", 1);
      continue;
    }
    mix(&r->d, sizeof(r->d));
    mix(&r->a0, sizeof(r->a0));
    mix(r->alpha, sizeof(double) * r->d);
    mix(r->beta, sizeof(double) * r->d);
  }
  return hsh;
}

// ra, rh: rational action and heatbath (RHMC), both or neither.
int trajectory_impl(wz_ctx* c, const wz_hmc_params* h, wz_traj_stats* st, const wz_rational* ra,
                    const wz_rational* rh) {
  const auto t0 = std::chrono::steady_clock::now();
  const int npf = h->npf;
  const int nm = c->nm;
  const int da = ra ? ra->d : 1, dh = rh ? rh->d : 1;
  ForceWS w;
  int rc = force_ws(c, npf > 0 ? npf : 1, &w, da > dh ? da : dh, da);
  if (rc) return rc;
  if (npf > 0 && !rh) WZ_CUDA_TRY(c, c->ws_apply.reserve(apply_ws_bytes<double>(c, WZ_OP_MDAG, npf * nm)));
  RatPoles rpa, rph;
  ForceOpts o;
  if (ra) {
    rpa = make_poles(ra, npf);
    rph = make_poles(rh, npf);
    o.ra = &rpa;
  }
  o.tol = h->tol;
  o.maxiter = h->maxiter > 0 ? h->maxiter : 100000;
  o.mixed = (h->flags & WZ_HMC_FP64_SOLVES) == 0;
  SolveOut acc;
  int nf = 0;
  cudaStream_t s = c->stream;
  unsigned long long* hc = (unsigned long long*)((char*)c->host_pinned + WZ_PINNED_SCRATCH_OFFSET);
  if (sizeof(double) * 5 * nm + 64 > WZ_PINNED_BYTES - WZ_PINNED_SCRATCH_OFFSET)
    return set_error(c, WZ_EINVAL, "too many members");
  double* hres = (double*)(hc + WZ_NCOUNTERS);
  // device state of this trajectory: counters zero, trajectory number
  for (int i = 0; i < WZ_NCOUNTERS; ++i) hc[i] = 0;
  hc[3] = h->traj_index;
  WZ_CUDA_TRY(c, cudaMemcpyAsync(c->counters, hc, WZ_NCOUNTERS * sizeof(unsigned long long), cudaMemcpyHostToDevice, s));
  const bool graph = c->use_graphs && !g_probe.active;
  if (graph) {
    // reserve the solver workspace now: nothing may allocate during the capture
    {
      const int nblk = xy_nblk(c->X, c->T * c->Z);
      const int nsys = nm * (npf > 0 ? npf : 1) * (da > dh ? da : dh);
      SolverWS<float> W1(c->V, nsys, nblk, false);
      SolverWS<double> W2(c->V, nsys, nblk, false);
      WZ_CUDA_TRY(c, c->ws_solver.reserve(o.mixed ? W1.total : W2.total));
    }
    TrajGraphKey key{};
    key.tau = h->tau;
    key.tol = h->tol;
    key.nsteps = h->nsteps;
    key.integrator = h->integrator;
    key.npf = npf;
    key.maxiter = o.maxiter;
    key.flags = h->flags;
    key.seed = h->seed;
    key.rational = rational_hash(ra, rh);
    key.ws_force = c->ws_force.ptr;
    key.ws_solver = c->ws_solver.ptr;
    key.ws_apply = c->ws_apply.ptr;
    key.b_force = c->ws_force.bytes;
    key.b_solver = c->ws_solver.bytes;
    key.b_apply = c->ws_apply.bytes;
    TrajGraph& T = c->traj_graph;
    // a capture that fails with the solvers' dependent launches is repeated
    // once with plain launches (and the context keeps to them)
    for (int attempt = 0; attempt < 2 && (!T.exec || memcmp(&key, &T.key, sizeof(key)) != 0); ++attempt) {
      T.release();
      WZ_CUDA_TRY(c, cudaStreamSynchronize(s));
      const unsigned long long l0 = tl_launches;
      cudaStream_t saved = c->stream;
      c->stream = c->cap_stream;
      ForceOpts oc = o;
      oc.inline_capture = true;
      cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed);
      unsigned long long body_h = 0;
      int rc2 = e == cudaSuccess ? enqueue_trajectory(c, w, h, oc, &acc, &nf, ra ? &rph : nullptr, &body_h)
                                 : WZ_ECUDA;
      cudaGraph_t gr = nullptr;
      cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &gr);
      c->stream = saved;
      T.outer_launches = tl_launches - l0;
      T.body_launches = c->inline_body_launches;
      T.body_launches_h = body_h;
      g_launches -= T.outer_launches;
      tl_launches = l0;
      if (e != cudaSuccess) return cuda_error(c, e, "trajectory capture");
      cudaError_t ei = cudaErrorUnknown;
      if (!rc2 && ee == cudaSuccess) {
        T.graph = gr;
        gr = nullptr;
        ei = cudaGraphInstantiate(&T.exec, T.graph, 0);
        if (ei == cudaSuccess) {
          T.force_evals = nf;
          T.key = key;
          break;
        }
      }
      if (gr) cudaGraphDestroy(gr);
      if (attempt == 0 && !c->pdl_capture_failed) {
        cudaGetLastError();
        T.release();
        c->pdl_capture_failed = true;
        c->err.clear();
        continue;
      }
      if (rc2) return rc2;
      if (ee != cudaSuccess) return cuda_error(c, ee, "trajectory cudaStreamEndCapture");
      return cuda_error(c, ei, "cudaGraphInstantiate (trajectory)");
    }
    WZ_CUDA_TRY(c, cudaGraphLaunch(T.exec, s));
    nf = T.force_evals;
  } else {
    rc = enqueue_trajectory(c, w, h, o, &acc, &nf, ra ? &rph : nullptr);
    if (rc) return rc;
  }
  WZ_CUDA_TRY(c, cudaMemcpyAsync(hres, w.res, 5 * nm * sizeof(double), cudaMemcpyDeviceToHost, s));
  WZ_CUDA_TRY(c, cudaMemcpyAsync(hc, c->counters, WZ_NCOUNTERS * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  WZ_CUDA_TRY(c, cudaStreamSynchronize(s));
  if (graph)
    count_launch(c->traj_graph.outer_launches + hc[2] * c->traj_graph.body_launches +
                 hc[4] * c->traj_graph.body_launches_h);
  if (hc[WZ_COUNTER_DEVICE_ERROR])
    return set_error(c, (int)(hc[WZ_COUNTER_DEVICE_ERROR] & 0xffffffffu), "trajectory: a device-side staged copy failed");
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int j = 0; st && j < nm; ++j) {
    st[j].H0 = hres[5 * j + 0];
    st[j].H1 = hres[5 * j + 1];
    st[j].dH = hres[5 * j + 2];
    st[j].u = hres[5 * j + 3];
    st[j].accept = (h->flags & WZ_HMC_NO_METROPOLIS) ? 1 : (hres[5 * j + 4] != 0.0);
    st[j].force_evals = nf;
    st[j].cg_iterations = (long long)hc[0];  // all members together
    st[j].reliable_updates = (int)hc[1];
    st[j].seconds = secs;
  }
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
  if (c->nm != 1) return set_error(c, WZ_EINVAL, "wz_force: single-lattice context expected");
  const auto t0 = std::chrono::steady_clock::now();
  const size_t f4 = sizeof(cplx<double>) * 4 * (size_t)c->V;
  const cplx<double>* e = (const cplx<double>*)eta;
  if (npf > 0 && !is_device_pointer(eta)) {
    WZ_CUDA_TRY(c, c->ws_stage.reserve(f4 * npf));
    WZ_CUDA_TRY(c, cudaMemcpyAsync(c->ws_stage.ptr, eta, f4 * npf, cudaMemcpyHostToDevice, c->stream));
    e = (const cplx<double>*)c->ws_stage.ptr;
  }
  SolveOut so;
  int rc = force_impl(c, e, npf, tol, parts, (cplx<double>*)grad, S_B, S_pf, &so);
  if (rc && rc != WZ_NOT_CONVERGED) return rc;
  if (stats) {
    stats->iterations = so.iterations;
    stats->total_iterations = so.total_iterations;
    stats->reliable_updates = so.reliable_updates;
    stats->converged = so.converged;
    stats->max_true_residual = so.max_true_residual;
    stats->site_applies = (double)(so.total_iterations + so.reliable_updates) * (double)c->V;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return rc;
}

int wz_md_integrate(wz_ctx* c, void* pi, const void* eta, int npf, const wz_hmc_params* h, wz_traj_stats* st) {
  if (!c) return WZ_EINVAL;
  if (!pi || !h || npf < 0 || (npf > 0 && !eta) || h->nsteps < 1 || h->tol <= 0.0)
    return set_error(c, WZ_EINVAL, "wz_md_integrate: bad argument");
  if (c->nm != 1) return set_error(c, WZ_EINVAL, "wz_md_integrate: single-lattice context expected");
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

int wz_action(wz_ctx* c, const void* eta, int npf, double tol, double* S_B, double* S_pf, wz_solve_stats* stats) {
  if (!c) return WZ_EINVAL;
  if (npf < 0 || (npf > 0 && !eta) || tol <= 0.0 || (!S_B && !S_pf))
    return set_error(c, WZ_EINVAL, "wz_action: bad argument");
  if (c->nm != 1) return set_error(c, WZ_EINVAL, "wz_action: single-lattice context expected");
  const auto t0 = std::chrono::steady_clock::now();
  const size_t f4 = sizeof(cplx<double>) * 4 * (size_t)c->V, f1 = f4 / 4;
  WZ_CUDA_TRY(c, c->ws_stage.reserve(f4 * npf + f1));
  char* stage = (char*)c->ws_stage.ptr;
  const cplx<double>* e = (const cplx<double>*)eta;
  if (npf > 0 && !is_device_pointer(eta)) {
    WZ_CUDA_TRY(c, cudaMemcpyAsync(stage, eta, f4 * npf, cudaMemcpyHostToDevice, c->stream));
    e = (const cplx<double>*)stage;
  }
  cplx<double>* grad = (cplx<double>*)(stage + f4 * npf);  // the gradient is computed and dropped
  const unsigned parts = (S_pf && npf > 0 ? WZ_FORCE_FERMION : 0u) | (S_B ? WZ_FORCE_BOSON : 0u);
  SolveOut so;
  int rc = force_impl(c, e, npf, tol, parts, grad, S_B, S_pf, &so);
  if (rc && rc != WZ_NOT_CONVERGED) return rc;
  if (S_pf && npf == 0) *S_pf = 0.0;
  if (stats) {
    stats->iterations = so.iterations;
    stats->total_iterations = so.total_iterations;
    stats->reliable_updates = so.reliable_updates;
    stats->converged = so.converged;
    stats->max_true_residual = so.max_true_residual;
    stats->site_applies = (double)(so.total_iterations + so.reliable_updates) * (double)c->V;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return rc;
}

static bool rational_ok(const wz_rational* r) {
  if (!r || r->d < 1 || r->d > WZ_RATIONAL_MAX) return false;
  for (int i = 0; i < r->d; ++i)
    if (!(r->beta[i] >= 0.0) || !std::isfinite(r->alpha[i])) return false;
  return std::isfinite(r->a0);
}

int wz_rhmc_force(wz_ctx* c, const void* eta, int npf, const wz_rational* action, double tol, unsigned parts,
                  void* grad, double* S_B, double* S_pf, wz_solve_stats* stats) {
  if (!c) return WZ_EINVAL;
  if (!grad || npf < 0 || (npf > 0 && !eta) || tol <= 0.0 || !rational_ok(action))
    return set_error(c, WZ_EINVAL, "wz_rhmc_force: bad argument");
  if (c->nm != 1) return set_error(c, WZ_EINVAL, "wz_rhmc_force: single-lattice context expected");
  const auto t0 = std::chrono::steady_clock::now();
  const size_t f4 = sizeof(cplx<double>) * 4 * (size_t)c->V;
  const cplx<double>* e = (const cplx<double>*)eta;
  if (npf > 0 && !is_device_pointer(eta)) {
    WZ_CUDA_TRY(c, c->ws_stage.reserve(f4 * npf));
    WZ_CUDA_TRY(c, cudaMemcpyAsync(c->ws_stage.ptr, eta, f4 * npf, cudaMemcpyHostToDevice, c->stream));
    e = (const cplx<double>*)c->ws_stage.ptr;
  }
  SolveOut so;
  int rc = force_impl(c, e, npf, tol, parts, (cplx<double>*)grad, S_B, S_pf, &so, action);
  if (rc && rc != WZ_NOT_CONVERGED) return rc;
  if (stats) {
    stats->iterations = so.iterations;
    stats->total_iterations = so.total_iterations;
    stats->reliable_updates = so.reliable_updates;
    stats->converged = so.converged;
    stats->max_true_residual = so.max_true_residual;
    stats->site_applies = (double)(so.total_iterations + so.reliable_updates) * (double)c->V;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return rc;
}

int wz_rhmc_trajectory(wz_ctx* c, const wz_hmc_params* h, const wz_rational* action, const wz_rational* heatbath,
                       wz_traj_stats* st) {
  if (!c) return WZ_EINVAL;
  if (!h || h->npf < 1 || h->nsteps < 1 || h->tol <= 0.0 || h->tau <= 0.0 || !rational_ok(action) ||
      !rational_ok(heatbath))
    return set_error(c, WZ_EINVAL, "wz_rhmc_trajectory: bad argument");
  if (c->nm != 1) return set_error(c, WZ_EINVAL, "wz_rhmc_trajectory: single-lattice context expected");
  return trajectory_impl(c, h, st, action, heatbath);
}

int wz_trajectory(wz_ctx* c, const wz_hmc_params* h, wz_traj_stats* st) {
  if (!c) return WZ_EINVAL;
  if (!h || h->npf < 0 || h->nsteps < 1 || h->tol <= 0.0 || h->tau <= 0.0)
    return set_error(c, WZ_EINVAL, "wz_trajectory: bad argument");
  if (c->nm != 1) return set_error(c, WZ_EINVAL, "wz_trajectory: single-lattice context expected");
  return trajectory_impl(c, h, st);
}

}  // extern "C"
