/*
 * wz.h - C ABI of the GB300 lattice Wess-Zumino fermion-matrix library.
 *
 * The library applies the fermion matrix of the lattice Wess-Zumino model with
 * Ginsparg-Wilson (overlap) fermions (Chen, Dzienkowski, Giedt):
 *
 *   M = Dslash + (m + c g phi) P_+ + (m^* + c g^* phi^*) P_-,
 *   Dslash = (1 - a D2/2)^-1 D1                                   (Eq. fmat)
 *
 * through a 4D lattice FFT (the "FFT trick" of Sec. 7.2), and uses it in
 * conjugate-gradient solves of M^dagger M x = b (Eq. theprob), optionally
 * preconditioned by the free operator M0^-1 (Sec. 7.3), in the pseudofermion
 * force and in hybrid Monte Carlo trajectories (Sec. 7.2).
 *
 * Conventions shared by every call
 * --------------------------------
 * - a = 1.  dims = {T, Z, Y, X}; T even (antiperiodic fermion time, Sec. 3.1);
 *   X == Y in {4, 6, 8, 12, 16, 32} (wz_supported_extent); (Z, T) one of the
 *   compiled pairs (4, 4), (6, 6), (8, 8), (12, 12), (16, 16), (32, 32),
 *   (8, 16), (16, 32), (8, 32) and (32, 64), the last the paper's 32^3 x 64.
 * - Spinor field: complex, interleaved (re, im), layout [nrhs][T][Z][Y][X][4],
 *   spin index fastest.  WZ_C64 = complex64 (2 x float), WZ_C128 = complex128.
 * - Scalar field phi: complex128 [T][Z][Y][X], periodic in every direction.
 * - Force / gradient: complex128 [T][Z][Y][X] holding (dS/dphi_R, dS/dphi_I).
 * - Chiral basis of Sec. 2.1: gamma_5 = diag(-1,-1,1,1), P_- = spins 0,1,
 *   P_+ = spins 2,3; direction mu = 0 is time, mu = 1, 2, 3 are x, y, z.
 * - Fourier convention f(p) = sum_x exp(-i p.x) f(x); p_t = pi (2n+1)/T.
 *
 * Ownership: all field pointers belong to the caller.  Device pointers are used
 * in place, asynchronously on the context stream.  Host pointers (pageable or
 * pinned) are accepted by wz_set_phi, wz_apply, wz_solve, wz_force and
 * wz_action: the call stages them through context-owned device buffers and
 * returns after the results are back in host memory.  The context owns its
 * tables, workspace and RNG state; it is not thread-safe.
 *
 * Launching: a solve replays a CUDA graph of its iteration loop (a WHILE
 * conditional node driven by the device-side convergence state), cached on
 * the context per solve shape; setting WZ_NO_GRAPHS=1 in the environment
 * before wz_create makes the context launch the same kernels eagerly.  The
 * first solve of a shape (process-wide) times candidate launch configurations
 * on the real problem and keeps the fastest: right-hand sides per group,
 * concurrent streams, programmatic dependent launch of the iteration kernels
 * and the zt passes' tiles per block.  WZ_RHS_GROUP / WZ_RHS_BRANCHES,
 * WZ_PDL (0 or 1) and WZ_ZT_TPB fix them instead; none of them changes the
 * arithmetic (the solutions are bitwise equal).
 *
 * Errors: every call returns a WZ_* status; nothing throws across the ABI.
 * wz_last_error returns a message for the most recent failure of that context.
 */
#ifndef WZ_H
#define WZ_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum wz_status {
  WZ_OK = 0,
  WZ_EINVAL = 1,          /* bad argument: null pointer, odd T, unsupported extent, ... */
  WZ_ENOMEM = 2,          /* device allocation failed */
  WZ_ECUDA = 3,           /* CUDA runtime error (message in wz_last_error) */
  WZ_NOT_CONVERGED = 4,   /* solver hit maxiter; x holds the best iterate, stats filled */
  WZ_EUNSUPPORTED = 5,    /* combination not built (e.g. an extent without kernels) */
  WZ_ETIMEOUT = 6,        /* a bounded device-side wait (staged copy) ran out; outputs undefined */
  WZ_ENONFINITE = 7       /* a solver norm became NaN or Inf (non-finite phi, b or couplings); x undefined */
};

enum wz_dtype { WZ_C64 = 0, WZ_C128 = 1 };

enum wz_op {
  WZ_OP_M = 0,            /* M psi                                     (Eq. fmat) */
  WZ_OP_MDAG = 1,         /* M^dagger psi = -Dslash psi + Y^dagger psi             */
  WZ_OP_MDAGM = 2,        /* (M^dagger M + shift) psi                  (Eq. yuier) */
  WZ_OP_DSLASH = 3,       /* Dslash psi                        (Sec. 3.2 probe) */
  WZ_OP_M0INV = 4,        /* M0^-1 psi, M0^-1 = M0^dagger/(D^dagger D + |m|^2) (Sec. 7.3) */
  WZ_OP_M0INV_DAG = 5,    /* (M0^-1)^dagger psi                                   */
  WZ_OP_MTILDE = 6,       /* M~ psi = M M0^-1 psi                   (Eq. theprob) */
  WZ_OP_MTILDE_DAG = 7,   /* M~^dagger psi                                        */
  WZ_OP_MTILDE_DAGM = 8,  /* (M~^dagger M~ + shift) psi                           */
  WZ_OP_D1 = 9,           /* D1 psi: gamma-odd part of the overlap, i gamma.sin p / omega
                             in momentum space (Sec. 2.2; the D1 of Eqs. uity, nzav) */
  WZ_OP_D = 10            /* D psi: the overlap operator D = 1 - V = D1 + D2, with
                             D2(p) = 1 - b(p)/omega(p) (Sec. 2.2, Eq. d1mom); used by the
                             locality probe of Sec. 3.2 */
};

/* Lattice and action parameters (Sec. 2.2, Eq. fmat, Eq. acws). */
typedef struct wz_params {
  int dims[4];            /* T, Z, Y, X */
  double m_re, m_im;      /* bare mass m */
  double g_re, g_im;      /* Yukawa coupling g */
  double r;               /* Wilson parameter (paper: 1) */
  double M0;              /* constant of the kernel A = M0 - D_W (paper: 1) */
  double yukawa;          /* c in c g phi P_+ : 2 in Eq. fmat, 1 in Sec. 7.1 */
} wz_params;

typedef struct wz_ctx wz_ctx;

/* Create a context on the current CUDA device.  stream is a cudaStream_t
 * (NULL = legacy default stream).  Computes the momentum-space tables
 * h(p) = 2/(omega+b) etc. in FP64 on the device (Sec. 3.1, Eq. d1mom).
 * Returns WZ_EINVAL for odd T, X != Y or an extent without kernels. */
int wz_create(const wz_params* p, void* stream, wz_ctx** out);
int wz_destroy(wz_ctx* ctx);
const char* wz_last_error(const wz_ctx* ctx);
/* 1 if an extent n has compiled kernels (spatial / time), else 0. */
int wz_supported_extent(int n);

/* Workspace budget (not part of the method).  A context grows its device
 * workspaces on demand: the solver's vectors, the apply intermediates, the
 * force and HMC fields.  wz_set_workspace_limit caps their total in bytes
 * (0 removes the cap).  A call that would need more returns WZ_ENOMEM, as
 * when cudaMalloc runs out of device memory; the refused growth releases
 * nothing, so the context stays usable for every call that fits.
 * wz_workspace_bytes returns what the workspaces hold now (tables, phi and
 * the caller's fields are not counted). */
int wz_set_workspace_limit(wz_ctx* ctx, size_t bytes);
size_t wz_workspace_bytes(const wz_ctx* ctx);

/* Set the scalar field phi (complex128 [T][Z][Y][X], host or device).  The
 * context keeps an FP64 copy and an FP32 copy for the inner solver. */
int wz_set_phi(wz_ctx* ctx, const void* phi);

/* out = op(in) for nrhs fields of the given dtype (wz_op).  shift is added
 * for the *_DAGM ops.  in and out may alias.  Asynchronous for device
 * pointers. */
int wz_apply(wz_ctx* ctx, int op, int dtype, const void* in, void* out, int nrhs, double shift);

/* Solver flags (bitwise or). */
enum wz_solve_flags {
  WZ_SOLVE_MIXED = 1,     /* FP32 iteration with FP64 reliable updates (Sec. 7.4 suggests
                             mixed precision after Clark et al.); else FP64 throughout */
  WZ_SOLVE_PC = 2         /* M0^-1 preconditioning of Sec. 7.3 (Eq. theprob); a shifted system
                             is solved as (M~^dag M~ + shift M0^-1dag M0^-1) x~ = b~, the
                             form Sec. 7.4 gives for Eq. yuier */
};

typedef struct wz_solve_stats {
  int iterations;          /* max over right-hand sides of inner CG iterations */
  int total_iterations;    /* sum over right-hand sides */
  int reliable_updates;    /* sum over RHS of FP64 residual recomputations */
  int converged;           /* right-hand sides that reached tol */
  double max_true_residual;/* max over RHS of ||b - (M^dag M + shift) x|| / ||b||, FP64,
                              of the ORIGINAL (unpreconditioned) system */
  double seconds;          /* host wall time of the call, including the final sync */
  double site_applies;     /* sum over systems of (inner iterations + reliable updates)
                              x sites of the system's lattice: the M^dag M work in site
                              units, comparable across lattices of different size */
} wz_solve_stats;

/* Solve (M^dagger M + shift) x = b for nrhs independent complex128 fields by
 * conjugate gradient (Sec. 7.2, Eqs. theprob, yuier), x0 = 0.  Each RHS stops
 * when its FP64 true relative residual ||b - A x|| / ||b|| <= tol (for
 * WZ_SOLVE_PC: the residual of the preconditioned system; the original one
 * is reported in stats).  b and x may be host or device pointers and must not
 * alias.  Synchronous: returns after the solution is in x.  Returns
 * WZ_NOT_CONVERGED (x = last iterate, stats filled) if maxiter inner
 * iterations did not suffice for some RHS, WZ_ENONFINITE (x undefined) as soon
 * as a norm of some RHS becomes NaN or Inf (non-finite b, phi or couplings).
 * resid (may be NULL) receives nrhs FP64 true relative residuals of the
 * original system. */
int wz_solve(wz_ctx* ctx, const void* b, void* x, int nrhs, double shift, double tol, int maxiter,
             unsigned flags, wz_solve_stats* stats, double* resid);

/* Shifted systems of a rational approximation (Eq. yuier): for every shift
 * beta_i (i < nshift <= 64, beta_i >= 0) and right-hand side b_j (j < nrhs),
 * solve (M^dagger M + beta_i) x_ij = b_j, all nshift * nrhs systems as
 * right-hand sides of one batched CG (each stops on its own residual, as in
 * wz_solve).  x holds nshift * nrhs complex128 fields ordered
 * [member][shift][rhs of the member] (a single lattice: [shift][rhs]).
 * Flags, tolerance, host/device pointers and return codes as wz_solve; stats
 * cover all systems, resid (may be NULL) gets nshift * nrhs residuals in x's
 * order. */
int wz_solve_multishift(wz_ctx* ctx, const void* b, void* x, int nrhs, int nshift, const double* shifts,
                        double tol, int maxiter, unsigned flags, wz_solve_stats* stats, double* resid);

/* ---- rational approximations (Eqs. jkjk, hbeq; Sec. 7.4) ----
 *
 * x^power ~ r(x) = a0 + sum_{i<d} alpha_i / (x + beta_i) on [lo, hi]: the
 * pseudofermion action uses power -1/4 (phase-quenched |Pf| = det(M^dag M)^1/4),
 * the heatbath +1/8.  The paper asks for error-minimising coefficients and prints
 * none; wz_rational_minimax computes the minimax RELATIVE error approximation of
 * type (d, d) (Remez exchange; see remez.cu for the method). */
#define WZ_RATIONAL_MAX 64
typedef struct wz_rational {
  int d;                          /* poles, 0 <= d <= WZ_RATIONAL_MAX */
  double a0;                      /* alpha_0 */
  double alpha[WZ_RATIONAL_MAX];  /* residues alpha_1 .. alpha_d (entries >= d unused) */
  double beta[WZ_RATIONAL_MAX];   /* shifts beta_1 .. beta_d > 0, ascending */
  double power;                   /* the exponent approximated (informational) */
  double lo, hi;                  /* interval asked for */
  double build_lo, build_hi;      /* interval the exchange ran on (wider where double
                                     precision could not resolve the optimum on [lo, hi]) */
  double err;                     /* max |r(x)/x^power - 1| over [lo, hi], measured */
} wz_rational;

/* Minimax relative approximation of x^power, 0 < |power| < 1, on 0 < lo < hi,
 * degree d.  Host-only computation (no context, no GPU).  WZ_EINVAL on bad
 * arguments, WZ_NOT_CONVERGED if the exchange failed. */
int wz_rational_minimax(double power, double lo, double hi, int d, wz_rational* out);

/* Spectral interval of the free operator M0^dagger M0 = D_mu^dag D_mu + |m|^2
 * (Sec. 7.3) over the lattice momenta: the range Sec. 7.4 uses for the
 * approximations at weak coupling.  lo, hi: host doubles.  Synchronous. */
int wz_spectral_bounds(wz_ctx* ctx, double* lo, double* hi);

/* out = r(M^dagger M) in = a0 in + sum_i alpha_i (M^dagger M + beta_i)^-1 in for
 * nrhs complex128 fields (host or device; out must not alias in), with the d
 * shifted solves of Eq. yuier batched in one CG to tolerance tol.  With
 * WZ_SOLVE_PC in flags the poles beta_i <= pc_cutoff are solved with the M0^-1
 * preconditioning (the paper uses it up to beta = 100, Sec. 7.4) and the rest
 * without (single-lattice contexts).  Synchronous; stats cover every solve. */
int wz_rational_apply(wz_ctx* ctx, const wz_rational* r, const void* in, void* out, int nrhs, double tol,
                      int maxiter, unsigned flags, double pc_cutoff, wz_solve_stats* stats);

/* ---- forces, actions, molecular dynamics, HMC (Eq. acws; Sec. 7.2) ----
 *
 * Bosonic action S_B = sum_x [2 phi^* (D2 phi) + W'^* (1 - D2/2) W'], W' = m phi + g phi^2,
 * scalars periodic (Eq. acws).  Pseudofermion action with one pole (Eq. jkjk with
 * alpha = 1, beta = 0): S_pf = sum_k eta_k^dag (M^dag M)^-1 eta_k.  Forces are
 * G = dS/dphi_R + i dS/dphi_I per site (complex128 [T][Z][Y][X]):
 *   G_B  = 4 (D2 phi) + 2 conj(m + 2 g phi) ((1 - D2/2) W')
 *   G_pf = -2 Re[Z^dag dM/dphi_R X] - 2i Re[Z^dag dM/dphi_I X], X = (M^dag M)^-1 eta, Z = M X
 * phi is the context's field (wz_set_phi / wz_get_phi). */
enum wz_force_parts { WZ_FORCE_FERMION = 1, WZ_FORCE_BOSON = 2 };
enum wz_hmc_flags {
  WZ_HMC_FP64_SOLVES = 1,    /* FP64 CG in the force (default: mixed FP32/FP64) */
  WZ_HMC_NO_METROPOLIS = 2   /* keep the end of the molecular dynamics (tests) */
};

typedef struct wz_hmc_params {
  double tau;              /* trajectory length */
  int nsteps;              /* integration steps */
  int integrator;          /* 0: leapfrog; 1: Omelyan 2MN, lambda = 0.1931833275037836 */
  int npf;                 /* pseudofermions (one CG right-hand side each) */
  double tol;              /* CG true relative residual of every force solve */
  int maxiter;             /* per solve (<= 0: 100000) */
  unsigned flags;          /* wz_hmc_flags */
  unsigned long long seed; /* Philox4x32-10 key (Salmon et al. SC'11) */
  unsigned int traj_index; /* counter word: trajectory number */
} wz_hmc_params;

typedef struct wz_traj_stats {
  double H0, H1, dH, u;    /* Hamiltonians (FP64), dH = H1 - H0, Metropolis uniform */
  int accept;
  int force_evals;
  long long cg_iterations; /* inner CG iterations summed over all solves and RHS */
  int reliable_updates;
  double seconds;
} wz_traj_stats;

/* Copy the context's phi (complex128, host or device pointer). */
int wz_get_phi(wz_ctx* ctx, void* phi);

/* grad = dS/dphi (complex128 [T][Z][Y][X], host or device) of S = S_B and/or
 * S_pf (parts = wz_force_parts) at the context's phi; eta: npf complex128
 * pseudofermion fields (host or device).  S_B and S_pf (may be NULL) receive
 * the actions.  The solves use mixed precision to FP64 true residual tol.
 * Synchronous.  WZ_NOT_CONVERGED if a solve hit its iteration cap. */
int wz_force(wz_ctx* ctx, const void* eta, int npf, double tol, unsigned parts, void* grad, double* S_B,
             double* S_pf, wz_solve_stats* stats);

/* S_B and S_pf (either may be NULL, not both) at the context's phi: the actions
 * of wz_force without the gradient.  Synchronous. */
int wz_action(wz_ctx* ctx, const void* eta, int npf, double tol, double* S_B, double* S_pf, wz_solve_stats* stats);

/* Molecular dynamics of length h->tau in h->nsteps steps from (phi, pi) with
 * fixed pseudofermions eta (npf, complex128): phi (context) and pi (complex128
 * [T][Z][Y][X], host or device, updated in place) evolve by d phi = pi,
 * d pi = -G.  Synchronous. */
int wz_md_integrate(wz_ctx* ctx, void* pi, const void* eta, int npf, const wz_hmc_params* h, wz_traj_stats* st);

/* One HMC trajectory on the context's phi: pi ~ N(0,1) per real component and
 * R_k ~ exp(-|R|^2) drawn on the device from Philox4x32-10 (key = seed,
 * counter = (site, draw, stream, traj_index)), eta_k = M^dag R_k,
 * H = |pi|^2/2 + S_B + S_pf in FP64, molecular dynamics, Metropolis on the
 * device with a Philox uniform; on rejection phi is restored.  Synchronous. */
int wz_trajectory(wz_ctx* ctx, const wz_hmc_params* h, wz_traj_stats* st);

/* RHMC (Secs. 7.2, 7.4): the pseudofermion action is S_pf = sum_k eta_k^dag
 * r_a(M^dag M) eta_k with r_a ~ x^-1/4 (wz_rational), its force the
 * alpha_i-weighted sum of single-pole forces at shifts beta_i.  As wz_force with
 * the rational action (r_a->d shifted solves per pseudofermion, batched). */
int wz_rhmc_force(wz_ctx* ctx, const void* eta, int npf, const wz_rational* action, double tol, unsigned parts,
                  void* grad, double* S_B, double* S_pf, wz_solve_stats* stats);

/* One RHMC trajectory: as wz_trajectory, with the heatbath eta_k = r_h(M^dag M) R_k
 * (r_h ~ x^1/8, Eq. hbeq) and the rational action r_a for H and the force.
 * S_pf at both ends is evaluated with r_a from the solves of the first and last
 * force evaluations.  h->npf pseudofermions; h->tol for every solve.  In graph
 * mode the whole trajectory (both solve kinds included) is one CUDA graph. */
int wz_rhmc_trajectory(wz_ctx* ctx, const wz_hmc_params* h, const wz_rational* action, const wz_rational* heatbath,
                       wz_traj_stats* st);

/* ---- observables ----
 *
 * Auxiliary-field VEV (Sec. 7.5): F~ = -(1 - D2/2)(m^* phi^* + g^* phi^*2) on the
 * equation of motion of Eq. lata; since (1 - D2/2)(p = 0) = 1 its volume average
 * is -(1/V) sum_x (m^* phi^* + g^* phi^*2).  F receives (re, im) per member of
 * the context (2 doubles for a single lattice).  Synchronous. */
int wz_aux_vev(wz_ctx* ctx, double* F);

/* Broken supersymmetric Ward-Takahashi identity of Eq. exid at the context's phi.
 * Summed over x the variation density of the action is the cubic form of
 * Eq. nzav; with the fermions integrated out (Majorana propagator -M^-1 C^-1,
 * C = gamma_0 gamma_2, whose sign and C^T = -C leave M^-1 C^-1 in WR) and the
 * fermion summed over the lattice (a uniform source:
 * four solves of M psi_b = C^-1 e_b, one per spin column b) both sides are
 * per-configuration 4 x 4 complex matrices, the common sqrt 2 left out:
 *   WL[a][b] = F_b C[a][b], F_b = sum_x F~ (b = 2, 3: P_+) or sum_x F~^* (b = 0, 1: P_-)
 *   WR[a][b] = sum_x [g (2 phi (D1 phi) P_+ + phi^2 D1 P_+) psi_b
 *                     + g^* (2 phi^* (D1 phi^*) P_- + phi^*2 D1 P_-) psi_b]_a
 * with D1 the gamma-odd part of the overlap (on the scalar: sum_mu gamma_mu
 * F^-1[i sin p_mu / omega F phi], periodic).  The identity is <WR> = <WL>.
 * WR, WL: 32 host doubles each, row-major [a][b], (re, im).  flags: WZ_SOLVE_MIXED
 * or 0 (FP64 solves to true residual tol).  Synchronous. */
int wz_ward_identity(wz_ctx* ctx, double tol, int maxiter, unsigned flags, double* WR, double* WL,
                     wz_solve_stats* stats);

/* Correlators of the naive lattice supercurrent (Eq. latsuc) with the scalar and
 * the fermion, Eq. sitre, at the context's phi, both x and y projected on zero
 * spatial momentum.  The current is S_mu(x) = Gamma_mu(x) chi(x),
 *   Gamma_mu = sqrt2 [(D1 phi) gamma_mu P_+ + (D1 phi^*) gamma_mu P_-
 *                     + W' gamma_mu P_- + W'^* gamma_mu P_+],   W' = m phi + g phi^2,
 * D1 on the scalar as in wz_ward_identity, and <chi(x) chi^T(z) C> = -M^-1(x, z).
 * The source z is weighted by the caller's field w (a point, a wall or Gaussian
 * noise with E[w(z) w^*(z')] = delta(z, z'), whose mean then sums all source
 * positions):
 *   psi_b = -M^-1 (w e_b)  (four solves, b = 0..3),   xi(t) = sum_zvec w(t, zvec)
 *   Q_mu(t)[a][b] = sum_xvec [Gamma_mu psi_b]_a(t, xvec),   Phi_0(t) = sum_yvec phi, Phi_1 = Phi_0^*
 *   R[s][mu][dx][dy][a][b] = sum_t' xi(t')^* sgn Phi_s(t' + dy) Q_mu(t' + dx)[a][b]
 * with times mod T and sgn = -1 where t' + dx >= T (the antiperiodic fermion
 * crossing the boundary), so dx, dy are sink times relative to the source.
 * w: complex128 [T][Z][Y][X], host or device (16-byte aligned), not modified.
 * R: host, 2 * 4 * T * T * 16 complex (re, im interleaved) in the index order
 * above.  flags: WZ_SOLVE_MIXED or 0.  Errors: WZ_EINVAL (null pointer, tol <= 0,
 * maxiter < 1, misaligned w, batched context); WZ_NOT_CONVERGED (R from the best
 * iterates); WZ_ENONFINITE (NaN or Inf in w or phi).  Synchronous. */
int wz_supercurrent(wz_ctx* ctx, const void* w, double tol, int maxiter, unsigned flags, double* R,
                    wz_solve_stats* stats);

/* Locality probe of Dslash (Sec. 3.2, Eq. uir): psi = Dslash eta for a unit
 * point source eta (spin 0 at the origin); f[r] = max ||psi(x)|| over the sites
 * at taxi-driver distance r = sum_mu min(|x_mu|, L_mu - |x_mu|).  f needs
 * T/2 + Z/2 + Y/2 + X/2 + 1 entries (nf); FP64.  Synchronous. */
int wz_locality(wz_ctx* ctx, double* f, int nf);
/* The same probe for another operator: op = WZ_OP_DSLASH (as wz_locality) or
 * WZ_OP_D, the overlap operator, whose |D(x, 0)| decays exponentially with
 * the taxi-driver distance (Sec. 3.2, after Hernandez et al.).  Errors as
 * wz_locality; WZ_EINVAL for another op. */
int wz_locality_op(wz_ctx* ctx, int op, double* f, int nf);

/* ---- one-loop lattice sums (Sec. 5, Tables sse, fse, ase) ----
 *
 * Counterterms over |g|^2 on an N^4 momentum lattice (a = 1, N even, 4 <= N <=
 * 4096, k periodic), bare mass ma (mL = N ma), external momentum
 * p = (0, 0, 0, 2 pi / N): z[0] = Z_phi - 1 = Sigma_phi(p) / sin^2(2 pi/N),
 * z[1] = Z_chi - 1 = -Sigma_chi(p)_3 / sin(2 pi/N), z[2] = Z_F - 1 = Sigma_F(0),
 * with the integrands of Sec. 5.2 (P = sin k, M = 1 - 2 sum sin^2(k/2),
 * s = sqrt(P^2 + M^2), r = 2(1 - M/s) + (ma^2/2)(1 + M/s)).  FP64 on the current
 * device, no context; synchronous.  WZ_EINVAL on bad arguments. */
int wz_one_loop(int N, double ma, double* z);

/* ---- batches of independent lattices (replicas of uneven extent and coupling) ----
 *
 * A batch holds n lattices, each with its own dims, m, g and phi (e.g. the
 * multicanonical replicas of Sec. 6 run side by side).  Lattices of equal
 * extent share one set of momentum tables and are processed together: one
 * launch per pass covers all right-hand sides of all lattices of that extent;
 * groups of different extent run concurrently on their own streams.  Lattice
 * i draws its HMC random numbers with the Philox key seed + i. */
typedef struct wz_batch wz_batch;
int wz_batch_create(const wz_params* params, int n, void* stream, wz_batch** out);
int wz_batch_destroy(wz_batch* batch);
const char* wz_batch_last_error(const wz_batch* batch);
int wz_batch_size(const wz_batch* batch);     /* lattices */
int wz_batch_groups(const wz_batch* batch);   /* extent groups */
/* phi of lattice i (complex128, host or device) */
int wz_batch_set_phi(wz_batch* batch, int i, const void* phi);
int wz_batch_get_phi(wz_batch* batch, int i, void* phi);
/* b[i], x[i]: nrhs complex128 fields of lattice i (host or device).  Solves
 * (M_i^dag M_i) x = b for every lattice like wz_solve (no preconditioning);
 * stats summed over the batch (iterations: maximum).  Synchronous. */
int wz_batch_solve(wz_batch* batch, const void* const* b, void* const* x, int nrhs, double tol, int maxiter,
                   unsigned flags, wz_solve_stats* stats);
/* One HMC trajectory of every lattice (wz_trajectory); st: n entries. */
int wz_batch_trajectory(wz_batch* batch, const wz_hmc_params* h, wz_traj_stats* st);

/* (M^dagger M + shift) psi like wz_apply(WZ_OP_MDAGM), without allocating.
 * The paper has no counterpart: this serves callers that cannot allocate
 * device memory at call time (all memory handed to their own pool, a loop in
 * which a possibly synchronising cudaMalloc is not acceptable, or code that
 * must not fail half-way with an out-of-memory error).  The pass
 * intermediates live in a file-scope device array of 32 MiB that every GPU
 * loading the library holds until exit; a call needing more (2 fields of
 * nrhs x V x 4 complex: e.g. at 16^4 up to 2 RHS in C128, 4 in C64) returns
 * WZ_EINVAL with a message.  in and out are device pointers of dtype on the
 * context's device, which must be current (WZ_EINVAL otherwise); they may
 * alias.  The first call on a device looks up the array's device address
 * (and may load the library's device code there): make it during set-up,
 * before any stream capture.  All calls share the array; calls that overlap
 * on the GPU race on it.  Asynchronous on the context stream. */
int wz_apply_mdagm_noalloc(wz_ctx* ctx, int dtype, const void* in, void* out, int nrhs, double shift);

/* ---- measurement (not part of the method; the paper times whole solves) ----
 * Process-wide count of kernels launched by the library so far. */
unsigned long long wz_kernel_launches(void);

/* Kernel probe.  wz_probe_begin arms a probe for one kernel class:
 *   kind 0 zt pass, 1 apply xy pass, 2..4 CG passes P1/P3/P5, 5..6 reliable-update
 *   passes; real_bytes 4 (FP32 kernels) or 8 (FP64 kernels).
 * Until wz_probe_end, every launch of that class is bracketed by CUDA events
 * on its stream (the first 32768 launches) and each block of a timed launch
 * that does work (is not gated off) adds the algorithmic bytes it moves --
 * the spinor, phi and table bytes it must read and write -- to a device
 * counter.  wz_probe_end synchronises the device and returns the summed
 * event time and the summed algorithmic bytes, both over the timed launches
 * only, so bytes / total_ms is the achieved rate of those launches. */
typedef struct wz_probe_result {
  long launches;        /* launches of the class while armed */
  long timed_launches;  /* launches bracketed by events */
  double total_ms;      /* summed event time of the timed launches */
  double bytes;         /* algorithmic bytes moved by the blocks of the timed launches */
} wz_probe_result;
int wz_probe_begin(int kind, int real_bytes);
int wz_probe_end(wz_probe_result* out);

/* Self-test of the bounded device waits (the failure path behind WZ_ETIMEOUT):
 * one block initialises an mbarrier, announces 16 transaction bytes that no
 * copy delivers, and polls it with mbarrier.try_wait at most `polls` times
 * (1 <= polls <= 65536; the staged passes use the same loop with
 * WZ_MBAR_SPIN_LIMIT polls).  *status receives WZ_ETIMEOUT when the wait ran
 * out as designed (WZ_OK would mean the phase completed); *cycles the SM clock
 * cycles the polling took, from which the duration of the passes' limit
 * follows.  No copy is issued and nothing is left in flight.  Runs on the
 * current device, synchronous. */
int wz_selftest_wait_timeout(int polls, int* status, long long* cycles);

/* FMA throughput of the current device (measurement, not part of the method):
 * 8 SM-resident blocks of 256 threads per SM, each thread running 8
 * independent chains of `iters` fused multiply-adds in FP64 (real_bytes 8) or
 * FP32 (4); *tflops = 2 x FMAs / event time of one launch after a warm-up,
 * *ms that time.  The roofline of the arithmetic-bound FP64 passes uses the
 * FP64 figure.  1 <= iters <= 2^24.  Synchronous; allocates and frees a small
 * output buffer. */
int wz_fma_peak(int real_bytes, int iters, double* tflops, double* ms);

#ifdef __cplusplus
}
#endif
#endif /* WZ_H */
