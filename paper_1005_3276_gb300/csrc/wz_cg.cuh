// Conjugate gradient on M^dagger M + sigma fused into the plane passes.
//
// CG on the Hermitian positive-definite operator A = M^dagger M + sigma
// (Eq. theprob, Eq. yuier; sigma = 0 for the plain problem), one independent
// recursion per right-hand side, all right-hand sides in the same launches.
// One iteration is five plane passes plus a one-warp-per-RHS scalar kernel:
//
//   P1 (xy)  x += alpha' p (alpha' of the previous iteration) ; p = r + beta p ; A = F_xy p
//   P2 (zt)  A <- Dslash(p) A                  (M0^-1(p) when preconditioned)
//   P3 (xy)  C = M p (position space) ; A = F_xy C' ; partial |C|^2 + sigma |p|^2
//   P4 (zt)  A <- -Dslash(p) A                 ((M0^-1)^dag(p) when preconditioned)
//   P5 (xy)  Ap = M^dag C + sigma p ; alpha = rr / (p.Ap) ; r -= alpha Ap ;
//            partial |r|^2
//   S        rr_new, beta = rr_new / rr, reliable-update and stop tests
//
// sigma is a property of each right-hand side (RhsState::shift): the d shifted
// systems (M^dag M + beta_i) X_i = eta of a rational approximation (Eq. jkjk,
// Eq. yuier) run as d right-hand sides of one solve.  Preconditioned, the
// shifted operator is M~^dag M~ + sigma M0^-1^dag M0^-1 (the form Sec. 7.4 gives
// for Eq. yuier): with u = M0^-1 p in position space, P3 forms C = p + Y u,
// adds sigma |u|^2 to p.Ap and transforms Y^dag C + sigma u, so that P5's
// C + M0^-1^dag(Y^dag C + sigma u) is the whole operator.
//
// p.Ap = |M p|^2 + sigma |p|^2 is known after P3, so P5 updates r without
// storing Ap; the x update of an iteration is deferred to the next P1, which
// reads p anyway (or to the reliable update, which folds it in).  Reductions are deterministic: per-thread
// partials, a fixed warp/block tree, one partial per block, and every
// consumer sums the block partials in the same order.
//
// Mixed precision (reliable updates, Clark et al. 2010; Sleijpen and van der
// Vorst 1996): the recursion runs in FP32; when |r| has dropped below delta
// times its value at the last update (or below tol |b|), the FP32 iterate is
// folded into the FP64 solution and the residual is recomputed in FP64:
//
//   RU_P1 (xy, FP64) x_hi += x_lo + alpha p (the pending update) ; x_lo = 0 ; A = F_xy x_hi
//   zt, P3, zt       (FP64 M^dagger M as above)
//   RU_P5 (xy, FP64) r = b - (M^dag M + sigma) x_hi ; r_lo = (float) r ; partial |r|^2
//   S_ru             converged if |r| <= tol |b|, else beta = |r|^2 / rr_prev
//
// The pure FP64 solver is the same code with FP64 iteration vectors and
// delta = 0 (the update then only runs as the final true-residual check).
#pragma once
#include "../../include/wz.h"
#include "wz_kernels.cuh"
#include "wz_tma.cuh"

// register budget of the CG passes, in 256-thread blocks per SM (3: 85
// registers a thread); measured against 1, 2 and 4 on the 16^4 x 12 RHS solve
#ifndef WZ_XY_MINB
#define WZ_XY_MINB 3
#endif

namespace wz {

struct RhsState {
  double rr;       // |r|^2 of the recursive residual
  double rr_prev;  // previous |r|^2 (beta after a reliable update)
  double beta;     // beta of the next direction update
  double bnorm2;   // |b|^2
  double rmax2;    // |r|^2 at the last reliable update
  double rtrue2;   // |b - A x|^2 at the last reliable update (FP64)
  double tol2;     // stop when |b - A x|^2 <= tol2 |b|^2
  double alpha;    // alpha of the last iteration, whose x += alpha p is still pending
  double shift;    // sigma of this system: A = M^dag M + sigma
  int run;         // iteration passes act on this RHS
  int ru;          // reliable update pending
  int active;      // not finished
  int iters;       // inner iterations
  int ru_count;    // reliable updates done (FP64 applies)
  int status;      // WZ_OK, WZ_NOT_CONVERGED, WZ_ENONFINITE (or a staged-copy error)
};

enum CGMode { CG_P1 = 0, CG_P3, CG_P5, RU_P1, RU_P5 };

template <typename R, typename LO> struct CGArgs {
  cplx<R>* A;           // momentum intermediate (in place)
  cplx<R>* Cb;          // M p (or M~ p) in position space
  cplx<R>* p;           // search direction; x_hi for the RU passes
  cplx<R>* r;           // residual (iteration precision)
  cplx<R>* x;           // iterate accumulated between reliable updates
  cplx<LO>* lo_x;       // RU_P1: low-precision iterate folded in and zeroed
  const cplx<LO>* lo_p; // RU_P1: search direction of the pending x update
  cplx<LO>* lo_r;       // RU_P5: residual written in the iteration precision
  const cplx<R>* b;     // RU_P5: right-hand side
  const cplx<R>* phi;    // [member][T][Z][Y][X]
  const SiteCoef<R>* kArr;  // couplings per member
  int rpm;              // right-hand sides per member
  int Z;                // planes per time slice (plane = t * Z + z)
  const R* twc;         // cos / sin (pi t / T): antiperiodic twist (see xy_pass)
  const R* tws;
  int shifted;          // some right-hand side has sigma != 0 (probe byte counts only)
  RhsState* st;
  double* part_out;     // [rhs][nblk] block partials written by this pass (may be null)
  const double* part_in;  // [rhs][nblk] block partials of p.Ap (CG_P5)
  int nblk;             // blocks per right-hand side
  int TZ;               // planes per right-hand side
  int gate_ru;          // 1: act on RHS with a pending reliable update; 0: on running RHS
  int rhs0;             // first right-hand side of this launch (blockIdx.y counts from it)
  unsigned long long* blk_count;  // probe: byte counter (may be null)
  unsigned long long probe_inc;   // probe: algorithmic bytes one block moves
  int pdl;              // host side: launch with programmatic stream serialization
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum of v over the block, valid on thread 0.  Whole warps only.
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  return t;
}

// Sum of the nblk partials of one RHS, in a fixed order; valid on lane 0.
__device__ __forceinline__ double sum_partials(const double* part, int nblk) {
  const int lane = threadIdx.x & 31;
  double t = 0.0;
  for (int i = lane; i < nblk; i += 32) t += part[i];
  return warp_sum(t);
}

template <typename R> __device__ __forceinline__ R norm2(cplx<R> a) { return a.x * a.x + a.y * a.y; }

// TMA bulk prefetch of a contiguous global range into L2 (16-byte aligned,
// size a multiple of 16): the phase-B operands of a plane are requested at
// block entry and arrive while the block is busy with its phase-A FFT.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Shared memory of xy_cg: the plane workspace (PPC planes with row padding),
// 33 reduction doubles, two mbarriers and, in the staged FP32 iteration passes,
// one buffer of PPC planes per staged operand.  Staged (bulk copies issued at
// block entry, so they overlap the phase-A FFT): P1 r, p and x (x into the
// workspace, which P1 only needs after phase B); P3 the momentum input A (into
// the workspace) and p; P5 A, C and r; P3 and the unpreconditioned P5 also the
// phi planes of the site term.  Extents up to 32 (at 32 one plane per block:
// 98 KB for P1, two blocks per SM).
template <typename R, int L, int MODE, bool PC> struct CGSmem {
  using S = XYShape<L>;
  static constexpr bool STAGE = sizeof(R) == 4 && L <= 32 && (MODE == CG_P1 || MODE == CG_P3 || MODE == CG_P5);
  static constexpr int NSTAGE = !STAGE ? 0 : (MODE == CG_P3 ? 1 : 2);
  static constexpr bool STAGE_PHI = STAGE && (MODE == CG_P3 || (MODE == CG_P5 && !PC));
  static constexpr int PLANE_ELEMS = L * L * 4;  // complex values of one plane, contiguous in global memory
  static constexpr size_t plane_bytes = sizeof(cplx<R>) * PLANE_ELEMS;
  static constexpr size_t phi_plane_bytes = sizeof(cplx<R>) * L * L;
  static constexpr size_t red_off = sizeof(cplx<R>) * S::PLANE * S::PPC;
  static constexpr size_t bar_off = (red_off + 33 * sizeof(double) + 15) & ~size_t(15);
  static constexpr size_t stage_off = (bar_off + 2 * sizeof(unsigned long long) + 127) & ~size_t(127);
  static constexpr size_t phi_off = stage_off + NSTAGE * S::PPC * plane_bytes;
  static constexpr size_t total = STAGE ? phi_off + (STAGE_PHI ? S::PPC * phi_plane_bytes : 0)
                                        : red_off + 33 * sizeof(double);
  static_assert(!STAGE || (plane_bytes % 16 == 0 && phi_plane_bytes % 16 == 0),
                "bulk copies move multiples of 16 bytes");
};

// Blocks per SM a CG pass is compiled for (its register budget): FP32 passes
// WZ_XY_MINB 256-thread blocks' worth of threads, but no more blocks than the
// pass's shared memory lets reside (228 KB per SM, 1 KB reserved a block), so
// that no pass is held to fewer registers than its occupancy allows; FP64
// passes (the FP64 solver and the reliable updates) two 256-thread blocks'
// worth (128 registers at 128 threads), one for 32-point lines (255).
template <typename R, int L, int MODE, bool PC> struct CGMinBlocks {
  static constexpr int by_threads = ((sizeof(R) == 8 ? (L >= 32 ? 1 : 2) : WZ_XY_MINB) * 256) / XYShape<L>::THREADS;
  static constexpr int by_smem = (int)((228u * 1024u) / (CGSmem<R, L, MODE, PC>::total + 1024u));
  static constexpr int value = by_threads < by_smem ? by_threads : (by_smem > 0 ? by_smem : 1);
};

template <typename R, typename LO, int L, int MODE, bool PC>
__global__ void __launch_bounds__(XYShape<L>::THREADS, (CGMinBlocks<R, L, MODE, PC>::value))
xy_cg(CGArgs<R, LO> a) {
  using S = XYShape<L>;
  using H = XYPhase<R, L>;
  using SM = CGSmem<R, L, MODE, PC>;
  constexpr bool STAGE = SM::STAGE;
  constexpr int PE = SM::PLANE_ELEMS;
  constexpr bool INV = (MODE == CG_P3 || MODE == CG_P5 || MODE == RU_P5);
  constexpr bool FWD = (MODE == CG_P1 || MODE == CG_P3 || MODE == RU_P1);
  extern __shared__ unsigned char smem_raw[];
  cplx<R>* sm = reinterpret_cast<cplx<R>*>(smem_raw);
  double* red = reinterpret_cast<double*>(smem_raw + SM::red_off);  // 33 doubles
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem_raw + SM::bar_off);
  cplx<R>* stg = reinterpret_cast<cplx<R>*>(smem_raw + SM::stage_off);  // [NSTAGE][PPC][PE]
  cplx<R>* sphi = reinterpret_cast<cplx<R>*>(smem_raw + SM::phi_off);   // [PPC][L * L]

  const int rhs = blockIdx.y + a.rhs0;
  RhsState* st = a.st + rhs;
  // Dependent launch: a pass waits for its predecessor (pdl_wait) before it
  // touches what that kernel writes, and every block waits before it leaves,
  // so that a grid completes only after the grid before it has.  The staged
  // FP32 passes issue the copies of the operands written two or more launches
  // back before that wait, so that they overlap the predecessor's tail: P1
  // (after the scalar kernel, which writes only the per-RHS state) r, p and x;
  // P3 and P5 (after a zt pass, which writes only A) p, C, r and phi.  Whether
  // to issue them early is decided from the gate as read before the wait (P1:
  // from whether the system is still active); the gate that counts is read
  // after the wait, and a block whose system does not run lets any copies it
  // issued land (bounded) and leaves.
  if constexpr (!STAGE) {
    pdl_wait();
    pdl_trigger();
    if (!(a.gate_ru ? st->ru : st->run)) return;  // whole block, before any barrier
  }

  // staged operands: one bulk copy per operand for the block's consecutive planes
  if constexpr (STAGE) {
    // bulk copies need 16-byte aligned shared and global addresses: checked,
    // the right-hand side is marked failed and no copy is issued otherwise
    const bool misaligned = ((smem_u32(sm) | smem_u32(stg) | smem_u32(sphi)) & 15u) != 0 ||
                            (((unsigned long long)a.r | (unsigned long long)a.p | (unsigned long long)a.x |
                              (unsigned long long)a.A | (unsigned long long)a.Cb | (unsigned long long)a.phi) &
                             15ull) != 0;
    if (__syncthreads_or(misaligned)) {
      pdl_wait();
      pdl_trigger();
      if (threadIdx.x == 0) {
        st->status = WZ_ECUDA;
        st->run = 0;
        st->ru = 0;
        st->active = 0;
      }
      return;
    }
    const int nlive = min(S::PPC, a.TZ - (int)blockIdx.x * S::PPC);
    const unsigned nb = (unsigned)(nlive * SM::plane_bytes);
    const long off0 = ((long)rhs * a.TZ + (long)blockIdx.x * S::PPC) * PE;
    // thread 0: the copies of the operands that do not come from the predecessor
    auto issue_operands = [&]() {
      if constexpr (MODE == CG_P1) {
        // p and x also in the first iteration (zeros), when alpha = beta = 0
        mbar_arrive_expect_tx(&bars[1], 3u * nb);
        bulk_g2s(stg, a.r + off0, nb, &bars[1]);
        bulk_g2s(stg + S::PPC * PE, a.p + off0, nb, &bars[1]);
        bulk_g2s(sm, a.x + off0, nb, &bars[1]);
      } else {
        // phi planes of the block's member (the planes are consecutive within it)
        const unsigned nphi = SM::STAGE_PHI ? (unsigned)(nlive * SM::phi_plane_bytes) : 0u;
        const long phi0 = ((long)(rhs / a.rpm) * a.TZ + (long)blockIdx.x * S::PPC) * (L * L);
        if constexpr (MODE == CG_P3) {
          mbar_arrive_expect_tx(&bars[1], nb + nphi);
          bulk_g2s(stg, a.p + off0, nb, &bars[1]);
        } else {
          mbar_arrive_expect_tx(&bars[1], 2 * nb + nphi);
          bulk_g2s(stg, a.Cb + off0, nb, &bars[1]);
          bulk_g2s(stg + S::PPC * PE, a.r + off0, nb, &bars[1]);
        }
        if constexpr (SM::STAGE_PHI) bulk_g2s(sphi, a.phi + phi0, nphi, &bars[1]);
      }
    };
    const bool hint = threadIdx.x == 0 && (MODE == CG_P1 ? *(volatile const int*)&st->active != 0
                                                         : *(volatile const int*)(a.gate_ru ? &st->ru : &st->run) != 0);
    if (threadIdx.x == 0) {
      mbar_init(&bars[0], 1);
      mbar_init(&bars[1], 1);
      mbar_fence_init();
    }
    const bool early = __syncthreads_or(hint);  // also publishes the initialised barriers
    if (threadIdx.x == 0 && early) issue_operands();
    pdl_wait();
    pdl_trigger();
    if (!__syncthreads_or((a.gate_ru ? st->ru : st->run) != 0)) {
      if (early) mbar_wait_bounded(&bars[1], 0);
      return;
    }
    if (threadIdx.x == 0) {
      if (!early) issue_operands();
      if constexpr (MODE != CG_P1) {
        // the momentum input A is the predecessor's output
        mbar_arrive_expect_tx(&bars[0], nb);
        bulk_g2s(sm, a.A + off0, nb, &bars[0]);
      }
    }
  }
  const double shift = st->shift;  // set before the iteration loop
  // a staged wait that ran out: mark this right-hand side failed, let the
  // copies in flight land (bounded) and leave as a whole block
  auto stage_failed = [&](bool ok) -> bool {
    if (!__syncthreads_or(!ok)) return false;
    if (threadIdx.x == 0) {
      st->status = WZ_ETIMEOUT;
      st->run = 0;
      st->ru = 0;
      st->active = 0;
    }
    if (MODE != CG_P1) mbar_wait_bounded(&bars[0], 0);
    mbar_wait_bounded(&bars[1], 0);
    return true;
  };

  const int tid = threadIdx.x;
  if (a.blk_count && tid == 0) atomicAdd(a.blk_count, a.probe_inc);
  const int pl_local = tid / S::TPP;
  const int w = (tid / 4) % L;
  const int s = tid & 3;
  const int plane_in = blockIdx.x * S::PPC + pl_local;
  const bool live = plane_in < a.TZ;
  const long plane = (long)rhs * a.TZ + plane_in;
  cplx<R>* P = sm + pl_local * S::PLANE;
  const long base = plane * (long)(L * L) * 4;

  cplx<R> v[L];
  R part = R(0);

  // operands of phase B, distinct arrays (lets the compiler hoist loads above stores)
  cplx<R>* __restrict__ Pp = a.p;
  cplx<R>* __restrict__ Pr = a.r;
  cplx<R>* __restrict__ Px = a.x;
  cplx<R>* __restrict__ Pc = a.Cb;
  const cplx<R>* __restrict__ Pb = a.b;
  cplx<LO>* __restrict__ Plx = a.lo_x;
  cplx<LO>* __restrict__ Plr = a.lo_r;
  if (live && (tid % S::TPP) == 0) {
    constexpr unsigned PB = L * L * 4 * sizeof(cplx<R>);
    const long pe = plane * (long)(L * L) * 4;
    if constexpr (MODE == CG_P5) {
      if (!PC && shift != 0.0) prefetch_l2(Pp + pe, PB);
      if constexpr (!STAGE) {
        prefetch_l2(Pc + pe, PB);
        prefetch_l2(Pr + pe, PB);
      }
    } else if constexpr (MODE == CG_P3) {
      if constexpr (!STAGE) prefetch_l2(Pp + pe, PB);
    } else if constexpr (MODE == RU_P5) {
      prefetch_l2(Pp + pe, PB);
      prefetch_l2(Pc + pe, PB);
      prefetch_l2(Pb + pe, PB);
    }
    if constexpr (MODE == CG_P5) (void)Px;
  }

  if constexpr (MODE == CG_P5) {
    // alpha = rr / p.Ap from the P3 partials: the same sum in every block
    if (tid < 32) {
      const double pAp = sum_partials(a.part_in + (long)rhs * a.nblk, a.nblk);
      if (tid == 0) red[32] = pAp > 0.0 ? st->rr / pAp : 0.0;
    }
  }
  if (INV) {
    if constexpr (STAGE) {
      // the plane's momentum input sits unpadded at the start of the workspace
      if (stage_failed(mbar_wait_bounded(&bars[0], 0))) return;
      if (live) {
        const cplx<R>* Ain = sm + pl_local * PE;
#pragma unroll
        for (int x = 0; x < L; ++x) v[x] = Ain[(x * L + w) * 4 + s];
      }
      __syncthreads();
      if (live) {
        fft_line<L, +1, R>(v);
#pragma unroll
        for (int x = 0; x < L; ++x) P[w * S::RP + x * 4 + s] = v[x];
      }
    } else {
      if (live) H::inv_x(a.A + base, P, w, s, v);
    }
    __syncthreads();
  }
  if constexpr (STAGE) {
    if (stage_failed(mbar_wait_bounded(&bars[1], 0))) return;
  }
  const cplx<R>* S0 = stg + pl_local * PE;                // first staged operand of this plane
  const cplx<R>* S1 = stg + S::PPC * PE + pl_local * PE;  // second
  const cplx<R>* SX = sm + pl_local * PE;                 // P1: staged x in the workspace
  R alpha = R(0), beta = R(0);
  if constexpr (MODE == CG_P5) alpha = (R)red[32];
  if constexpr (MODE == CG_P1) {
    beta = (R)st->beta;
    alpha = (R)st->alpha;  // pending x update of the previous iteration
  }
  const double alpha_pending = (MODE == RU_P1) ? st->alpha : 0.0;
  const R sigma = (R)shift;

  if (live) {
    const int x = w;
    const long site0 = plane * (long)(L * L) + x;
    const int member = rhs / a.rpm;
    const long phib = ((long)member * a.TZ + plane_in) * (L * L) + x;
    const SiteCoef<R> kc = a.kArr[member];
    const int tt = plane_in / a.Z;
    const cplx<R> twb{a.twc[tt], a.tws[tt]}, twf{a.twc[tt], -a.tws[tt]};
    if (INV) {
      H::inv_y(P, w, s, v);
#pragma unroll
      for (int y = 0; y < L; ++y) v[y] = twb * v[y];
    }
#pragma unroll
    for (int y = 0; y < L; ++y) {
      const long e = (site0 + y * L) * 4 + s;
      const int el = (y * L + x) * 4 + s;  // within the plane (staged copies)
      if constexpr (MODE == CG_P1) {
        // beta == 0 and alpha == 0 (first step): p = r without reading the previous p
        cplx<R> pv = STAGE ? S0[el] : Pr[e];
        if (beta != R(0) || alpha != R(0)) {
          const cplx<R> po = STAGE ? S1[el] : Pp[e];
          if (alpha != R(0)) Px[e] = (STAGE ? SX[el] : Px[e]) + alpha * po;
          pv = pv + beta * po;
        }
        Pp[e] = pv;
        v[y] = pv;
      } else if constexpr (MODE == CG_P3) {
        const cplx<R> pe = STAGE ? S0[el] : Pp[e];
        const cplx<R> f = SM::STAGE_PHI ? sphi[pl_local * (L * L) + y * L + x] : a.phi[phib + y * L];
        if constexpr (PC) {
          const cplx<R> u = v[y];  // M0^-1 p
          const cplx<R> cv = pe + site_coef<R, false, false>(kc, f, s) * u;
          Pc[e] = cv;
          part += norm2(cv) + sigma * norm2(u);
          v[y] = site_coef<R, true, false>(kc, f, s) * cv;
          if (sigma != R(0)) v[y] = v[y] + sigma * u;
        } else {
          v[y] = v[y] + site_coef<R, false, true>(kc, f, s) * pe;
          Pc[e] = v[y];
          part += norm2(v[y]) + sigma * norm2(pe);
        }
      } else if constexpr (MODE == CG_P5 || MODE == RU_P5) {
        const cplx<R> cv = STAGE ? S0[el] : Pc[e];
        cplx<R> ap;
        if constexpr (PC) ap = cv + v[y];
        else ap = v[y] + site_coef<R, true, true>(
                      kc, SM::STAGE_PHI ? sphi[pl_local * (L * L) + y * L + x] : a.phi[phib + y * L], s) * cv;
        if (!PC && sigma != R(0)) ap = ap + sigma * Pp[e];  // p, or x_hi for RU_P5
        if constexpr (MODE == CG_P5) {
          const cplx<R> rn = (STAGE ? S1[el] : Pr[e]) - alpha * ap;
          Pr[e] = rn;
          part += norm2(rn);
        } else {
          const cplx<R> rn = Pb[e] - ap;
          Plr[e] = cplx<LO>{(LO)rn.x, (LO)rn.y};
          part += norm2(rn);
        }
      } else if constexpr (MODE == RU_P1) {
        const cplx<LO> xl = Plx[e];
        const cplx<LO> pl = a.lo_p[e];
        const cplx<R> xv = Pp[e] + cplx<R>{(R)xl.x, (R)xl.y} + (R)alpha_pending * cplx<R>{(R)pl.x, (R)pl.y};
        Pp[e] = xv;
        Plx[e] = cplx<LO>{LO(0), LO(0)};
        v[y] = xv;
      }
    }
    if (FWD) {
#pragma unroll
      for (int y = 0; y < L; ++y) v[y] = twf * v[y];
    }
  }
  // P1 staged x in the workspace: every thread is done with it before fwd_y
  if constexpr (STAGE && MODE == CG_P1) __syncthreads();
  if constexpr (FWD) {
    if (live) H::fwd_y(v, P, w, s);
  }
  if constexpr (FWD) {
    __syncthreads();
    if (live) H::fwd_x(P, a.A + base, w, s, v);
  }
  if (a.part_out) {
    const double t = block_sum((double)part, red);
    if (tid == 0) a.part_out[(long)rhs * a.nblk + blockIdx.x] = t;
  }
}

// r = (R) b, x = p = 0, partial |b|^2 (FP64).  Grid (nblk, nrhs).
template <typename R>
__global__ void cg_init(const cplx<double>* b, cplx<R>* r, cplx<R>* x, cplx<R>* p, long n_per_rhs, double* part,
                        int nblk) {
  __shared__ double red[33];
  const int rhs = blockIdx.y;
  double t = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n_per_rhs; i += (long)nblk * blockDim.x) {
    const long e = (long)rhs * n_per_rhs + i;
    const cplx<double> bv = b[e];
    r[e] = cplx<R>{(R)bv.x, (R)bv.y};
    x[e] = cplx<R>{R(0), R(0)};
    p[e] = cplx<R>{R(0), R(0)};
    t += bv.x * bv.x + bv.y * bv.y;
  }
  t = block_sum(t, red);
  if (threadIdx.x == 0) part[(long)rhs * nblk + blockIdx.x] = t;
}

// Shifts of the systems of one solve, passed by value (so that a captured
// solve carries them): system q solves (M^dag M + beta[(q / inner) % d]) x = b.
// A plain solve has d = 1; the d poles of a rational approximation applied to
// npf right-hand sides per member are laid out [member][pole][rhs] (inner = npf).
#define WZ_SHIFT_MAX 64
struct ShiftSpec {
  int d = 1;
  int inner = 1;
  double beta[WZ_SHIFT_MAX] = {0.0};
  __host__ __device__ double of(int q) const { return beta[(q / inner) % d]; }
  // right-hand side (input field) of system q: [member][rhs] without the pole index
  __host__ __device__ long src(int q) const { return (long)(q / (inner * d)) * inner + q % inner; }
  bool any() const {
    for (int i = 0; i < d; ++i)
      if (beta[i] != 0.0) return true;
    return false;
  }
};

// bs[q] = b[sh.src(q)]: the right-hand side of every shifted system.  Grid (nb, nsys).
static __global__ void gather_rhs(const cplx<double>* b, cplx<double>* bs, long n_per_rhs, ShiftSpec sh) {
  const int q = blockIdx.y;
  const cplx<double>* src = b + sh.src(q) * n_per_rhs;
  cplx<double>* dst = bs + (long)q * n_per_rhs;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n_per_rhs; i += (long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// One warp per RHS.
static __global__ void cg_scalar_init(RhsState* st, const double* part, int nblk, double tol2, ShiftSpec sh) {
  RhsState* s = st + blockIdx.x;
  const double t = sum_partials(part + (long)blockIdx.x * nblk, nblk);
  if (threadIdx.x == 0) {
    s->bnorm2 = t;
    s->rr = t;
    s->rr_prev = t;
    s->beta = 0.0;
    s->rmax2 = t;
    s->rtrue2 = t;
    s->tol2 = tol2;
    s->alpha = 0.0;
    s->shift = sh.of(blockIdx.x);
    s->iters = 0;
    s->ru_count = 0;
    s->ru = 0;
    // a non-finite |b|^2 (NaN or Inf in the right-hand side) stops the system at once
    s->status = isfinite(t) ? WZ_OK : WZ_ENONFINITE;
    s->active = isfinite(t) && t > 0.0;
    s->run = s->active;
  }
}

// counters (may be null): [0] inner iterations summed over RHS, [1] reliable
// updates, [2] trips of a solver graph's WHILE loop
static __global__ void cg_scalar_iter(RhsState* st, const double* part, const double* part_pAp, int nblk,
                                      double delta2, int maxiter, unsigned long long* counters) {
  RhsState* s = st + blockIdx.x;
  pdl_wait();
  pdl_trigger();
  if (!s->run) return;
  const double t = sum_partials(part + (long)blockIdx.x * nblk, nblk);
  // the alpha P5 used (the same sum, in the same order): pending for the next P1
  const double pAp = sum_partials(part_pAp + (long)blockIdx.x * nblk, nblk);
  if (threadIdx.x == 0) {
    if (!isfinite(t) || !isfinite(pAp)) {  // NaN or Inf in the operator or the iterates
      s->status = WZ_ENONFINITE;
      s->run = 0;
      s->ru = 0;
      s->active = 0;
      return;
    }
    s->alpha = pAp > 0.0 ? s->rr / pAp : 0.0;
    s->iters += 1;
    if (counters) atomicAdd(&counters[0], 1ULL);
    s->beta = t / s->rr;
    s->rr_prev = s->rr;
    s->rr = t;
    if (t <= delta2 * s->rmax2 || t <= s->tol2 * s->bnorm2 || s->iters >= maxiter) {
      s->ru = 1;
      s->run = 0;
    }
  }
}

static __global__ void cg_scalar_ru(RhsState* st, const double* part, int nblk, int maxiter,
                                    unsigned long long* counters) {
  RhsState* s = st + blockIdx.x;
  pdl_wait();
  pdl_trigger();
  if (!s->ru) return;
  const double t = sum_partials(part + (long)blockIdx.x * nblk, nblk);
  if (threadIdx.x == 0) {
    s->ru = 0;
    s->ru_count += 1;
    if (counters) atomicAdd(&counters[1], 1ULL);
    s->rtrue2 = t;
    s->alpha = 0.0;  // RU_P1 folded the pending update into x_hi
    if (!isfinite(t)) {
      s->active = 0;
      s->run = 0;
      s->status = WZ_ENONFINITE;
    } else if (t <= s->tol2 * s->bnorm2) {
      s->active = 0;
      s->run = 0;
      s->status = WZ_OK;
    } else if (s->iters >= maxiter) {
      s->active = 0;
      s->run = 0;
      s->status = WZ_NOT_CONVERGED;
    } else {
      s->beta = t / s->rr_prev;
      s->rr = t;
      s->rmax2 = t;
      s->run = 1;
    }
  }
}

// Condition of the solver graph's WHILE node: continue while some RHS is
// active, and never beyond cap trips.
static __global__ void cg_loop_cond(cudaGraphConditionalHandle h, const RhsState* st, int nrhs, int* trips, int cap,
                                    unsigned long long* counters, int slot) {
  if (threadIdx.x != 0) return;
  int any = 0;
  for (int j = 0; j < nrhs; ++j) any |= st[j].active;
  const int t = ++*trips;
  if (counters) counters[slot] += 1ULL;
  cudaGraphSetConditional(h, (any && t < cap) ? 1u : 0u);
}

}  // namespace wz
