// Plane-pass kernels of the FFT-based fermion-matrix apply.
//
// The Dirac operator of Eq. fmat, Dslash = (1 - D2/2)^-1 D1, is diagonal in
// momentum space with Dslash(p) = i h(p) gamma_mu sin p_mu, h = 2/(omega + b)
// (Sec. 3.1, Eq. d1mom).  It is applied as "FFT, multiply, inverse FFT" (the
// FFT trick of Sec. 7.2).  A 4D FFT of a spinor field [rhs][T][Z][Y][X][4]
// is split into two plane passes that each keep one whole plane on chip:
//
//   xy pass : one (rhs, t, z) plane of Y x X sites, contiguous in memory;
//             its "phase B" owns y-lines in POSITION space, so every
//             site-local term (mass, Yukawa, CG vector updates, force
//             contractions) is fused there.
//   zt pass : a tile of C consecutive (p_x, p_y) columns for all (z, t);
//             forward FFT over (z, t), momentum-space spin multiply, inverse
//             FFT.  In place.  The antiperiodic twist exp(-+i pi t/T) is a
//             per-plane constant applied by the xy passes in position space.
//
// M = xy_fwd -> zt(+Dslash) -> xy_inv(+Y psi); M^dagger M fuses the middle xy
// passes (inverse, + Y psi, store M psi, forward) so it takes five passes.
//
// Every thread owns one line (N values of one spin component) in registers
// and transforms it with wz::fft_line; lines cross between directions through
// shared memory.  The four spin components of a site sit in four adjacent
// lanes, so the spin multiply of the zt pass exchanges the opposite-chirality
// components with warp shuffles.
#pragma once
#include "../../include/wz.h"
#include "wz_fft.cuh"
#include "wz_tma.cuh"

namespace wz {

// ----------------------------------------------------------------------------- dependent launch
// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// programmatic stream serialization may be scheduled while its predecessor on
// the stream is still running.  pdl_wait() returns once every prerequisite grid
// has completed and its memory writes are visible (at once for a plain launch);
// pdl_trigger() lets the successor be scheduled as soon as every block of this
// grid has called it or exited.  The kernels of the solver chain call both at
// entry, before their first global-memory access: a successor that starts
// early overlaps only its launch and block set-up with this grid's tail, and a
// grid triggers only after its own wait, so the grid before the predecessor
// has completed whenever a successor starts.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ----------------------------------------------------------------------------- site terms
// Y      = (m + c g phi) P_+ + (m^* + c g^* phi^*) P_-       (Eq. fmat)
// Y_int  =      c g phi  P_+ +        c g^* phi^*  P_-
// P_- acts on spin components 0, 1 and P_+ on 2, 3 (gamma_5 = diag(-1,-1,1,1)).
template <typename R> struct SiteCoef {
  R m_re, m_im;    // bare mass m
  R cg_re, cg_im;  // c * g with c the Yukawa coefficient (2 in Eq. fmat)
  R g_re, g_im;    // g itself (superpotential W' = m phi + g phi^2, Eq. acws)
};

// Members: a context can hold several lattices of the same extent (a batch of
// replicas with their own phi, m and g).  Right-hand side j belongs to member
// j / rpm; phi is stored [member][T][Z][Y][X] and kArr[member] holds the couplings.

// coefficient multiplying spin component s at a site with field value f
template <typename R, bool DAG, bool WITH_MASS>
__device__ __forceinline__ cplx<R> site_coef(const SiteCoef<R>& k, cplx<R> f, int s) {
  // y_plus = [m] + c g f
  cplx<R> yp = cplx<R>{k.cg_re, k.cg_im} * f;
  if (WITH_MASS) yp = yp + cplx<R>{k.m_re, k.m_im};
  // s >= 2: y_plus ; s < 2: conj(y_plus); dagger conjugates both
  const bool use_conj = (s < 2) != DAG;
  return use_conj ? conj(yp) : yp;
}

// ----------------------------------------------------------------------------- xy pass
enum XYMode {
  XY_FWD = 0,          // A_out = F_xy psi
  XY_FWD_YINTDAG,      // A_out = F_xy (Y_int^dag psi)
  XY_INV,              // v_out = F_xy^-1 A_in
  XY_INV_Y,            // v_out = F^-1 A_in + Y psi
  XY_INV_YDAG,         // v_out = F^-1 A_in + Y^dag psi (+ shift psi2)
  XY_INV_Y_FWD,        // v = F^-1 A_in + Y psi -> v_out ; A_out = F v
  XY_INV_PC,           // v_out = psi + Y_int F^-1 A_in
  XY_INV_PC_FWD,       // v = psi + Y_int F^-1 A_in -> v_out ; A_out = F (Y_int^dag v)
  XY_INV_ADD,          // v_out = psi + F^-1 A_in (+ shift psi2)
};

template <int M> struct XYModeInfo {
  static constexpr bool inv = !(M == XY_FWD || M == XY_FWD_YINTDAG);
  static constexpr bool fwd = (M == XY_FWD || M == XY_FWD_YINTDAG || M == XY_INV_Y_FWD || M == XY_INV_PC_FWD);
};

template <typename R> struct XYArgs {
  const cplx<R>* A_in;   // momentum-space input (inverse passes)
  cplx<R>* A_out;        // momentum-space output (forward passes)
  const cplx<R>* psi;    // position-space operand of the site term
  const cplx<R>* psi2;   // + shift * psi2 (XY_INV_YDAG, XY_INV_ADD), may be null
  cplx<R>* v_out;        // position-space result of phase B
  const cplx<R>* phi;    // scalar fields [member][T][Z][Y][X]
  const SiteCoef<R>* kArr;  // couplings per member
  int rpm;               // right-hand sides per member
  R shift;
  int nplanes;           // nrhs * T * Z
  int TZ;                // planes per right-hand side
  int Z;                 // planes per time slice (plane = t * Z + z)
  const R* twc;          // cos(pi t / T): antiperiodic twist, applied in position space
  const R* tws;          // sin(pi t / T)
  int* fail;             // set to WZ_ETIMEOUT if a staged copy did not complete (may be null)
  unsigned long long* blk_count;  // probe: byte counter (may be null)
  unsigned long long probe_inc;   // probe: algorithmic bytes one block moves
};

// Threads per plane: 4 * L (one per (line, spin)); PPC planes per block, the
// largest count with at most WZ_XY_MAX_THREADS threads and whole warps (block
// reductions shuffle over full warps).
#ifndef WZ_XY_MAX_THREADS
#define WZ_XY_MAX_THREADS 128
#endif
constexpr int xy_ppc(int tpp) {
  int k0 = 1;  // fewest planes that make whole warps
  while ((k0 * tpp) % 32) ++k0;
  int best = k0;
  for (int k = k0; k * tpp <= WZ_XY_MAX_THREADS; k += k0) best = k;
  return best;
}
template <int L> struct XYShape {
  static constexpr int TPP = 4 * L;
  static constexpr int PPC = xy_ppc(TPP);
  static constexpr int THREADS = TPP * PPC;
  static constexpr int RP = 4 * (L + 1);  // smem row pitch (complex), one site of padding
  static constexpr int PLANE = L * RP;
  static_assert(THREADS % 32 == 0, "xy block must be whole warps");
};

// Phase helpers shared by the xy kernels.  A thread owns (line w, spin s) of
// the plane P in shared memory (row pitch RP, one site of padding per row).
template <typename R, int L> struct XYPhase {
  using S = XYShape<L>;
  // phase A: inverse FFT along x of momentum row p_y = w (global), result into P.
  // Momentum-space planes are stored xy-transposed, [p_x][p_y][spin], so that
  // the lanes of a warp (consecutive p_y, spin) read one contiguous run.
  static __device__ __forceinline__ void inv_x(const cplx<R>* Ap, cplx<R>* P, int w, int s, cplx<R> (&v)[L]) {
#pragma unroll
    for (int x = 0; x < L; ++x) v[x] = Ap[(x * L + w) * 4 + s];
    fft_line<L, +1, R>(v);
#pragma unroll
    for (int x = 0; x < L; ++x) P[w * S::RP + x * 4 + s] = v[x];
  }
  // phase B entry: column x = w of P, inverse FFT along y -> position space
  static __device__ __forceinline__ void inv_y(const cplx<R>* P, int w, int s, cplx<R> (&v)[L]) {
#pragma unroll
    for (int y = 0; y < L; ++y) v[y] = P[y * S::RP + w * 4 + s];
    fft_line<L, +1, R>(v);
  }
  // phase B exit: forward FFT along y, column x = w back into P (the same
  // cells inv_y of this thread read, so no barrier is needed before it)
  static __device__ __forceinline__ void fwd_y(cplx<R> (&v)[L], cplx<R>* P, int w, int s) {
    fft_line<L, -1, R>(v);
#pragma unroll
    for (int y = 0; y < L; ++y) P[y * S::RP + w * 4 + s] = v[y];
  }
  // phase C: row p_y = w of P, forward FFT along x, store momentum output
  // (xy-transposed, see inv_x)
  static __device__ __forceinline__ void fwd_x(const cplx<R>* P, cplx<R>* Ap, int w, int s, cplx<R> (&v)[L]) {
#pragma unroll
    for (int x = 0; x < L; ++x) v[x] = P[w * S::RP + x * 4 + s];
    fft_line<L, -1, R>(v);
#pragma unroll
    for (int x = 0; x < L; ++x) Ap[(x * L + w) * 4 + s] = v[x];
  }
};

// Shared memory of xy_pass: the plane workspace; with STAGE (FP32, extents up
// to 32, 16-byte aligned operands) also one buffer of PPC planes for psi, the
// phi planes and an mbarrier.  A_in is staged into the workspace (consumed by
// phase A before the workspace is rewritten), psi and phi into their buffers,
// all by bulk copies issued at block entry; psi2 (a shift term) is read directly.
template <typename R, int L, int MODE, bool STAGE> struct XYSmem {
  using S = XYShape<L>;
  using I = XYModeInfo<MODE>;
  static constexpr bool USES_PSI = MODE != XY_INV;
  static constexpr bool USES_PHI = !(MODE == XY_FWD || MODE == XY_INV || MODE == XY_INV_ADD);
  static constexpr int PLANE_ELEMS = L * L * 4;
  static constexpr size_t plane_bytes = sizeof(cplx<R>) * PLANE_ELEMS;
  static constexpr size_t phi_plane_bytes = sizeof(cplx<R>) * L * L;
  static constexpr size_t work = sizeof(cplx<R>) * S::PLANE * S::PPC;
  static constexpr size_t psi_off = (work + 127) & ~size_t(127);
  static constexpr size_t phi_off = psi_off + (USES_PSI ? S::PPC * plane_bytes : 0);
  static constexpr size_t bar_off = (phi_off + (USES_PHI ? S::PPC * phi_plane_bytes : 0) + 15) & ~size_t(15);
  static constexpr size_t total = STAGE ? bar_off + 16 : work;
  static_assert(plane_bytes % 16 == 0 && phi_plane_bytes % 16 == 0, "bulk copies move multiples of 16 bytes");
};

template <typename R, int L, int MODE, bool STAGE>
__global__ void __launch_bounds__(XYShape<L>::THREADS)
xy_pass(XYArgs<R> a) {
  using S = XYShape<L>;
  using I = XYModeInfo<MODE>;
  using XS = XYSmem<R, L, MODE, STAGE>;
  constexpr int PE = XS::PLANE_ELEMS;
  extern __shared__ unsigned char smem_raw[];
  cplx<R>* sm = reinterpret_cast<cplx<R>*>(smem_raw);
  const cplx<R>* spsi = reinterpret_cast<const cplx<R>*>(smem_raw + XS::psi_off);  // [PPC][PE]
  const cplx<R>* sphi = reinterpret_cast<const cplx<R>*>(smem_raw + XS::phi_off);  // [PPC][L * L]
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw + XS::bar_off);

  const int tid = threadIdx.x;
  const int pl_local = tid / S::TPP;
  const int w = (tid / 4) % L;  // line coordinate (y in phase A/C, x in phase B)
  const int s = tid & 3;
  const long plane = (long)blockIdx.x * S::PPC + pl_local;
  const bool live = plane < a.nplanes;
  cplx<R>* P = sm + pl_local * S::PLANE;
  const long base = plane * (long)(L * L) * 4;  // complex offset of the plane
  if (a.blk_count && tid == 0) atomicAdd(a.blk_count, a.probe_inc);

  if constexpr (STAGE) {
    // the host launches this form only for 16-byte aligned operands and
    // right-hand sides of whole blocks of planes (TZ % PPC == 0)
    if (tid == 0) {
      mbar_init(bar, 1);
      mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0) {
      const long p0 = (long)blockIdx.x * S::PPC;
      const long nlive = (a.nplanes - p0) < S::PPC ? (a.nplanes - p0) : S::PPC;
      const unsigned nb = (unsigned)(nlive * XS::plane_bytes);
      const unsigned nphi = XS::USES_PHI ? (unsigned)(nlive * XS::phi_plane_bytes) : 0u;
      mbar_arrive_expect_tx(bar, (I::inv ? nb : 0u) + (XS::USES_PSI ? nb : 0u) + nphi);
      if constexpr (I::inv) bulk_g2s(sm, a.A_in + p0 * PE, nb, bar);
      if constexpr (XS::USES_PSI) bulk_g2s(smem_raw + XS::psi_off, a.psi + p0 * PE, nb, bar);
      if constexpr (XS::USES_PHI) {
        const long member = (p0 / a.TZ) / a.rpm;
        bulk_g2s(smem_raw + XS::phi_off, a.phi + (member * a.TZ + p0 % a.TZ) * (L * L), nphi, bar);
      }
    }
    if (__syncthreads_or(!mbar_wait_bounded(bar, 0))) {
      if (tid == 0 && a.fail) *a.fail = WZ_ETIMEOUT;
      mbar_wait_bounded(bar, 0);
      return;
    }
  }

  cplx<R> v[L];

  // ---------------- phase A: inverse FFT along x of the momentum input
  if (I::inv) {
    if constexpr (STAGE) {
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
      if (live) XYPhase<R, L>::inv_x(a.A_in + base, P, w, s, v);
    }
    __syncthreads();
  }

  // ---------------- phase B: y-line at fixed x = w, spin s, in position space
  if (live) {
    const int x = w;
    const long site0 = plane * (long)(L * L) + x;  // site index of (x, y=0)
    const int member = (int)(plane / a.TZ) / a.rpm;
    const long phib = ((long)member * a.TZ + plane % a.TZ) * (long)(L * L) + x;
    const SiteCoef<R> kc = a.kArr[member];
    // antiperiodic time: the field is multiplied by exp(-i pi t/T) before the
    // forward transform and by exp(+i pi t/T) after the inverse one, so that
    // the plain DFT over t lands on p_t = pi (2n + 1)/T (Sec. 3.1)
    const int tt = (int)((plane % a.TZ) / a.Z);
    const cplx<R> twb{a.twc[tt], a.tws[tt]}, twf{a.twc[tt], -a.tws[tt]};
    if (I::inv) {
#pragma unroll
      for (int y = 0; y < L; ++y) v[y] = P[y * S::RP + x * 4 + s];
      fft_line<L, +1, R>(v);
#pragma unroll
      for (int y = 0; y < L; ++y) v[y] = twb * v[y];
    }
#pragma unroll
    for (int y = 0; y < L; ++y) {
      const long e = (site0 + y * L) * 4 + s;
      const int el = pl_local * PE + (y * L + x) * 4 + s;  // staged copies
      cplx<R> ps{R(0), R(0)}, f{R(0), R(0)};
      if constexpr (XS::USES_PSI) ps = STAGE ? spsi[el] : a.psi[e];
      if constexpr (XS::USES_PHI) f = STAGE ? sphi[pl_local * (L * L) + y * L + x] : a.phi[phib + y * L];
      if constexpr (MODE == XY_FWD) {
        v[y] = ps;
      } else if constexpr (MODE == XY_FWD_YINTDAG) {
        v[y] = site_coef<R, true, false>(kc, f, s) * ps;
      } else if constexpr (MODE == XY_INV_Y || MODE == XY_INV_Y_FWD) {
        v[y] = v[y] + site_coef<R, false, true>(kc, f, s) * ps;
      } else if constexpr (MODE == XY_INV_YDAG) {
        v[y] = v[y] + site_coef<R, true, true>(kc, f, s) * ps;
        if (a.psi2) v[y] = v[y] + a.shift * a.psi2[e];
      } else if constexpr (MODE == XY_INV_PC || MODE == XY_INV_PC_FWD) {
        v[y] = ps + site_coef<R, false, false>(kc, f, s) * v[y];
      } else if constexpr (MODE == XY_INV_ADD) {
        v[y] = ps + v[y];
        if (a.psi2) v[y] = v[y] + a.shift * a.psi2[e];
      }
      if constexpr (MODE != XY_FWD && MODE != XY_FWD_YINTDAG) {
        if (a.v_out) a.v_out[e] = v[y];
      }
      if constexpr (MODE == XY_INV_PC_FWD) {
        v[y] = site_coef<R, true, false>(kc, f, s) * v[y];
      }
    }
    if (I::fwd) {
#pragma unroll
      for (int y = 0; y < L; ++y) v[y] = twf * v[y];
      fft_line<L, -1, R>(v);
    }
  }
  if (!I::fwd) return;
  // phase B of thread (x, s) rewrites exactly the smem cells it read, so no
  // barrier is needed between its reads and these writes (the staged A_in of
  // an inverse-forward mode was consumed before the barrier of phase A)
  if (live) {
#pragma unroll
    for (int y = 0; y < L; ++y) P[y * S::RP + w * 4 + s] = v[y];
  }
  __syncthreads();

  // ---------------- phase C: forward FFT along x, store momentum output
  if (live) XYPhase<R, L>::fwd_x(P, a.A_out + base, w, s, v);
}

// ----------------------------------------------------------------------------- zt pass
enum ZTMul {
  ZT_DSLASH = 0,   // out = sign * i h gamma.sin p  in
  ZT_M0INV,        // out = (-Dslash + m^* P_+ + m P_-) / den  in
  ZT_M0INV_DAG,    // out = ( Dslash + m P_+ + m^* P_-) / den  in
  ZT_SCALAR,       // periodic scalar pair packed in spin slots: slot 0 *= D2(p), slot 1 *= K(p)
  ZT_GRAD,         // periodic scalar copied into the four slots: slot mu *= i sin p_mu / omega(p)
                   // (the components of D1 acting on a scalar field; table in hV = 1/(omega V))
  ZT_OVERLAP,      // out = (D2(p) + i gamma.sin p / omega(p)) in: the overlap D = D1 + D2 (Sec. 2.2);
                   // tables in hV = 1/(omega V) and dV = D2/V
};

template <typename R> struct ZTArgs {
  cplx<R>* A;          // in/out, momentum in (x, y), position in (z, t)
  const R* hV;         // h(p) / V
  const R* hdV;        // h(p) / (den(p) V)
  const R* dV;         // 1 / (den(p) V)
  const R* d2sV;       // D2(p) / V on the periodic grid (ZT_SCALAR)
  const R* ksV;        // K(p) / V = (1 - D2(p)/2) / V on the periodic grid (ZT_SCALAR)
  const R* sinT;       // sin p_t  (antiperiodic momenta), length T
  const R* sinZ;
  const R* sinY;
  const R* sinX;
  const R* twc;        // cos(pi t / T)
  const R* tws;        // sin(pi t / T)
  R sign;              // +1 or -1 for ZT_DSLASH
  R m_re, m_im;
  int ntiles;          // ceil(XY / C)
  int X, XY;
  const int* gate;     // optional per-RHS run flag: tiles of rhs are skipped if gate[rhs * gate_stride] == 0
  int gate_stride;
  int* fail;           // WZ_ETIMEOUT (copy wait ran out) or WZ_ECUDA (misaligned tile) at fail[rhs * fail_stride]
  int fail_stride;
  int rhs0;            // first right-hand side of this launch (launches may cover a group of RHS)
  int ntot;            // tiles of this launch: (right-hand sides of the launch) x ntiles (set by the launcher)
  unsigned long long* blk_count;  // probe: byte counter (may be null)
  unsigned long long probe_inc;   // probe: algorithmic bytes one tile moves
  int pdl;             // host side: launch with programmatic stream serialization
  int tpb;             // host side: tiles per block at least (0: as many blocks as are resident)
};

// Columns per tile: C0 columns (8 C0 B FP32 / 16 C0 B FP64 contiguous per
// (z, t) row) for lines up to 16; one column for 32-point lines, whose tiles
// are 32 KB (FP32) already and whose threads need the registers of a
// 32-point line.
#ifndef WZ_ZT_C0
#define WZ_ZT_C0 4
#endif
template <typename R, int NMAX> struct ZTTile {
  static constexpr int C = NMAX <= 16 ? WZ_ZT_C0 : 1;
};

// Spin components per thread: FP32 lines up to 16 hold the two adjacent
// spins of one chirality (16-byte shared-memory accesses, two independent
// FFT chains, half the shuffles of the spin multiply); FP64 and 32-point
// lines hold one (register budget).
template <typename R> constexpr int zt_spt(int nmax) { return (sizeof(R) == 4 && nmax <= 16) ? 2 : 1; }

// the tile's columns, doubled until the z-phase threads make whole warps
constexpr int zt_columns(int c, int nz, int tpc) { return (nz * c * tpc) % 32 ? zt_columns(2 * c, nz, tpc) : c; }

// the column count of zt_pass<R, nz, nt> (ZTShape::C), also from run-time extents
template <typename R> constexpr int zt_cols_of(int nz, int nt) {
  return zt_columns((nz > nt ? nz : nt) <= 16 ? WZ_ZT_C0 : 1, nz, 4 / zt_spt<R>(nz > nt ? nz : nt));
}

template <typename R, int NZ, int NT> struct ZTShape {
  static constexpr int NMAX = NZ > NT ? NZ : NT;
  static constexpr int SPT = zt_spt<R>(NMAX);
  static constexpr int TPC = 4 / SPT;  // threads per (line, column)
  static constexpr int C = zt_cols_of<R>(NZ, NT);
  static constexpr int THREADS = NMAX * C * TPC;
  static_assert(C == zt_columns(ZTTile<R, NMAX>::C, NZ, TPC), "column rule");
  // every warp must lie entirely inside or outside the t-phase (it shuffles)
  static_assert((NZ * C * TPC) % 32 == 0, "z extent too small for the column tile");
  // Tiles in flight per block: the FP32 passes are bound by memory and copy
  // the next tile while they transform the current one (two buffers); the
  // FP64 passes are bound by arithmetic and keep one buffer.
  static constexpr int NBUF = sizeof(R) == 4 ? 2 : 1;
  // register budget, as resident threads per SM the pass is compiled for
  // (FP32: 384 threads = 170 registers, two 16-point lines or one 32-point
  // line a thread; FP64: one block -- two blocks of 128 registers measured
  // 5% slower on the FP64 16^4 apply)
  static constexpr int RESIDENT = sizeof(R) == 8 ? THREADS : 384;
  static constexpr int MINB = RESIDENT / THREADS > 0 ? RESIDENT / THREADS : 1;
};

// Dynamic shared memory of zt_pass: NBUF buffers, each a tile [t][z][c][s]
// at a 128-byte aligned start followed by the staged table boxes, then one
// mbarrier per buffer.  The momentum tables of the multiply ([p_t][p_z][column],
// one or two of them) are staged in FP32 for lines up to 16, as a (CB, NZ, NT)
// box of CB >= C columns starting at a multiple of CB, CB columns making at
// least one 16-byte row; the FP64 and 32-point passes read them from global
// memory (L2).  The kernel has no static shared memory, which would move the
// dynamic start.
template <typename R, int NZ, int NT, int MUL> struct ZTSmem {
  using S = ZTShape<R, NZ, NT>;
  static constexpr int C = S::C;
  static constexpr unsigned tile = NZ * NT * C * 4 * sizeof(cplx<R>);
  static constexpr bool STAGE_TAB = sizeof(R) == 4 && S::NMAX <= 16;
  static constexpr int CB = (int)(C * sizeof(R)) >= 16 ? C : (int)(16 / sizeof(R));  // box columns
  static_assert(CB % C == 0, "a tile's columns must fall inside one table box");
  static constexpr int NTAB = STAGE_TAB ? ((MUL == ZT_DSLASH || MUL == ZT_GRAD) ? 1 : 2) : 0;
  static constexpr unsigned tab = NZ * NT * CB * sizeof(R);
  static constexpr unsigned tab_stride = (tab + 127) & ~127u;  // every box starts 128-byte aligned
  static constexpr unsigned tab_off = (tile + 127) & ~127u;    // within a buffer
  static constexpr unsigned buf = (tab_off + NTAB * tab_stride + 127) & ~127u;
  static constexpr unsigned bar_off = S::NBUF * buf;
  static constexpr unsigned total = bar_off + 8 * S::NBUF;
  static constexpr unsigned tx_bytes = tile + NTAB * tab;  // bytes one tile's copies deliver
};

// Forward FFT over (z, t), momentum-space multiply and inverse FFT of one tile
// in shared memory (all threads of the block; barriers inside).
// The per-axis sin p of a thread's t-phase column, loaded before the z-phase so
// that their latency is hidden behind it.
template <typename R> struct ZTSin {
  R x, y, z;
};
template <typename R, int NZ, int NT>
__device__ __forceinline__ ZTSin<R> zt_sines(const ZTArgs<R>& a, int tile) {
  using S = ZTShape<R, NZ, NT>;
  const int c = (threadIdx.x / S::TPC) % S::C;
  const int pz = threadIdx.x / (S::TPC * S::C);
  const int col_raw = tile * S::C + c;
  const int col = col_raw < a.XY ? col_raw : 0;
  const int px = col / a.X, py = col - px * a.X;  // momentum planes are xy-transposed (X == Y)
  return ZTSin<R>{__ldg(a.sinX + px), __ldg(a.sinY + py), __ldg(a.sinZ + (pz < NZ ? pz : 0))};
}

// one spin component per thread
template <typename R, int NZ, int NT, int MUL>
__device__ __forceinline__ void zt_transform1(cplx<R>* sm, const R* tab0, const R* tab1, const ZTArgs<R>& a,
                                              int tile, ZTSin<R> sn) {
  using ZS = ZTSmem<R, NZ, NT, MUL>;
  constexpr int C = ZTShape<R, NZ, NT>::C;
  const int tid = threadIdx.x;
  const int s = tid & 3;
  const int c = (tid >> 2) % C;
  const int q = tid / (4 * C);  // t in the z-phase, z in the t-phase
  const int col_raw = tile * C + c;  // (p_x, p_y) column = p_x * Y + p_y
  const int col = col_raw < a.XY ? col_raw : 0;  // table lookups of lanes past the ragged end

  cplx<R> v[NT > NZ ? NT : NZ];

  // ---------------- z-phase (forward): thread owns (t = q, column, s)
  if (q < NT) {
    const int t = q;
    // (the antiperiodic twist of the fermion is applied by the xy passes)
#pragma unroll
    for (int z = 0; z < NZ; ++z) v[z] = sm[((t * NZ + z) * C + c) * 4 + s];
    fft_ptr<NZ, -1, R>(v);
#pragma unroll
    for (int z = 0; z < NZ; ++z) sm[((t * NZ + z) * C + c) * 4 + s] = v[z];
  }
  __syncthreads();

  // ---------------- t-phase: forward over t, spin multiply, inverse over t
  if (q < NZ) {
    const int pz = q;
#pragma unroll
    for (int t = 0; t < NT; ++t) v[t] = sm[((t * NZ + pz) * C + c) * 4 + s];
    fft_ptr<NT, -1, R>(v);

    const R sx = sn.x, sy = sn.y, sz = sn.z;
    const int lane = threadIdx.x & 31;
    const int ulane = (lane & ~3) | (s < 2 ? 2 : 0);  // opposite-chirality pair
    const R sg = s < 2 ? R(1) : R(-1);
#pragma unroll
    for (int pt = 0; pt < NT; ++pt) {
      const long pidx = ((long)pt * NZ + pz) * a.XY + col;
      const int tix = (pt * NZ + pz) * ZS::CB + (tile * C) % ZS::CB + c;  // staged tables
      // sin p_t, p_t = pi (2 pt + 1) / T: a compile-time entry of the twiddle table
      static_assert(WZ_TW_N % (2 * NT) == 0, "antiperiodic momenta must lie on the twiddle grid");
      const R st = Tw<R>::cosk(((2 * pt + 1) * (WZ_TW_N / (2 * NT)) + 3 * WZ_TW_N / 4) % WZ_TW_N);
      // row of  sum_mu s_mu gamma_mu  acting on the opposite-chirality pair (u, w)
      cplx<R> cu, cw;
      if ((s & 1) == 0) {
        cu = cplx<R>{st, sg * sz};
        cw = cplx<R>{sg * sy, sg * sx};
      } else {
        cu = cplx<R>{-sg * sy, sg * sx};
        cw = cplx<R>{st, -sg * sz};
      }
      cplx<R> u, ww;
      u.x = __shfl_sync(0xffffffffu, v[pt].x, ulane);
      u.y = __shfl_sync(0xffffffffu, v[pt].y, ulane);
      ww.x = __shfl_sync(0xffffffffu, v[pt].x, ulane + 1);
      ww.y = __shfl_sync(0xffffffffu, v[pt].y, ulane + 1);
      const cplx<R> g = cu * u + cw * ww;  // (gamma . sin p  in)_s
      if constexpr (MUL == ZT_SCALAR) {
        const R sc = s == 0 ? (ZS::NTAB ? tab0[tix] : a.d2sV[pidx]) : (s == 1 ? (ZS::NTAB ? tab1[tix] : a.ksV[pidx]) : R(0));
        v[pt] = sc * v[pt];
      } else if constexpr (MUL == ZT_GRAD) {
        // periodic momenta: sin(2 pi pt / T) from the twiddle table; slot s is direction mu = s (t, x, y, z)
        static_assert(WZ_TW_N % NT == 0, "periodic momenta must lie on the twiddle grid");
        const R stp = Tw<R>::cosk((pt * (WZ_TW_N / NT) + 3 * WZ_TW_N / 4) % WZ_TW_N);
        const R smu = s == 0 ? stp : (s == 1 ? sx : (s == 2 ? sy : sz));
        v[pt] = (smu * (ZS::NTAB ? tab0[tix] : a.hV[pidx])) * mul_i(v[pt]);
      } else if constexpr (MUL == ZT_DSLASH) {
        const R hh = a.sign * (ZS::NTAB ? tab0[tix] : a.hV[pidx]);
        v[pt] = hh * mul_i(g);
      } else if constexpr (MUL == ZT_OVERLAP) {
        const R w1 = ZS::NTAB ? tab0[tix] : a.hV[pidx], d2 = ZS::NTAB ? tab1[tix] : a.dV[pidx];
        v[pt] = w1 * mul_i(g) + d2 * v[pt];
      } else {
        const R hd = ZS::NTAB ? tab0[tix] : a.hdV[pidx], dd = ZS::NTAB ? tab1[tix] : a.dV[pidx];
        // mass on the diagonal: M0^-1 has m^* on P_+ and m on P_-; the dagger swaps
        const bool mconj = (MUL == ZT_M0INV) ? (s >= 2) : (s < 2);
        const cplx<R> mm{a.m_re, mconj ? -a.m_im : a.m_im};
        const R sd = (MUL == ZT_M0INV) ? R(-1) : R(1);
        v[pt] = (sd * hd) * mul_i(g) + dd * (mm * v[pt]);
      }
    }
    fft_ptr<NT, +1, R>(v);
#pragma unroll
    for (int t = 0; t < NT; ++t) sm[((t * NZ + pz) * C + c) * 4 + s] = v[t];
  }
  __syncthreads();

  // ---------------- z-phase (inverse), back into the tile
  if (q < NT) {
    const int t = q;
#pragma unroll
    for (int z = 0; z < NZ; ++z) v[z] = sm[((t * NZ + z) * C + c) * 4 + s];
    fft_ptr<NZ, +1, R>(v);
#pragma unroll
    for (int z = 0; z < NZ; ++z) sm[((t * NZ + z) * C + c) * 4 + s] = v[z];
  }
}

// Two spin components (2h, 2h + 1: one chirality) per thread, FP32.  The
// multiply needs the other chirality's pair, which the partner thread (lane
// ^ 1) holds: two complex shuffles give both of this thread's outputs.
template <int NZ, int NT, int MUL>
__device__ __forceinline__ void zt_transform2(cplx<float>* sm, const float* tab0, const float* tab1,
                                              const ZTArgs<float>& a, int tile, ZTSin<float> sn) {
  using R = float;
  using ZS = ZTSmem<R, NZ, NT, MUL>;
  constexpr int C = ZTShape<R, NZ, NT>::C;
  const int tid = threadIdx.x;
  const int h = tid & 1;           // spin pair: components 2h, 2h + 1
  const int c = (tid >> 1) % C;
  const int q = tid / (2 * C);     // t in the z-phase, z in the t-phase
  float4* sm4 = reinterpret_cast<float4*>(sm);  // [t][z][c][h]: one spin pair per 16 bytes
  constexpr int N = NT > NZ ? NT : NZ;
  cplx<R> v0[N], v1[N];

  // ---------------- z-phase (forward): thread owns (t = q, column, pair)
  if (q < NT) {
    const int t = q;
#pragma unroll
    for (int z = 0; z < NZ; ++z) {
      const float4 f = sm4[((t * NZ + z) * C + c) * 2 + h];
      v0[z] = cplx<R>{f.x, f.y};
      v1[z] = cplx<R>{f.z, f.w};
    }
    fft_ptr<NZ, -1, R>(v0);
    fft_ptr<NZ, -1, R>(v1);
#pragma unroll
    for (int z = 0; z < NZ; ++z) sm4[((t * NZ + z) * C + c) * 2 + h] = make_float4(v0[z].x, v0[z].y, v1[z].x, v1[z].y);
  }
  __syncthreads();

  // ---------------- t-phase: forward over t, spin multiply, inverse over t
  if (q < NZ) {
    const int pz = q;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const float4 f = sm4[((t * NZ + pz) * C + c) * 2 + h];
      v0[t] = cplx<R>{f.x, f.y};
      v1[t] = cplx<R>{f.z, f.w};
    }
    fft_ptr<NT, -1, R>(v0);
    fft_ptr<NT, -1, R>(v1);

    const R sx = sn.x, sy = sn.y, sz = sn.z;
    const int partner = (threadIdx.x & 31) ^ 1;
    const R sg = h == 0 ? R(1) : R(-1);  // +1 on P_- (spins 0, 1), -1 on P_+ (spins 2, 3)
    const cplx<R> ue{R(0), sg * sz}, we{sg * sy, sg * sx};      // even spin: (st + i sg sz) u + (sg sy + i sg sx) w
    const cplx<R> uo{-sg * sy, sg * sx}, wo{R(0), -sg * sz};    // odd spin: (-sg sy + i sg sx) u + (st - i sg sz) w
#pragma unroll
    for (int pt = 0; pt < NT; ++pt) {
      const int tix = (pt * NZ + pz) * ZS::CB + (tile * C) % ZS::CB + c;  // staged tables
      static_assert(WZ_TW_N % (2 * NT) == 0, "antiperiodic momenta must lie on the twiddle grid");
      const R st = Tw<R>::cosk(((2 * pt + 1) * (WZ_TW_N / (2 * NT)) + 3 * WZ_TW_N / 4) % WZ_TW_N);
      if constexpr (MUL == ZT_SCALAR) {
        // slot 0 *= D2(p), slot 1 *= K(p), slots 2, 3 = 0 (periodic scalar pair)
        v0[pt] = (h == 0 ? tab0[tix] : R(0)) * v0[pt];
        v1[pt] = (h == 0 ? tab1[tix] : R(0)) * v1[pt];
      } else if constexpr (MUL == ZT_GRAD) {
        static_assert(WZ_TW_N % NT == 0, "periodic momenta must lie on the twiddle grid");
        const R stp = Tw<R>::cosk((pt * (WZ_TW_N / NT) + 3 * WZ_TW_N / 4) % WZ_TW_N);
        const R w1 = tab0[tix];
        v0[pt] = ((h == 0 ? stp : sy) * w1) * mul_i(v0[pt]);  // slots 0 (t) / 2 (y)
        v1[pt] = ((h == 0 ? sx : sz) * w1) * mul_i(v1[pt]);   // slots 1 (x) / 3 (z)
      } else {
        cplx<R> u, w;  // the other chirality's pair (even, odd) at this momentum
        u.x = __shfl_sync(0xffffffffu, v0[pt].x, partner);
        u.y = __shfl_sync(0xffffffffu, v0[pt].y, partner);
        w.x = __shfl_sync(0xffffffffu, v1[pt].x, partner);
        w.y = __shfl_sync(0xffffffffu, v1[pt].y, partner);
        const cplx<R> ge = cplx<R>{st, ue.y} * u + we * w;  // (gamma . sin p  in) of the even spin
        const cplx<R> go = uo * u + cplx<R>{st, wo.y} * w;  // ... of the odd spin
        if constexpr (MUL == ZT_DSLASH) {
          const R hh = a.sign * tab0[tix];
          v0[pt] = hh * mul_i(ge);
          v1[pt] = hh * mul_i(go);
        } else if constexpr (MUL == ZT_OVERLAP) {
          const R w1 = tab0[tix], d2 = tab1[tix];
          v0[pt] = w1 * mul_i(ge) + d2 * v0[pt];
          v1[pt] = w1 * mul_i(go) + d2 * v1[pt];
        } else {
          const R hd = tab0[tix], dd = tab1[tix];
          // mass on the diagonal: M0^-1 has m^* on P_+ and m on P_-; the dagger swaps
          const bool mconj = (MUL == ZT_M0INV) ? (h == 1) : (h == 0);
          const cplx<R> mm{a.m_re, mconj ? -a.m_im : a.m_im};
          const R sd = (MUL == ZT_M0INV) ? R(-1) : R(1);
          v0[pt] = (sd * hd) * mul_i(ge) + dd * (mm * v0[pt]);
          v1[pt] = (sd * hd) * mul_i(go) + dd * (mm * v1[pt]);
        }
      }
    }
    fft_ptr<NT, +1, R>(v0);
    fft_ptr<NT, +1, R>(v1);
#pragma unroll
    for (int t = 0; t < NT; ++t) sm4[((t * NZ + pz) * C + c) * 2 + h] = make_float4(v0[t].x, v0[t].y, v1[t].x, v1[t].y);
  }
  __syncthreads();

  // ---------------- z-phase (inverse), back into the tile
  if (q < NT) {
    const int t = q;
#pragma unroll
    for (int z = 0; z < NZ; ++z) {
      const float4 f = sm4[((t * NZ + z) * C + c) * 2 + h];
      v0[z] = cplx<R>{f.x, f.y};
      v1[z] = cplx<R>{f.z, f.w};
    }
    fft_ptr<NZ, +1, R>(v0);
    fft_ptr<NZ, +1, R>(v1);
#pragma unroll
    for (int z = 0; z < NZ; ++z) sm4[((t * NZ + z) * C + c) * 2 + h] = make_float4(v0[z].x, v0[z].y, v1[z].x, v1[z].y);
  }
}

template <typename R, int NZ, int NT, int MUL>
__device__ __forceinline__ void zt_transform(cplx<R>* sm, const R* tab0, const R* tab1, const ZTArgs<R>& a,
                                             int tile, ZTSin<R> sn) {
  if constexpr (ZTShape<R, NZ, NT>::SPT == 2) {
    static_assert(sizeof(R) == 4 && ZTSmem<R, NZ, NT, MUL>::NTAB > 0, "two spins a thread: FP32, staged tables");
    zt_transform2<NZ, NT, MUL>(sm, tab0, tab1, a, tile, sn);
  } else {
    zt_transform1<R, NZ, NT, MUL>(sm, tab0, tab1, a, tile, sn);
  }
}

// Persistent zt pass.  A tile is C consecutive (p_x, p_y) columns of one
// right-hand side for all (z, t); the launch covers a.ntot tiles (its
// right-hand sides times a.ntiles) and block b takes tiles b, b + G, b + 2G,
// ... (G blocks), skipping the tiles of right-hand sides that are gated off.
// A tile [t][z][c][s] arrives in shared memory by one 3D tensor copy (TMA)
// plus its table boxes, is transformed in place, and leaves by one tensor
// store.  With two buffers the copy of the block's next tile is issued before
// the current one is transformed, into the buffer whose store has been read
// out, so loads, transforms and stores of successive tiles overlap.  Ragged
// last tiles: the copy fills columns past X * Y with zeros, the store clips
// them.  Every wait is bounded; a wait that runs out marks the right-hand
// side failed, lets the copies in flight land (bounded) and ends the block.
template <typename R, int NZ, int NT, int MUL>
__global__ void __launch_bounds__(ZTShape<R, NZ, NT>::THREADS, ZTShape<R, NZ, NT>::MINB)
zt_pass(ZTArgs<R> a, const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmT0,
        const __grid_constant__ CUtensorMap tmT1) {
  using S = ZTShape<R, NZ, NT>;
  using ZS = ZTSmem<R, NZ, NT, MUL>;
  constexpr int C = S::C;
  constexpr int NBUF = S::NBUF;
  constexpr int U = sizeof(cplx<R>) / 8;  // 8-byte tensor elements per complex value
  extern __shared__ unsigned char smem_raw[];
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem_raw + ZS::bar_off);
  const int tid = threadIdx.x;
  const int G = gridDim.x;
  pdl_wait();  // the gates and the tiles are the predecessor's output
  pdl_trigger();

  // the next tile of this block at or after q whose right-hand side runs
  // (the gates are not written while the pass runs: every thread agrees)
  auto next_live = [&](int q) {
    if (a.gate)
      while (q < a.ntot && !a.gate[(long)(q / a.ntiles + a.rhs0) * a.gate_stride]) q += G;
    return q;
  };
  int q = next_live(blockIdx.x);
  if (q >= a.ntot) return;  // whole block, before any barrier

  // tensor copies need 128-byte aligned shared-memory tiles: checked, the
  // block records the failure and leaves without any copy if they are not
  if (__syncthreads_or((smem_u32(smem_raw) & 127u) != 0)) {
    if (tid == 0 && a.fail) a.fail[(long)(q / a.ntiles + a.rhs0) * a.fail_stride] = WZ_ECUDA;
    return;
  }
  if (tid == 0) {
#pragma unroll
    for (int b = 0; b < NBUF; ++b) mbar_init(&bars[b], 1);
    mbar_fence_init();
  }
  __syncthreads();
  // thread 0: copies of tile qq (tile and table boxes) into buffer b
  auto issue = [&](int qq, int b) {
    const int rhs = qq / a.ntiles + a.rhs0, tile = qq % a.ntiles;
    unsigned char* buf = smem_raw + b * ZS::buf;
    mbar_arrive_expect_tx(&bars[b], ZS::tx_bytes);
    tma_load_3d(buf, &tmA, tile * C * 4 * U, 0, rhs * NT, &bars[b]);
    const int tx0 = (tile * C / ZS::CB) * ZS::CB;  // table box start (multiple of CB columns)
    if constexpr (ZS::NTAB >= 1) tma_load_3d(buf + ZS::tab_off, &tmT0, tx0, 0, 0, &bars[b]);
    if constexpr (ZS::NTAB >= 2) tma_load_3d(buf + ZS::tab_off + ZS::tab_stride, &tmT1, tx0, 0, 0, &bars[b]);
  };
  if (tid == 0) issue(q, 0);

  unsigned long long ntile = 0;
  int qn = next_live(q + G);
  for (int j = 0; q < a.ntot; ++j) {
    const int b = j % NBUF;
    const unsigned parity = (unsigned)(j / NBUF) & 1u;  // uses of barrier b so far, mod 2
    const int rhs = q / a.ntiles + a.rhs0, tile = q % a.ntiles;
    const ZTSin<R> sn = zt_sines<R, NZ, NT>(a, tile);
    if constexpr (NBUF == 2) {
      // the other buffer held the previous tile: once its store has read it
      // out, it takes the copy of the next tile
      if (tid == 0 && qn < a.ntot) {
        bulk_wait_read_all();
        issue(qn, b ^ 1);
      }
    }
    if (__syncthreads_or(!mbar_wait_bounded(&bars[b], parity))) {
      if (tid == 0) {
        if (a.fail) a.fail[(long)rhs * a.fail_stride] = WZ_ETIMEOUT;
        if (NBUF == 2 && qn < a.ntot) mbar_wait_bounded(&bars[b ^ 1], (unsigned)((j + 1) / NBUF) & 1u);
        mbar_wait_bounded(&bars[b], parity);
        bulk_wait_read_all();
      }
      return;
    }
    unsigned char* buf = smem_raw + b * ZS::buf;
    // the tile after next: its gate is read while this tile is transformed
    const int qnn = qn < a.ntot ? next_live(qn + G) : qn;
    zt_transform<R, NZ, NT, MUL>(reinterpret_cast<cplx<R>*>(buf), reinterpret_cast<const R*>(buf + ZS::tab_off),
                                 reinterpret_cast<const R*>(buf + ZS::tab_off + ZS::tab_stride), a, tile, sn);
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tma_store_3d(&tmA, tile * C * 4 * U, 0, rhs * NT, buf);
      bulk_commit();
      if constexpr (NBUF == 1) {
        if (qn < a.ntot) {
          bulk_wait_read_all();
          issue(qn, 0);
        }
      }
    }
    ++ntile;
    q = qn;
    qn = qnn;
  }
  if (tid == 0) {
    bulk_wait_read_all();  // the shared memory must outlive the last store's read
    if (a.blk_count) atomicAdd(a.blk_count, ntile * a.probe_inc);
  }
}

}  // namespace wz
