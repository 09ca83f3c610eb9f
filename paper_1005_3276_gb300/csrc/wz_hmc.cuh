// Forces, actions and HMC field updates (Eq. acws, Secs. 7.2 and 7.4).
//
//   S_B   = sum_x [ 2 phi^* (D2 phi) + W'^* (K W') ],  W' = m phi + g phi^2,
//           K = 1 - D2/2, scalars periodic in every direction          (Eq. acws)
//   S_pf  = sum_k eta_k^dag (M^dag M)^-1 eta_k   (single pole of Eq. jkjk)
//   G     = dS/dphi_R + i dS/dphi_I
//   G_B   = 4 (D2 phi) + 2 conj(m + 2 g phi) (K W')
//   G_pf  = -2 Re[Z^dag dM/dphi_R X] - 2i Re[Z^dag dM/dphi_I X],  X = (M^dag M)^-1 eta, Z = M X
//           dM/dphi_R = c g P_+ + c g^* P_-,  dM/dphi_I = i c g P_+ - i c g^* P_-
//
// Kernels (FP64; all site-local work is fused into the last xy pass):
//   xy_force      inverse xy of F(M X without the site term), Z = . + Y X, the
//                 site contraction above for one pseudofermion per plane -> G_k
//   xy_boson_fwd  forward xy of the packed scalar field [phi, W', 0, 0]
//   xy_boson_inv  inverse xy of [D2 phi, K W', ., .] (zt pass ZT_SCALAR), G_B,
//                 + sum_k G_k in fixed order, partial S_B per block
// plus Philox draws and the field updates of the molecular dynamics.
#pragma once
#include "wz_cg.cuh"

namespace wz {

// r(x) = a0 + sum_i alpha_i / (x + beta_i) applied to systems laid out
// [member][pole][rhs] (inner = rhs per member): the weights of a rational
// action's force and the combination a0 in + sum_i alpha_i X_i (Eq. jkjk).
// d = 0 marks the single-pole action (weight 1, no combination).
struct PoleSum {
  int d = 0;
  int inner = 1;
  double a0 = 0.0;
  double alpha[WZ_SHIFT_MAX] = {0.0};
  __host__ __device__ double weight(int q) const { return d ? alpha[(q / inner) % d] : 1.0; }
};

template <typename R> struct ForceArgs {
  const cplx<R>* A;       // momentum intermediate (input of the inverse passes)
  cplx<R>* A_out;         // xy_boson_fwd output
  const cplx<R>* X;       // xy_force: solutions X_k [npf][T][Z][Y][X][4]
  cplx<R>* Gk;            // xy_force: per-pseudofermion forces [npf][V]
  const cplx<R>* Gk_in;   // xy_boson_inv: forces to add, [npf][V] (may be null)
  int npf;
  cplx<R>* G;             // xy_boson_inv: total force [V] (may be null)
  double* part;           // xy_boson_inv: block partials of S_B
  const cplx<R>* phi;     // [member][V]
  const SiteCoef<R>* kArr;  // couplings per member
  int rpm;                // pseudofermions per member (xy_force)
  int Z;                  // planes per time slice
  const R* twc;           // antiperiodic twist cos / sin (pi t / T) (xy_force)
  const R* tws;
  int TZ;
  int nblk;
  long V;
  PoleSum pw;             // xy_force: per-system weight alpha_i of the rational action
};

template <typename R>
__device__ __forceinline__ R quad_sum(R v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  return v;
}

// grid (nblk, npf); one pseudofermion per grid row
template <int L>
__global__ void __launch_bounds__(XYShape<L>::THREADS) xy_force(ForceArgs<double> a) {
  using R = double;
  using S = XYShape<L>;
  using H = XYPhase<R, L>;
  extern __shared__ unsigned char smem_raw[];
  cplx<R>* sm = reinterpret_cast<cplx<R>*>(smem_raw);
  const int k = blockIdx.y;
  const int tid = threadIdx.x, pl_local = tid / S::TPP, w = (tid / 4) % L, s = tid & 3;
  const int plane_in = blockIdx.x * S::PPC + pl_local;
  const bool live = plane_in < a.TZ;
  const long plane = (long)k * a.TZ + plane_in;
  cplx<R>* P = sm + pl_local * S::PLANE;
  const long base = plane * (long)(L * L) * 4;
  cplx<R> v[L];
  if (live) H::inv_x(a.A + base, P, w, s, v);
  __syncthreads();
  if (live) {
    H::inv_y(P, w, s, v);
    const int tt = plane_in / a.Z;
    const cplx<R> twb{a.twc[tt], a.tws[tt]};
#pragma unroll
    for (int y = 0; y < L; ++y) v[y] = twb * v[y];
  }
  const int member = k / a.rpm;
  const SiteCoef<R> kc = a.kArr[member];
  const cplx<R> cg{kc.cg_re, kc.cg_im};
  const R wk = a.pw.weight(k);
  // chirality weight: spins 2,3 (P_+) carry c g, spins 0,1 (P_-) carry c g^*
  const cplx<R> wgt = s >= 2 ? cg : conj(cg);
  const R sgn = s >= 2 ? R(1) : R(-1);
#pragma unroll
  for (int y = 0; y < L; ++y) {
    R dr = 0, di = 0;
    const long site = (long)plane_in * (L * L) + y * L + w;  // within one field
    if (live) {
      const long e = (plane * (long)(L * L) + y * L + w) * 4 + s;
      const cplx<R> x = a.X[e];
      const cplx<R> f = a.phi[member * a.V + site];
      const cplx<R> z = v[y] + site_coef<R, false, true>(kc, f, s) * x;  // Z = M X
      const cplx<R> zx = conj(z) * x;
      const cplx<R> t = wgt * zx;
      dr = -R(2) * wk * t.x;        // -2 Re[w Z^* X]
      di = R(2) * wk * sgn * t.y;   // -2 Re[+-i w Z^* X] = +-2 Im[w Z^* X]
    }
    dr = quad_sum(dr);
    di = quad_sum(di);
    if (live && s == 0) a.Gk[(long)k * a.V + site] = cplx<R>{dr, di};
  }
}

// 1D grid over the T*Z planes of the packed scalar field
template <int L>
__global__ void __launch_bounds__(XYShape<L>::THREADS) xy_boson_fwd(ForceArgs<double> a) {
  using R = double;
  using S = XYShape<L>;
  using H = XYPhase<R, L>;
  extern __shared__ unsigned char smem_raw[];
  cplx<R>* sm = reinterpret_cast<cplx<R>*>(smem_raw);
  const int tid = threadIdx.x, pl_local = tid / S::TPP, w = (tid / 4) % L, s = tid & 3;
  const int member = blockIdx.y;
  const int plane_in = blockIdx.x * S::PPC + pl_local;
  const bool live = plane_in < a.TZ;
  cplx<R>* P = sm + pl_local * S::PLANE;
  const long base = ((long)member * a.TZ + plane_in) * (L * L) * 4;
  const SiteCoef<R> kc = a.kArr[member];
  cplx<R> v[L];
  if (live) {
#pragma unroll
    for (int y = 0; y < L; ++y) {
      const cplx<R> f = a.phi[member * a.V + (long)plane_in * (L * L) + y * L + w];
      if (s == 0) v[y] = f;
      else if (s == 1) v[y] = cplx<R>{kc.m_re, kc.m_im} * f + cplx<R>{kc.g_re, kc.g_im} * (f * f);
      else v[y] = cplx<R>{0, 0};
    }
    H::fwd_y(v, P, w, s);
  }
  __syncthreads();
  if (live) H::fwd_x(P, a.A_out + base, w, s, v);
}

template <int L>
__global__ void __launch_bounds__(XYShape<L>::THREADS) xy_boson_inv(ForceArgs<double> a) {
  using R = double;
  using S = XYShape<L>;
  using H = XYPhase<R, L>;
  extern __shared__ unsigned char smem_raw[];
  cplx<R>* sm = reinterpret_cast<cplx<R>*>(smem_raw);
  double* red = reinterpret_cast<double*>(sm + S::PLANE * S::PPC);
  const int tid = threadIdx.x, pl_local = tid / S::TPP, w = (tid / 4) % L, s = tid & 3;
  const int lane = tid & 31;
  const int member = blockIdx.y;
  const int plane_in = blockIdx.x * S::PPC + pl_local;
  const bool live = plane_in < a.TZ;
  cplx<R>* P = sm + pl_local * S::PLANE;
  const long base = ((long)member * a.TZ + plane_in) * (L * L) * 4;
  cplx<R> v[L];
  if (live) H::inv_x(a.A + base, P, w, s, v);
  __syncthreads();
  if (live) H::inv_y(P, w, s, v);
  double part = 0.0;
  const SiteCoef<R> kc = a.kArr[member];
  const cplx<R> m{kc.m_re, kc.m_im}, g{kc.g_re, kc.g_im};
#pragma unroll
  for (int y = 0; y < L; ++y) {
    cplx<R> d2, kw;  // (D2 phi) from spin slot 0, (K W') from slot 1 of this site
    d2.x = __shfl_sync(0xffffffffu, v[y].x, lane & ~3);
    d2.y = __shfl_sync(0xffffffffu, v[y].y, lane & ~3);
    kw.x = __shfl_sync(0xffffffffu, v[y].x, (lane & ~3) | 1);
    kw.y = __shfl_sync(0xffffffffu, v[y].y, (lane & ~3) | 1);
    if (live && s == 0) {
      const long site = member * a.V + (long)plane_in * (L * L) + y * L + w;
      const cplx<R> f = a.phi[site];
      const cplx<R> W = m * f + g * (f * f);
      const cplx<R> dW = m + R(2) * (g * f);  // W'' = m + 2 g phi
      cplx<R> G = R(4) * d2 + R(2) * (conj(dW) * kw);
      // this member's pseudofermion forces, in a fixed order
      const long gk0 = (long)member * a.npf * a.V + (site - member * a.V);
      for (int j = 0; j < a.npf; ++j) G = G + a.Gk_in[gk0 + (long)j * a.V];
      if (a.G) a.G[site] = G;
      part += R(2) * re_conj_mul(d2, f) + re_conj_mul(kw, W);  // 2 Re[phi^* D2 phi] + Re[W'^* K W']
    }
  }
  const double t = block_sum(part, red);
  if (tid == 0) a.part[(long)member * a.nblk + blockIdx.x] = t;
}

// ----------------------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11).  counter (c0..c3), key (k0, k1); 10 rounds with the published
// multipliers and Weyl increments.
struct Philox4 { unsigned int v[4]; };

__device__ __forceinline__ Philox4 philox4x32_10(unsigned int c0, unsigned int c1, unsigned int c2,
                                                 unsigned int c3, unsigned int k0, unsigned int k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned int hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const unsigned int hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const unsigned int n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return Philox4{{c0, c1, c2, c3}};
}

// uniform in (0, 1] from a 53-bit integer (a << 21) | (b >> 11)
__device__ __forceinline__ double unit53(unsigned int a, unsigned int b) {
  const unsigned long long n = ((unsigned long long)a << 21) | (unsigned long long)(b >> 11);
  return ((double)n + 1.0) * 0x1.0p-53;
}

// Box-Muller pair from one Philox call
__device__ __forceinline__ cplx<double> gauss_pair(Philox4 w) {
  const double u1 = unit53(w.v[0], w.v[1]), u2 = unit53(w.v[2], w.v[3]);
  const double rho = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  return cplx<double>{rho * cs, rho * sn};
}

enum { STREAM_MOMENTUM = 1, STREAM_PSEUDOFERMION = 2, STREAM_ACCEPT = 3 };

// A member draws with the key seed + id (id = the lattice's index in its
// batch; 0 for a single lattice), so a batch reproduces every lattice's
// draws whatever the grouping.
__device__ __forceinline__ Philox4 member_draw(unsigned long long seed, int id, unsigned c0, unsigned c1,
                                               unsigned c2, unsigned c3) {
  const unsigned long long key = seed + (unsigned long long)id;
  return philox4x32_10(c0, c1, c2, c3, (unsigned)key, (unsigned)(key >> 32));
}

// pi(x): Re, Im ~ N(0, 1); counter (site, 0, STREAM_MOMENTUM, traj); fields [member][V]
// traj: device word holding the trajectory number (the counter word c3)
static __global__ void draw_momenta(cplx<double>* pi, long V, int nm, const int* mid, unsigned long long seed,
                             const unsigned long long* trajp) {
  const unsigned traj = (unsigned)*trajp;
  const long n = (long)nm * V;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    pi[i] = gauss_pair(member_draw(seed, mid[i / V], (unsigned)(i % V), 0u, STREAM_MOMENTUM, traj));
}

// R_k(x, s): density exp(-|R|^2); counter (site, 4k + s, STREAM_PSEUDOFERMION, traj),
// k the pseudofermion within its member; fields [member][npf][V][4]
static __global__ void draw_sources(cplx<double>* R, int npf, long V, int nm, const int* mid, unsigned long long seed,
                             const unsigned long long* trajp) {
  const unsigned traj = (unsigned)*trajp;
  const long n = (long)nm * npf * V * 4;
  const double sc = 0.70710678118654752440;  // sqrt(1/2)
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int s = (int)(i & 3);
    const long site = (i >> 2) % V;
    const long kk = (i >> 2) / V;  // member * npf + k
    const int member = (int)(kk / npf), k = (int)(kk % npf);
    const cplx<double> z =
        gauss_pair(member_draw(seed, mid[member], (unsigned)site, (unsigned)(4 * k + s), STREAM_PSEUDOFERMION, traj));
    R[i] = cplx<double>{sc * z.x, sc * z.y};
  }
}

// out[m][j] = a0 in[m][j] + sum_i alpha_i X[m][i][j] (n complex values per
// field; ps.inner fields per member).  Grid (nb, members * inner).
static __global__ void pole_combine(const cplx<double>* in, const cplx<double>* X, cplx<double>* out, long n,
                                    PoleSum ps) {
  const int q = blockIdx.y;
  const int member = q / ps.inner, j = q % ps.inner;
  const cplx<double>* src = in + (long)q * n;
  const cplx<double>* xs = X + ((long)member * ps.d * ps.inner + j) * n;
  const long pstride = (long)ps.inner * n;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    cplx<double> acc = ps.a0 * src[i];
    for (int p = 0; p < ps.d; ++p) acc = acc + ps.alpha[p] * xs[p * pstride + i];
    out[(long)q * n + i] = acc;
  }
}

// partials of sum Re[conj(a) b] over n complex values per member, grid (nblk, members)
static __global__ void dot_re_partials(const cplx<double>* a, const cplx<double>* b, long n, double* part) {
  __shared__ double red[33];
  const long off = (long)blockIdx.y * n;
  double t = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    t += re_conj_mul(a[off + i], b[off + i]);
  t = block_sum(t, red);
  if (threadIdx.x == 0) part[(long)blockIdx.y * gridDim.x + blockIdx.x] = t;
}

// phi += eps * pi (FP64 and its FP32 copy)
static __global__ void update_phi(cplx<double>* phi, cplx<float>* phi32, const cplx<double>* pi, double eps, long V) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < V; i += (long)gridDim.x * blockDim.x) {
    const cplx<double> f = phi[i] + eps * pi[i];
    phi[i] = f;
    phi32[i] = cplx<float>{(float)f.x, (float)f.y};
  }
}

// pi -= eps * G
static __global__ void update_pi(cplx<double>* pi, const cplx<double>* G, double eps, long V) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < V; i += (long)gridDim.x * blockDim.x)
    pi[i] = pi[i] - eps * G[i];
}

// Metropolis on the device, one thread per member: sums that member's H
// partials in a fixed order, draws u and decides.  out[5 j ..] = [H0, H1, dH, u, accept]
struct HParts {
  const double* kin0; int nkin0;   // sum |pi|^2 at the start      ([member][n] each)
  const double* sb0; int nsb0;     // S_B at the start
  const double* spf0; int nspf0;   // sum |R|^2
  const double* kin1; int nkin1;
  const double* sb1; int nsb1;
  const double* spf1; int nspf1;   // sum Re eta^dag X at the end
};

__device__ __forceinline__ double serial_sum(const double* p, int n) {
  double t = 0.0;
  for (int i = 0; i < n; ++i) t += p[i];
  return t;
}

static __global__ void metropolis(HParts h, double* out, int nm, const int* mid, unsigned long long seed,
                           const unsigned long long* trajp) {
  const unsigned traj = (unsigned)*trajp;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nm) return;
  const double H0 = 0.5 * serial_sum(h.kin0 + (long)j * h.nkin0, h.nkin0) +
                    serial_sum(h.sb0 + (long)j * h.nsb0, h.nsb0) + serial_sum(h.spf0 + (long)j * h.nspf0, h.nspf0);
  const double H1 = 0.5 * serial_sum(h.kin1 + (long)j * h.nkin1, h.nkin1) +
                    serial_sum(h.sb1 + (long)j * h.nsb1, h.nsb1) + serial_sum(h.spf1 + (long)j * h.nspf1, h.nspf1);
  const double dH = H1 - H0;
  const Philox4 w = member_draw(seed, mid[j], 0u, 0u, STREAM_ACCEPT, traj);
  const double u = unit53(w.v[0], w.v[1]);
  const bool acc = dH <= 0.0 || u <= exp(-dH);
  double* o = out + 5 * j;
  o[0] = H0;
  o[1] = H1;
  o[2] = dH;
  o[3] = u;
  o[4] = acc ? 1.0 : 0.0;
}

// on rejection of member j: phi_j = phi0_j (FP64 and FP32 copies); fields [member][V]
static __global__ void restore_phi(cplx<double>* phi, cplx<float>* phi32, const cplx<double>* phi0, const double* res,
                            long V, int nm) {
  const long n = (long)nm * V;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    if (res[5 * (i / V) + 4] != 0.0) continue;
    phi[i] = phi0[i];
    phi32[i] = cplx<float>{(float)phi0[i].x, (float)phi0[i].y};
  }
}

}  // namespace wz
