// Broken supersymmetric Ward-Takahashi identity of Eq. exid, per configuration.
//
// Summed over x, the variation density of the action is the cubic expression
// of Eq. nzav; with the fermions integrated out at fixed phi and the fermion
// summed over y, both sides are per-configuration quantities (the common sqrt 2
// left out; the Majorana propagator is -M^-1 C^-1, and its sign together with
// C^T = -C leaves M^-1 C^-1 in W_R):
//
//   W_L[a][b] = F_b C[a][b], F_b = sum_x F~ (b = 2, 3) or sum_x F~^* (b = 0, 1)
//   W_R[a][b] = sum_x [Kop psi_b]_a(x),  psi_b = M^-1 C^-1 u_b,  u_b(x) = e_b
//   Kop psi  = g (2 phi (D1 phi) P_+ psi + phi^2 D1 P_+ psi)
//            + g^* (2 phi^* (D1 phi^*) P_- psi + phi^*2 D1 P_- psi)
//
// D1 on spinors is the Dslash multiply with 1/omega in place of h (WZ_OP_D1);
// D1 on a periodic scalar f is sum_mu gamma_mu f_mu with f_mu = F^-1[i sin p_mu /
// omega F f], computed as one FP64 plane-pass transform of f copied into the
// four slots (zt mode ZT_GRAD).  D1 maps P_+ into P_- and back, so D1 P_+ psi =
// P_- D1 psi and D1 P_- psi = P_+ D1 psi: one D1 application per column.
// The identity states <W_R> = <W_L>; in the continuum both vanish.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "apply_impl.cuh"
#include "solver.h"
#include "wz_probe.h"

namespace wz {

namespace {

struct C4 {
  double re[4][4], im[4][4];
};

// chiral basis of Sec. 2.1: gamma_0 = [[0, 1], [1, 0]], gamma_k = [[0, i sigma_k], [-i sigma_k, 0]]
void gamma_matrix(int mu, C4* g) {
  memset(g, 0, sizeof(*g));
  // sigma_k as (re, im) 2x2
  const double s_re[3][2][2] = {{{0, 1}, {1, 0}}, {{0, 0}, {0, 0}}, {{1, 0}, {0, -1}}};
  const double s_im[3][2][2] = {{{0, 0}, {0, 0}}, {{0, -1}, {1, 0}}, {{0, 0}, {0, 0}}};
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      if (mu == 0) {
        g->re[i][2 + j] = g->re[2 + i][j] = (i == j) ? 1.0 : 0.0;
      } else {
        const int k = mu - 1;
        // upper right: i sigma = (-Im sigma, Re sigma); lower left: -i sigma
        g->re[i][2 + j] = -s_im[k][i][j];
        g->im[i][2 + j] = s_re[k][i][j];
        g->re[2 + i][j] = s_im[k][i][j];
        g->im[2 + i][j] = -s_re[k][i][j];
      }
    }
}

void mat_mul(const C4& a, const C4& b, C4* c) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double r = 0, m = 0;
      for (int k = 0; k < 4; ++k) {
        r += a.re[i][k] * b.re[k][j] - a.im[i][k] * b.im[k][j];
        m += a.re[i][k] * b.im[k][j] + a.im[i][k] * b.re[k][j];
      }
      c->re[i][j] = r;
      c->im[i][j] = m;
    }
}

// C = gamma_0 gamma_2; real orthogonal in this basis, so C^-1 = C^T
void charge_conjugation(C4* C, C4* Cinv) {
  C4 g0, g2;
  gamma_matrix(0, &g0);
  gamma_matrix(2, &g2);
  mat_mul(g0, g2, C);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      Cinv->re[i][j] = C->re[j][i];
      Cinv->im[i][j] = -C->im[j][i];
    }
}

struct Sources {
  double re[4][4], im[4][4];  // [b][s]: spin s of the uniform source of column b
};

// out[b][x][s] = source[b][s] for every site x
__global__ void uniform_sources(cplx<double>* out, long V, Sources src) {
  const int b = blockIdx.y;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < 4 * V; i += (long)gridDim.x * blockDim.x) {
    const int s = (int)(i & 3);
    out[(long)b * 4 * V + i] = cplx<double>{src.re[b][s], src.im[b][s]};
  }
}

// out[x][mu] = f(x) (or f^*) for the four slots of the gradient transform
__global__ void copy_to_slots(const cplx<double>* f, int conjugate, cplx<double>* out, long V) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < 4 * V; i += (long)gridDim.x * blockDim.x) {
    const cplx<double> v = f[i >> 2];
    out[i] = conjugate ? conj(v) : v;
  }
}

// Block partials of sum_x [Kop psi_b]_a(x), grid (nblk, 4 columns b):
// part[((b * nblk) + block) * 4 + a] (complex).
__global__ void ward_contract(const cplx<double>* phi, const cplx<double>* psi, const cplx<double>* d1psi,
                              const cplx<double>* f, const cplx<double>* fs, cplx<double> g, long V,
                              cplx<double>* part) {
  __shared__ double red[33];
  const int b = blockIdx.y;
  const cplx<double> I{0.0, 1.0};
  cplx<double> acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
  for (long x = blockIdx.x * (long)blockDim.x + threadIdx.x; x < V; x += (long)gridDim.x * blockDim.x) {
    const cplx<double> ph = phi[x], phs = conj(ph);
    const cplx<double>* p = psi + ((long)b * V + x) * 4;
    const cplx<double>* d = d1psi + ((long)b * V + x) * 4;
    const cplx<double>* fx = f + x * 4;
    const cplx<double>* fsx = fs + x * 4;
    // (D1 phi) P_+ psi = sum_mu f_mu gamma_mu (0, 0, p2, p3): upper components
    const cplx<double> gp0 = fx[0] * p[2] + fx[1] * (I * p[3]) + fx[2] * p[3] + fx[3] * (I * p[2]);
    const cplx<double> gp1 = fx[0] * p[3] + fx[1] * (I * p[2]) - fx[2] * p[2] - fx[3] * (I * p[3]);
    // (D1 phi^*) P_- psi = sum_mu fs_mu gamma_mu (p0, p1, 0, 0): lower components
    const cplx<double> gm2 = fsx[0] * p[0] - fsx[1] * (I * p[1]) - fsx[2] * p[1] - fsx[3] * (I * p[0]);
    const cplx<double> gm3 = fsx[0] * p[1] - fsx[1] * (I * p[0]) + fsx[2] * p[0] + fsx[3] * (I * p[1]);
    const cplx<double> two{2.0, 0.0};
    const cplx<double> gs = conj(g);
    acc[0] = acc[0] + g * (two * ph * gp0 + (ph * ph) * d[0]);  // D1 P_+ psi = P_- D1 psi
    acc[1] = acc[1] + g * (two * ph * gp1 + (ph * ph) * d[1]);
    acc[2] = acc[2] + gs * (two * phs * gm2 + (phs * phs) * d[2]);  // D1 P_- psi = P_+ D1 psi
    acc[3] = acc[3] + gs * (two * phs * gm3 + (phs * phs) * d[3]);
  }
  for (int a = 0; a < 4; ++a) {
    const double sr = block_sum(acc[a].x, red);
    __syncthreads();
    const double si = block_sum(acc[a].y, red);
    __syncthreads();
    if (threadIdx.x == 0) part[((long)b * gridDim.x + blockIdx.x) * 4 + a] = cplx<double>{sr, si};
  }
}

// W[a * 4 + b] = sum over the nblk block partials of column b, component a (fixed order)
__global__ void ward_reduce(const cplx<double>* part, int nblk, cplx<double>* W) {
  const int i = threadIdx.x;
  if (i >= 16) return;
  const int a = i / 4, b = i % 4;
  cplx<double> s{0.0, 0.0};
  for (int k = 0; k < nblk; ++k) s = s + part[((long)b * nblk + k) * 4 + a];
  W[i] = s;
}

// D1 phi (or D1 phi^*) components: out[x][mu] = F^-1[i sin p_mu / omega F f](x), periodic grid
int scalar_d1(wz_ctx* c, int conjugate, cplx<double>* slots, cplx<double>* out, cplx<double>* A) {
  const long V = c->V;
  count_launch();
  copy_to_slots<<<(unsigned)((4 * V + 255) / 256 < 4096 ? (4 * V + 255) / 256 : 4096), 256, 0, c->stream>>>(
      c->phi64, conjugate, slots, V);
  WZ_CUDA_TRY(c, cudaGetLastError());
  XYArgs<double> xa = xy_args<double>(c, 1);
  xa.twc = c->t64.twc1;  // a periodic field: no antiperiodic twist
  xa.tws = c->t64.tws0;
  xa.kArr = c->k64;
  xa.rpm = 1;
  xa.nplanes = c->T * c->Z;
  xa.psi = slots;
  xa.A_out = A;
  WZ_CUDA_TRY(c, launch_xy<double>(c->X, XY_FWD, xa, c->stream));
  ZTArgs<double> za = zt_args<double>(c, 1.0);
  za.A = A;
  za.hV = c->t64.w1sV;
  WZ_CUDA_TRY(c, launch_zt<double>(c->Z, c->T, ZT_GRAD, za, 1, c->stream));
  XYArgs<double> xi = xa;
  xi.A_in = A;
  xi.A_out = nullptr;
  xi.psi = nullptr;
  xi.v_out = out;
  WZ_CUDA_TRY(c, launch_xy<double>(c->X, XY_INV, xi, c->stream));
  return WZ_OK;
}

}  // namespace

}  // namespace wz

using namespace wz;

extern "C" int wz_ward_identity(wz_ctx* c, double tol, int maxiter, unsigned flags, double* WR, double* WL,
                                wz_solve_stats* stats) {
  if (!c) return WZ_EINVAL;
  if (!WR || !WL || tol <= 0.0 || maxiter < 1) return set_error(c, WZ_EINVAL, "wz_ward_identity: bad argument");
  if (c->nm != 1) return set_error(c, WZ_EINVAL, "wz_ward_identity: single-lattice context expected");
  const auto t0 = std::chrono::steady_clock::now();
  const long V = c->V;
  const size_t f4 = sizeof(cplx<double>) * 4 * (size_t)V;
  // workspace: sources / M^dag sources (4), psi (4), D1 psi (4), two gradient fields, slots
  const size_t need = f4 * (4 + 4 + 4 + 2 + 1);
  WZ_CUDA_TRY(c, c->ws_force.reserve(need));
  cplx<double>* src = (cplx<double>*)c->ws_force.ptr;
  cplx<double>* psi = src + 4 * 4 * V;
  cplx<double>* d1psi = psi + 4 * 4 * V;
  cplx<double>* fgrad = d1psi + 4 * 4 * V;
  cplx<double>* fsgrad = fgrad + 4 * V;
  cplx<double>* slots = fsgrad + 4 * V;
  WZ_CUDA_TRY(c, c->ws_apply.reserve(apply_ws_bytes<double>(c, WZ_OP_MDAG, 4)));
  cplx<double>* A = (cplx<double>*)c->ws_apply.ptr;

  // uniform sources C^-1 e_b, then psi_b = M^-1 C^-1 u_b = (M^dag M)^-1 M^dag C^-1 u_b
  C4 C, Cinv;
  charge_conjugation(&C, &Cinv);
  Sources so{};
  for (int b = 0; b < 4; ++b)
    for (int s = 0; s < 4; ++s) {
      so.re[b][s] = Cinv.re[s][b];
      so.im[b][s] = Cinv.im[s][b];
    }
  count_launch();
  uniform_sources<<<dim3(256, 4), 256, 0, c->stream>>>(psi, V, so);
  WZ_CUDA_TRY(c, cudaGetLastError());
  int rc = apply_op<double>(c, WZ_OP_MDAG, psi, src, 4, 0.0, A);
  if (rc) return rc;
  SolveOut sol;
  rc = (flags & WZ_SOLVE_MIXED) ? solve_impl<float>(c, src, psi, 4, single_shift(0.0), tol, maxiter, false, 0.1, &sol)
                                : solve_impl<double>(c, src, psi, 4, single_shift(0.0), tol, maxiter, false, 0.0, &sol);
  if (rc && rc != WZ_NOT_CONVERGED) return rc;
  const int solve_rc = rc;
  rc = apply_op<double>(c, WZ_OP_D1, psi, d1psi, 4, 0.0, A);
  if (rc) return rc;
  if ((rc = scalar_d1(c, 0, slots, fgrad, A))) return rc;
  if ((rc = scalar_d1(c, 1, slots, fsgrad, A))) return rc;

  const int nblk = 128;
  WZ_CUDA_TRY(c, c->ws_red.reserve(sizeof(cplx<double>) * (4 * 4 * nblk + 16)));
  cplx<double>* part = (cplx<double>*)c->ws_red.ptr;
  count_launch();
  ward_contract<<<dim3(nblk, 4), 256, 0, c->stream>>>(c->phi64, psi, d1psi, fgrad, fsgrad,
                                                       cplx<double>{c->p.g_re, c->p.g_im}, V, part);
  WZ_CUDA_TRY(c, cudaGetLastError());
  count_launch();
  ward_reduce<<<1, 32, 0, c->stream>>>(part, nblk, part + 4 * 4 * nblk);
  WZ_CUDA_TRY(c, cudaGetLastError());
  // row-major [a][b] complex is the (re, im) layout of WR
  WZ_CUDA_TRY(c, cudaMemcpyAsync(WR, part + 4 * 4 * nblk, sizeof(cplx<double>) * 16, cudaMemcpyDeviceToHost,
                                 c->stream));
  WZ_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  // left side: F_b C[a][b], F_b = sum_x F~ for b in P_+ (2, 3), its conjugate for b in P_- (0, 1)
  double F[2];
  if ((rc = wz_aux_vev(c, F))) return rc;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      const double fr = F[0] * (double)V, fi = (b >= 2 ? F[1] : -F[1]) * (double)V;
      WL[2 * (a * 4 + b)] = fr * C.re[a][b] - fi * C.im[a][b];
      WL[2 * (a * 4 + b) + 1] = fr * C.im[a][b] + fi * C.re[a][b];
    }
  if (stats) {
    stats->iterations = sol.iterations;
    stats->total_iterations = sol.total_iterations;
    stats->reliable_updates = sol.reliable_updates;
    stats->converged = sol.converged;
    stats->max_true_residual = sol.max_true_residual;
    stats->site_applies = (double)(sol.total_iterations + sol.reliable_updates) * (double)c->V;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (solve_rc == WZ_NOT_CONVERGED) return set_error(c, WZ_NOT_CONVERGED, "wz_ward_identity: solve reached maxiter");
  return WZ_OK;
}

// ---------------------------------------------------------------------------
// Correlators of the naive lattice supercurrent (Eq. latsuc) with the scalar and
// the fermion (Eq. sitre), x and y at zero spatial momentum:
//
//   S_mu(x)  = Gamma_mu(x) chi(x),  Gamma_mu = sqrt2 [(D1 phi) gamma_mu P_+ + (D1 phi^*) gamma_mu P_-
//                                                     + W' gamma_mu P_- + W'^* gamma_mu P_+]
//   psi_b    = -M^-1 (w e_b),  Q_mu(t)[a][b] = sum_xvec [Gamma_mu psi_b]_a(t, xvec)
//   R[s][mu][dx][dy][a][b] = sum_t' xi(t')^* sgn Phi_s(t' + dy) Q_mu(t' + dx)[a][b]
//
// with W' = m phi + g phi^2, xi(t) = sum_zvec w, Phi_0 = sum_yvec phi, Phi_1 = Phi_0^*
// and sgn = -1 where the fermion crosses the antiperiodic boundary (t' + dx >= T).
// In the chiral basis gamma_mu = [[0, A_mu], [B_mu, 0]]: gamma_mu P_+ psi is the
// upper 2-vector u = A_mu psi_lo, gamma_mu P_- psi the lower l = B_mu psi_up, and
// D1 f = sum_nu f_nu gamma_nu maps u to the lower sum_nu f_nu B_nu u and l to the
// upper sum_nu f_nu A_nu l.  Per site: upper = (D1 phi^*) l + W'^* u, lower =
// (D1 phi) u + W' l.  Sums are in a fixed order (block partials, then chunks).

namespace wz {

namespace {

struct GammaBlocks {
  double Are[4][2][2], Aim[4][2][2], Bre[4][2][2], Bim[4][2][2];
};

GammaBlocks gamma_blocks() {
  GammaBlocks gb;
  for (int mu = 0; mu < 4; ++mu) {
    C4 g;
    gamma_matrix(mu, &g);
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        gb.Are[mu][i][j] = g.re[i][2 + j];
        gb.Aim[mu][i][j] = g.im[i][2 + j];
        gb.Bre[mu][i][j] = g.re[2 + i][j];
        gb.Bim[mu][i][j] = g.im[2 + i][j];
      }
  }
  return gb;
}

// out[b][x][s] = w(x) delta(s, b)
__global__ void spin_sources(const cplx<double>* w, cplx<double>* out, long V) {
  const int b = blockIdx.y;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < 4 * V; i += (long)gridDim.x * blockDim.x)
    out[(long)b * 4 * V + i] = ((int)(i & 3) == b) ? w[i >> 2] : cplx<double>{0.0, 0.0};
}

// Block partials of sum_xvec [Gamma_mu psi_b]_a(t, xvec) / sqrt2 with psi_b = M^-1 (w e_b),
// grid (nchunk, T, 4 columns b): part[((b * T + t) * nchunk + chunk) * 16 + mu * 4 + a].
__global__ void current_contract(const cplx<double>* phi, const cplx<double>* psi, const cplx<double>* f,
                                 const cplx<double>* fs, cplx<double> m, cplx<double> g, long V, long V3,
                                 GammaBlocks gb, cplx<double>* part) {
  __shared__ double red[33];
  const int b = blockIdx.z, t = blockIdx.y, nchunk = gridDim.x;
  cplx<double> acc[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) acc[k] = cplx<double>{0.0, 0.0};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < V3; i += (long)nchunk * blockDim.x) {
    const long x = (long)t * V3 + i;
    const cplx<double> ph = phi[x];
    const cplx<double> Wp = m * ph + g * (ph * ph), Wps = conj(Wp);
    const cplx<double>* p = psi + ((long)b * V + x) * 4;
    const cplx<double> up[2] = {p[0], p[1]}, lo[2] = {p[2], p[3]};
    cplx<double> Bf[2][2], Afs[2][2];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int q = 0; q < 2; ++q) Bf[r][q] = Afs[r][q] = cplx<double>{0.0, 0.0};
#pragma unroll
    for (int nu = 0; nu < 4; ++nu) {
      const cplx<double> fn = f[x * 4 + nu], fsn = fs[x * 4 + nu];
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          Bf[r][q] = Bf[r][q] + fn * cplx<double>{gb.Bre[nu][r][q], gb.Bim[nu][r][q]};
          Afs[r][q] = Afs[r][q] + fsn * cplx<double>{gb.Are[nu][r][q], gb.Aim[nu][r][q]};
        }
    }
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      cplx<double> u[2], l[2];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        u[r] = cplx<double>{gb.Are[mu][r][0], gb.Aim[mu][r][0]} * lo[0] +
               cplx<double>{gb.Are[mu][r][1], gb.Aim[mu][r][1]} * lo[1];
        l[r] = cplx<double>{gb.Bre[mu][r][0], gb.Bim[mu][r][0]} * up[0] +
               cplx<double>{gb.Bre[mu][r][1], gb.Bim[mu][r][1]} * up[1];
      }
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        acc[mu * 4 + r] = acc[mu * 4 + r] + Afs[r][0] * l[0] + Afs[r][1] * l[1] + Wps * u[r];
        acc[mu * 4 + 2 + r] = acc[mu * 4 + 2 + r] + Bf[r][0] * u[0] + Bf[r][1] * u[1] + Wp * l[r];
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const double sr = block_sum(acc[k].x, red);
    __syncthreads();
    const double si = block_sum(acc[k].y, red);
    __syncthreads();
    if (threadIdx.x == 0) part[(((long)b * gridDim.y + t) * nchunk + blockIdx.x) * 16 + k] = cplx<double>{sr, si};
  }
}

// Block partials of the time-slice sums of phi (k = 0) and w (k = 1), grid (nchunk, T, 2):
// part[(k * T + t) * nchunk + chunk]
__global__ void slice_sums(const cplx<double>* phi, const cplx<double>* w, long V3, cplx<double>* part) {
  __shared__ double red[33];
  const int k = blockIdx.z, t = blockIdx.y, nchunk = gridDim.x;
  const cplx<double>* fld = k ? w : phi;
  double sr = 0.0, si = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < V3; i += (long)nchunk * blockDim.x) {
    const cplx<double> v = fld[(long)t * V3 + i];
    sr += v.x;
    si += v.y;
  }
  sr = block_sum(sr, red);
  __syncthreads();
  si = block_sum(si, red);
  if (threadIdx.x == 0) part[((long)k * gridDim.y + t) * nchunk + blockIdx.x] = cplx<double>{sr, si};
}

// Q[(b * T + t) * 16 + mu * 4 + a] and S[k * T + t] (k = 0: Phi_0, 1: xi): the chunk partials
// summed in chunk order
__global__ void sc_reduce(const cplx<double>* qpart, const cplx<double>* spart, int T, int nchunk, cplx<double>* Q,
                          cplx<double>* S) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int nq = 64 * T;
  cplx<double> s{0.0, 0.0};
  if (i < nq) {
    const int k = i % 16, bt = i / 16;
    for (int ch = 0; ch < nchunk; ++ch) s = s + qpart[((long)bt * nchunk + ch) * 16 + k];
    Q[i] = s;
  } else if (i < nq + 2 * T) {
    const int j = i - nq;
    for (int ch = 0; ch < nchunk; ++ch) s = s + spart[(long)j * nchunk + ch];
    S[j] = s;
  }
}

// R[((((s * 4 + mu) * T + dx) * T + dy) * 4 + a) * 4 + b], the factor -sqrt2 of Gamma and psi applied here
__global__ void sc_combine(const cplx<double>* Q, const cplx<double>* S, int T, cplx<double>* R) {
  const long n = 128L * T * T;
  const long o = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (o >= n) return;
  const int b = (int)(o & 3), a = (int)((o >> 2) & 3);
  long r = o >> 4;
  const int dy = (int)(r % T);
  r /= T;
  const int dx = (int)(r % T);
  r /= T;
  const int mu = (int)(r % 4), s = (int)(r / 4);
  cplx<double> acc{0.0, 0.0};
  for (int tp = 0; tp < T; ++tp) {
    const cplx<double> xi = conj(S[T + tp]);
    cplx<double> ph = S[(tp + dy) % T];
    if (s) ph = conj(ph);
    int tq = tp + dx;
    const double sg = tq >= T ? -1.0 : 1.0;
    if (tq >= T) tq -= T;
    acc = acc + sg * (xi * ph * Q[((long)b * T + tq) * 16 + mu * 4 + a]);
  }
  R[o] = (-1.4142135623730951) * acc;
}

}  // namespace

}  // namespace wz

extern "C" int wz_supercurrent(wz_ctx* c, const void* w, double tol, int maxiter, unsigned flags, double* R,
                               wz_solve_stats* stats) {
  if (!c) return WZ_EINVAL;
  if (!w || !R || tol <= 0.0 || maxiter < 1) return set_error(c, WZ_EINVAL, "wz_supercurrent: bad argument");
  if (c->nm != 1) return set_error(c, WZ_EINVAL, "wz_supercurrent: single-lattice context expected");
  const auto t0 = std::chrono::steady_clock::now();
  const long V = c->V;
  const int T = c->T;
  const long V3 = V / T;
  const size_t f4 = sizeof(cplx<double>) * 4 * (size_t)V;
  const cplx<double>* wd = (const cplx<double>*)w;
  if (!is_device_pointer(w)) {
    WZ_CUDA_TRY(c, c->ws_stage.reserve(sizeof(cplx<double>) * (size_t)V));
    WZ_CUDA_TRY(c, cudaMemcpyAsync(c->ws_stage.ptr, w, sizeof(cplx<double>) * (size_t)V, cudaMemcpyHostToDevice,
                                   c->stream));
    wd = (const cplx<double>*)c->ws_stage.ptr;
  } else if (((unsigned long long)w) & 15ull) {
    return set_error(c, WZ_EINVAL, "wz_supercurrent: w must be 16-byte aligned");
  }
  // workspace: sources / M^dag sources (4), psi (4), two gradient fields, slots
  WZ_CUDA_TRY(c, c->ws_force.reserve(f4 * (4 + 4 + 2 + 1)));
  cplx<double>* src = (cplx<double>*)c->ws_force.ptr;
  cplx<double>* psi = src + 4 * 4 * V;
  cplx<double>* fgrad = psi + 4 * 4 * V;
  cplx<double>* fsgrad = fgrad + 4 * V;
  cplx<double>* slots = fsgrad + 4 * V;
  WZ_CUDA_TRY(c, c->ws_apply.reserve(apply_ws_bytes<double>(c, WZ_OP_MDAG, 4)));
  cplx<double>* A = (cplx<double>*)c->ws_apply.ptr;

  count_launch();
  spin_sources<<<dim3(256, 4), 256, 0, c->stream>>>(wd, psi, V);
  WZ_CUDA_TRY(c, cudaGetLastError());
  int rc = apply_op<double>(c, WZ_OP_MDAG, psi, src, 4, 0.0, A);
  if (rc) return rc;
  SolveOut sol;
  rc = (flags & WZ_SOLVE_MIXED) ? solve_impl<float>(c, src, psi, 4, single_shift(0.0), tol, maxiter, false, 0.1, &sol)
                                : solve_impl<double>(c, src, psi, 4, single_shift(0.0), tol, maxiter, false, 0.0, &sol);
  if (rc && rc != WZ_NOT_CONVERGED) return rc;
  const int solve_rc = rc;
  if ((rc = scalar_d1(c, 0, slots, fgrad, A))) return rc;
  if ((rc = scalar_d1(c, 1, slots, fsgrad, A))) return rc;

  const int nchunk = (int)std::min<long>(64, std::max<long>(1, (V3 + 2047) / 2048));
  const size_t nqp = (size_t)4 * T * nchunk * 16, nsp = (size_t)2 * T * nchunk, nq = (size_t)64 * T,
               ns = (size_t)2 * T, nr = (size_t)128 * T * T;
  WZ_CUDA_TRY(c, c->ws_red.reserve(sizeof(cplx<double>) * (nqp + nsp + nq + ns + nr)));
  cplx<double>* qpart = (cplx<double>*)c->ws_red.ptr;
  cplx<double>* spart = qpart + nqp;
  cplx<double>* Q = spart + nsp;
  cplx<double>* S = Q + nq;
  cplx<double>* Rd = S + ns;
  count_launch();
  current_contract<<<dim3(nchunk, T, 4), 256, 0, c->stream>>>(c->phi64, psi, fgrad, fsgrad,
                                                              cplx<double>{c->p.m_re, c->p.m_im},
                                                              cplx<double>{c->p.g_re, c->p.g_im}, V, V3,
                                                              gamma_blocks(), qpart);
  WZ_CUDA_TRY(c, cudaGetLastError());
  count_launch();
  slice_sums<<<dim3(nchunk, T, 2), 256, 0, c->stream>>>(c->phi64, wd, V3, spart);
  WZ_CUDA_TRY(c, cudaGetLastError());
  count_launch();
  sc_reduce<<<(unsigned)((nq + ns + 127) / 128), 128, 0, c->stream>>>(qpart, spart, T, nchunk, Q, S);
  WZ_CUDA_TRY(c, cudaGetLastError());
  count_launch();
  sc_combine<<<(unsigned)((nr + 127) / 128), 128, 0, c->stream>>>(Q, S, T, Rd);
  WZ_CUDA_TRY(c, cudaGetLastError());
  WZ_CUDA_TRY(c, cudaMemcpyAsync(R, Rd, sizeof(cplx<double>) * nr, cudaMemcpyDeviceToHost, c->stream));
  WZ_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (stats) {
    stats->iterations = sol.iterations;
    stats->total_iterations = sol.total_iterations;
    stats->reliable_updates = sol.reliable_updates;
    stats->converged = sol.converged;
    stats->max_true_residual = sol.max_true_residual;
    stats->site_applies = (double)(sol.total_iterations + sol.reliable_updates) * (double)c->V;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (solve_rc == WZ_NOT_CONVERGED) return set_error(c, WZ_NOT_CONVERGED, "wz_supercurrent: solve reached maxiter");
  return WZ_OK;
}
