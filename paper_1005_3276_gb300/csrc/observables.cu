// Observables: the auxiliary-field VEV (Sec. 7.5) and the locality probe of
// the Dirac operator (Sec. 3.2, Eq. uir).
#include <cstring>
#include <vector>

#include "apply_impl.cuh"
#include "wz_ctx.h"

namespace wz {

// Sum over the sites of one member of w = m^* phi^* + g^* phi^*2, block
// partials [member][nb] (re, im).  On the equation of motion of Eq. lata,
// F~ = -(1 - D2/2) w and (1 - D2/2)(p = 0) = 1, so (1/V) sum_x F~ = -(1/V) sum_x w.
static __global__ void aux_w_partials(const cplx<double>* phi, const SiteCoef<double>* k, long V, double* part) {
  __shared__ double red[33];
  const int member = blockIdx.y;
  const SiteCoef<double> kc = k[member];
  const cplx<double> ms{kc.m_re, -kc.m_im}, gs{kc.g_re, -kc.g_im};
  double sr = 0.0, si = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < V; i += (long)gridDim.x * blockDim.x) {
    const cplx<double> f = conj(phi[member * V + i]);
    const cplx<double> w = ms * f + gs * (f * f);
    sr += w.x;
    si += w.y;
  }
  sr = block_sum(sr, red);
  __syncthreads();
  si = block_sum(si, red);
  if (threadIdx.x == 0) {
    part[2 * ((long)member * gridDim.x + blockIdx.x)] = sr;
    part[2 * ((long)member * gridDim.x + blockIdx.x) + 1] = si;
  }
}

// Locality probe: for psi = Dslash applied to a unit point source at the
// origin, fmax[r] = max over sites with taxi-driver distance r of the spinor
// norm ||psi(x)|| (Eq. uir).  Norms are non-negative, so their IEEE bit
// patterns order like the values and the maximum is taken with integer atomics
// (order independent, hence deterministic).
static __global__ void locality_max(const cplx<double>* psi, int T, int Z, int Y, int X, unsigned long long* fmax) {
  const long V = (long)T * Z * Y * X;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < V; i += (long)gridDim.x * blockDim.x) {
    const int x = (int)(i % X), y = (int)((i / X) % Y), z = (int)((i / ((long)X * Y)) % Z);
    const int t = (int)(i / ((long)X * Y * Z));
    const int r = min(t, T - t) + min(z, Z - z) + min(y, Y - y) + min(x, X - x);
    double n2 = 0.0;
    for (int s = 0; s < 4; ++s) {
      const cplx<double> v = psi[4 * i + s];
      n2 += v.x * v.x + v.y * v.y;
    }
    const double n = sqrt(n2);
    unsigned long long bits;
    memcpy(&bits, &n, sizeof(bits));
    atomicMax(&fmax[r], bits);
  }
}

// min / max over the momenta of den(p) = D_mu^dag D_mu + |m|^2 = 1 / (dV V)
// (positive, so the IEEE bit patterns order like the values).
static __global__ void den_minmax(const double* dV, long V, unsigned long long* mm) {
  double lo = HUGE_VAL, hi = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < V; i += (long)gridDim.x * blockDim.x) {
    const double den = 1.0 / (dV[i] * (double)V);
    lo = fmin(lo, den);
    hi = fmax(hi, den);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    unsigned long long bl, bh;
    memcpy(&bl, &lo, sizeof(bl));
    memcpy(&bh, &hi, sizeof(bh));
    atomicMin(&mm[0], bl);
    atomicMax(&mm[1], bh);
  }
}

}  // namespace wz

using namespace wz;

extern "C" {

int wz_aux_vev(wz_ctx* c, double* F) {
  if (!c || !F) return set_error(c, WZ_EINVAL, "wz_aux_vev: null pointer");
  const int nb = 64;
  WZ_CUDA_TRY(c, c->ws_red.reserve(sizeof(double) * 2 * nb * c->nm));
  count_launch();
  aux_w_partials<<<dim3(nb, c->nm), 256, 0, c->stream>>>(c->phi64, c->k64, c->V, (double*)c->ws_red.ptr);
  WZ_CUDA_TRY(c, cudaGetLastError());
  std::vector<double> h(2 * nb * c->nm);
  WZ_CUDA_TRY(c, cudaMemcpyAsync(h.data(), c->ws_red.ptr, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->stream));
  WZ_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  for (int j = 0; j < c->nm; ++j) {
    double sr = 0.0, si = 0.0;
    for (int b = 0; b < nb; ++b) {
      sr += h[2 * (j * nb + b)];
      si += h[2 * (j * nb + b) + 1];
    }
    F[2 * j] = -sr / (double)c->V;
    F[2 * j + 1] = -si / (double)c->V;
  }
  return WZ_OK;
}

int wz_locality(wz_ctx* c, double* f, int nf) { return wz_locality_op(c, WZ_OP_DSLASH, f, nf); }

int wz_locality_op(wz_ctx* c, int op, double* f, int nf) {
  if (!c || !f) return set_error(c, WZ_EINVAL, "wz_locality: null pointer");
  if (op != WZ_OP_DSLASH && op != WZ_OP_D) return set_error(c, WZ_EINVAL, "wz_locality_op: op must be Dslash or D");
  const int rmax = c->T / 2 + c->Z / 2 + c->Y / 2 + c->X / 2;
  if (nf < rmax + 1) return set_error(c, WZ_EINVAL, "wz_locality: f needs T/2 + Z/2 + Y/2 + X/2 + 1 entries");
  const size_t field = sizeof(cplx<double>) * 4 * (size_t)c->V;
  WZ_CUDA_TRY(c, c->ws_stage.reserve(2 * field + sizeof(unsigned long long) * (rmax + 1)));
  cplx<double>* src = (cplx<double>*)c->ws_stage.ptr;
  cplx<double>* psi = src + 4 * c->V;
  unsigned long long* fmax = (unsigned long long*)(psi + 4 * c->V);
  const cplx<double> one{1.0, 0.0};
  WZ_CUDA_TRY(c, cudaMemsetAsync(src, 0, field, c->stream));
  WZ_CUDA_TRY(c, cudaMemcpyAsync(src, &one, sizeof(one), cudaMemcpyHostToDevice, c->stream));  // spin 0 at the origin
  WZ_CUDA_TRY(c, cudaMemsetAsync(fmax, 0, sizeof(unsigned long long) * (rmax + 1), c->stream));
  WZ_CUDA_TRY(c, c->ws_apply.reserve(apply_ws_bytes<double>(c, op, 1)));
  int rc = apply_op<double>(c, op, src, psi, 1, 0.0, (cplx<double>*)c->ws_apply.ptr);
  if (rc) return rc;
  count_launch();
  const long blocks = (c->V + 255) / 256;
  locality_max<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, c->stream>>>(psi, c->T, c->Z, c->Y, c->X, fmax);
  WZ_CUDA_TRY(c, cudaGetLastError());
  std::vector<unsigned long long> h(rmax + 1);
  WZ_CUDA_TRY(c, cudaMemcpyAsync(h.data(), fmax, sizeof(unsigned long long) * (rmax + 1), cudaMemcpyDeviceToHost,
                                 c->stream));
  WZ_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  for (int r = 0; r <= rmax; ++r) memcpy(&f[r], &h[r], sizeof(double));
  for (int r = rmax + 1; r < nf; ++r) f[r] = 0.0;
  return WZ_OK;
}

int wz_spectral_bounds(wz_ctx* c, double* lo, double* hi) {
  if (!c || !lo || !hi) return set_error(c, WZ_EINVAL, "wz_spectral_bounds: null pointer");
  WZ_CUDA_TRY(c, c->ws_red.reserve(2 * sizeof(unsigned long long)));
  unsigned long long* mm = (unsigned long long*)c->ws_red.ptr;
  const double inf = HUGE_VAL;
  unsigned long long init[2] = {0, 0};
  memcpy(&init[0], &inf, sizeof(double));
  unsigned long long* h = (unsigned long long*)((char*)c->host_pinned + WZ_PINNED_SCRATCH_OFFSET);
  h[0] = init[0];
  h[1] = init[1];
  WZ_CUDA_TRY(c, cudaMemcpyAsync(mm, h, 2 * sizeof(unsigned long long), cudaMemcpyHostToDevice, c->stream));
  count_launch();
  const long blocks = (c->V + 255) / 256;
  den_minmax<<<(unsigned)(blocks < 1024 ? blocks : 1024), 256, 0, c->stream>>>(c->t64.dV, c->V, mm);
  WZ_CUDA_TRY(c, cudaGetLastError());
  WZ_CUDA_TRY(c, cudaMemcpyAsync(h, mm, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
  WZ_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  memcpy(lo, &h[0], sizeof(double));
  memcpy(hi, &h[1], sizeof(double));
  return WZ_OK;
}

}  // extern "C"
