// C ABI entry points: context, tables, phi, apply.
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "apply_impl.cuh"
#include "solver.h"
#include "wz_cg.cuh"
#include "wz_ctx.h"

namespace wz {

Probe g_probe;
std::atomic<unsigned long long> g_launches{0};
thread_local unsigned long long tl_launches = 0;

int set_error(wz_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_error(wz_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string("CUDA error ") + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ") at " + where;
  return set_error(c, e == cudaErrorMemoryAllocation ? WZ_ENOMEM : WZ_ECUDA, m);
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool extent_supported(int n) {
  switch (n) {
#define WZ_CASE(k) \
  case k: return true;
    WZ_FOR_EXTENTS(WZ_CASE)
#undef WZ_CASE
  }
  return false;
}

bool zt_supported(int nz, int nt) {
#define WZ_CASE(z, t) \
  if (nz == z && nt == t) return true;
  WZ_FOR_ZT_PAIRS(WZ_CASE)
#undef WZ_CASE
  return false;
}

// ----------------------------------------------------------------------------- tables (a0)
// One thread per fermion momentum p = (pi(2nt+1)/T, 2pi nz/Z, 2pi ny/Y, 2pi nx/X):
//   b = M0 - r sum_mu 2 sin^2(p_mu/2),  omega = sqrt(b^2 + sum sin^2 p_mu),
//   h = 2/(omega + b),  den = h^2 sum sin^2 p_mu + |m|^2              (Sec. 3.1, 7.3)
// Evaluated in FP64; the FP32 table is the rounded FP64 value.  Tables are
// stored in the xy-transposed momentum order [pt][pz][px][py] of the zt pass.
struct TableArgs {
  int T, Z, Y, X;
  double r, M0, m2, invV;
  double *hV, *hdV, *dV, *d2sV, *ksV, *w1V, *w1sV, *d2fV;
  float *hVf, *hdVf, *dVf, *d2sVf, *ksVf, *w1Vf, *w1sVf, *d2fVf;
};

__global__ void momentum_tables_kernel(TableArgs a) {
  const long V = (long)a.T * a.Z * a.Y * a.X;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < V; i += (long)gridDim.x * blockDim.x) {
    const int nx = (int)(i % a.X);
    const int ny = (int)((i / a.X) % a.Y);
    const int nz = (int)((i / ((long)a.X * a.Y)) % a.Z);
    const int nt = (int)(i / ((long)a.X * a.Y * a.Z));
    // angles in units of pi
    const double ang[4] = {(2.0 * nt + 1.0) / a.T, 2.0 * nz / a.Z, 2.0 * ny / a.Y, 2.0 * nx / a.X};
    double s2 = 0.0, w = 0.0;
    for (int mu = 0; mu < 4; ++mu) {
      double sn, cs;
      sincospi(ang[mu], &sn, &cs);
      s2 += sn * sn;
      w += 1.0 - cs;  // 2 sin^2(p/2)
    }
    const double b = a.M0 - a.r * w;
    const double omega = sqrt(b * b + s2);
    const double h = 2.0 / (omega + b);
    const double den = h * h * s2 + a.m2;
    // stored in the xy-transposed momentum order of the zt pass: [pt][pz][px][py]
    const long j = (((long)nt * a.Z + nz) * a.X + nx) * a.Y + ny;
    a.hV[j] = h * a.invV;
    a.hdV[j] = h / den * a.invV;
    a.dV[j] = a.invV / den;
    a.w1V[j] = a.invV / omega;
    // D2 = 1 - b/omega = sum sin^2 / (omega (omega + b)) = h sum sin^2 / (2 omega):
    // the same value without the cancellation of 1 - b/omega at small p
    a.d2fV[j] = 0.5 * h * s2 / omega * a.invV;
    a.d2fVf[j] = (float)a.d2fV[j];
    a.hVf[j] = (float)a.hV[j];
    a.hdVf[j] = (float)a.hdV[j];
    a.dVf[j] = (float)a.dV[j];
    a.w1Vf[j] = (float)a.w1V[j];
    // scalar symbols on the periodic grid (p_t = 2 pi nt / T): D2 = 1 - b/omega,
    // K = 1 - D2/2 (Eq. acws); at the zone corners sum sin^2 = 0 and omega = |b|
    double s2p = 0.0, wp = 0.0;
    for (int mu = 0; mu < 4; ++mu) {
      double sn, cs;
      sincospi(mu == 0 ? 2.0 * nt / a.T : ang[mu], &sn, &cs);
      s2p += sn * sn;
      wp += 1.0 - cs;
    }
    const double bp = a.M0 - a.r * wp;
    const double op = sqrt(bp * bp + s2p);
    const double D2 = op > 0.0 ? 1.0 - bp / op : 1.0;
    a.d2sV[j] = D2 * a.invV;
    a.ksV[j] = (1.0 - 0.5 * D2) * a.invV;
    a.d2sVf[j] = (float)a.d2sV[j];
    a.ksVf[j] = (float)a.ksV[j];
    a.w1sV[j] = a.invV / op;  // op >= 1 at the zone corners (b odd there)
    a.w1sVf[j] = (float)a.w1sV[j];
  }
}

// per-axis tables: [sinT(T) sinZ(Z) sinY(Y) sinX(X) twc(T) tws(T) ones(T) zeros(T)]
__global__ void axis_tables_kernel(int T, int Z, int Y, int X, double* d, float* f) {
  const int n = 5 * T + Z + Y + X;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double v;
    if (i < T) {
      v = sinpi((2.0 * i + 1.0) / T);
    } else if (i < T + Z) {
      v = sinpi(2.0 * (i - T) / Z);
    } else if (i < T + Z + Y) {
      v = sinpi(2.0 * (i - T - Z) / Y);
    } else if (i < T + Z + Y + X) {
      v = sinpi(2.0 * (i - T - Z - Y) / X);
    } else if (i < 2 * T + Z + Y + X) {
      v = cospi((double)(i - (T + Z + Y + X)) / T);
    } else if (i < 3 * T + Z + Y + X) {
      v = sinpi((double)(i - (2 * T + Z + Y + X)) / T);
    } else if (i < 4 * T + Z + Y + X) {
      v = 1.0;
    } else {
      v = 0.0;
    }
    d[i] = v;
    f[i] = (float)v;
  }
}

template <typename R> static void carve(Tables<R>& t, R* base, long V, int T, int Z, int Y, int X) {
  t.hV = base;
  t.hdV = base + V;
  t.dV = base + 2 * V;
  t.d2sV = base + 3 * V;
  t.ksV = base + 4 * V;
  t.w1V = base + 5 * V;
  t.w1sV = base + 6 * V;
  t.d2fV = base + 7 * V;
  R* ax = base + 8 * V;
  t.sinT = ax;
  t.sinZ = ax + T;
  t.sinY = ax + T + Z;
  t.sinX = ax + T + Z + Y;
  t.twc = ax + T + Z + Y + X;
  t.tws = ax + 2 * T + Z + Y + X;
  t.twc1 = ax + 3 * T + Z + Y + X;
  t.tws0 = ax + 4 * T + Z + Y + X;
}

static int build_tables(wz_ctx* c) {
  const long V = c->V;
  const long naxis = 5L * c->T + c->Z + c->Y + c->X;
  const long n = 8 * V + naxis;
  WZ_CUDA_TRY(c, cudaMalloc(&c->t64.block, n * sizeof(double)));
  WZ_CUDA_TRY(c, cudaMalloc(&c->t32.block, n * sizeof(float)));
  carve(c->t64, (double*)c->t64.block, V, c->T, c->Z, c->Y, c->X);
  carve(c->t32, (float*)c->t32.block, V, c->T, c->Z, c->Y, c->X);
  TableArgs a;
  a.T = c->T;
  a.Z = c->Z;
  a.Y = c->Y;
  a.X = c->X;
  a.r = c->p.r;
  a.M0 = c->p.M0;
  a.m2 = c->p.m_re * c->p.m_re + c->p.m_im * c->p.m_im;
  a.invV = 1.0 / (double)V;
  a.hV = c->t64.hV;
  a.hdV = c->t64.hdV;
  a.dV = c->t64.dV;
  a.d2sV = c->t64.d2sV;
  a.ksV = c->t64.ksV;
  a.w1V = c->t64.w1V;
  a.w1sV = c->t64.w1sV;
  a.d2fV = c->t64.d2fV;
  a.d2fVf = c->t32.d2fV;
  a.w1Vf = c->t32.w1V;
  a.w1sVf = c->t32.w1sV;
  a.hVf = c->t32.hV;
  a.hdVf = c->t32.hdV;
  a.dVf = c->t32.dV;
  a.d2sVf = c->t32.d2sV;
  a.ksVf = c->t32.ksV;
  const int blocks = (int)((V + 255) / 256 < 1024 ? (V + 255) / 256 : 1024);
  count_launch(2);
  momentum_tables_kernel<<<blocks, 256, 0, c->stream>>>(a);
  WZ_CUDA_TRY(c, cudaGetLastError());
  axis_tables_kernel<<<1, 256, 0, c->stream>>>(c->T, c->Z, c->Y, c->X, c->t64.sinT, c->t32.sinT);
  WZ_CUDA_TRY(c, cudaGetLastError());
  return WZ_OK;
}

__global__ void phi_to_f32_kernel(const cplx<double>* in, cplx<float>* out, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    out[i] = cplx<float>{(float)in[i].x, (float)in[i].y};
}

// Stage nbytes of a host or device source into a device pointer usable by kernels.
static int stage_in(wz_ctx* c, const void* src, size_t nbytes, void* dev_dst) {
  WZ_CUDA_TRY(c, cudaMemcpyAsync(dev_dst, src, nbytes, cudaMemcpyDefault, c->stream));
  return WZ_OK;
}

template <typename R>
static int apply_typed(wz_ctx* c, int op, const void* in, void* out, int nrhs, double shift) {
  const size_t field = sizeof(cplx<R>) * 4 * (size_t)c->V * nrhs;
  WZ_CUDA_TRY(c, c->ws_apply.reserve(apply_ws_bytes<R>(c, op, nrhs)));
  const bool din = is_device_pointer(in), dout = is_device_pointer(out);
  const cplx<R>* pin = (const cplx<R>*)in;
  cplx<R>* pout = (cplx<R>*)out;
  if (!din || !dout) {
    WZ_CUDA_TRY(c, c->ws_stage.reserve(2 * field));
    cplx<R>* sin_ = (cplx<R>*)c->ws_stage.ptr;
    cplx<R>* sout = sin_ + 4 * c->V * nrhs;
    if (!din) {
      int rc = stage_in(c, in, field, sin_);
      if (rc) return rc;
      pin = sin_;
    }
    if (!dout) pout = sout;
  }
  int rc = apply_op<R>(c, op, pin, pout, nrhs, (R)shift, (cplx<R>*)c->ws_apply.ptr);
  if (rc) return rc;
  if (!dout) {
    WZ_CUDA_TRY(c, cudaMemcpyAsync(out, pout, field, cudaMemcpyDeviceToHost, c->stream));
    WZ_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  } else if (!din) {
    WZ_CUDA_TRY(c, cudaStreamSynchronize(c->stream));  // host input must stay valid until copied
  }
  return WZ_OK;
}


}  // namespace wz

using namespace wz;

namespace wz {

// Shared body of wz_solve and wz_solve_multishift: nb right-hand sides in b,
// nsys systems (x has nsys fields), system q solves (M^dag M + sh.of(q)) x_q =
// b[sh.src(q)].  Host buffers are staged through the context.
static int solve_common(wz_ctx* c, const void* b, int nb, void* x, const ShiftSpec& sh, int nsys, double tol,
                        int maxiter, unsigned flags, wz_solve_stats* stats, double* resid, const char* who) {
  const std::string name(who);
  if (!b || !x || nb < 0 || tol <= 0.0 || maxiter < 1) return set_error(c, WZ_EINVAL, name + ": bad argument");
  if (b == x) return set_error(c, WZ_EINVAL, name + ": b and x must not alias");
  if (c->nm > 1 && nb % c->nm) return set_error(c, WZ_EINVAL, name + ": nrhs must be a multiple of the members");
  const auto t0 = std::chrono::steady_clock::now();
  if (nsys == 0) {
    if (stats) *stats = wz_solve_stats{};
    return WZ_OK;
  }
  const size_t f1 = sizeof(cplx<double>) * 4 * (size_t)c->V;
  const size_t fb = f1 * nb, fx = f1 * nsys;
  const bool db = is_device_pointer(b), dx = is_device_pointer(x);
  const cplx<double>* pb = (const cplx<double>*)b;
  cplx<double>* px = (cplx<double>*)x;
  if (!db || !dx) {
    WZ_CUDA_TRY(c, c->ws_stage.reserve(fb + fx));
    cplx<double>* sb = (cplx<double>*)c->ws_stage.ptr;
    if (!db) {
      WZ_CUDA_TRY(c, cudaMemcpyAsync(sb, b, fb, cudaMemcpyHostToDevice, c->stream));
      pb = sb;
    }
    if (!dx) px = sb + 4L * c->V * nb;
  }
  const bool pc = (flags & WZ_SOLVE_PC) != 0;
  if (pc && !c->same_mass) return set_error(c, WZ_EINVAL, name + ": M0^-1 preconditioning needs one mass for all members");
  SolveOut o;
  int rc = (flags & WZ_SOLVE_MIXED) ? solve_impl<float>(c, pb, px, nsys, sh, tol, maxiter, pc, 0.1, &o)
                                    : solve_impl<double>(c, pb, px, nsys, sh, tol, maxiter, pc, 0.0, &o);
  if (rc != WZ_OK && rc != WZ_NOT_CONVERGED) return rc;
  if (resid) {
    std::vector<double> rel(nsys);
    int rc2 = true_residuals(c, pb, px, nsys, sh, rel.data());
    if (rc2) return rc2;
    memcpy(resid, rel.data(), sizeof(double) * nsys);
  }
  if (!dx) {
    WZ_CUDA_TRY(c, cudaMemcpyAsync(x, px, fx, cudaMemcpyDeviceToHost, c->stream));
  }
  WZ_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (stats) {
    stats->iterations = o.iterations;
    stats->total_iterations = o.total_iterations;
    stats->reliable_updates = o.reliable_updates;
    stats->converged = o.converged;
    stats->max_true_residual = o.max_true_residual;
    stats->site_applies = (double)(o.total_iterations + o.reliable_updates) * (double)c->V;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (rc == WZ_NOT_CONVERGED) set_error(c, rc, name + ": maxiter reached before tol");
  return rc;
}

}  // namespace wz

extern "C" {

int wz_supported_extent(int n) { return extent_supported(n) ? 1 : 0; }

}  // extern "C"

namespace wz {

// Context over nm lattices of the same extent (members); member 0 is the
// lattice of the single-lattice API.
int create_ctx(const wz_params* ps, int nm, void* stream, wz_ctx** out) {
  if (!ps || !out || nm < 1) return WZ_EINVAL;
  *out = nullptr;
  const wz_params* p = ps;
  const int T = p->dims[0], Z = p->dims[1], Y = p->dims[2], X = p->dims[3];
  if (T <= 0 || Z <= 0 || Y <= 0 || X <= 0 || (T % 2) != 0) return WZ_EINVAL;
  if (X != Y || !extent_supported(X) || !zt_supported(Z, T)) return WZ_EUNSUPPORTED;
  for (int i = 0; i < nm; ++i) {
    if (ps[i].r <= 0.0) return WZ_EINVAL;
    for (int d = 0; d < 4; ++d)
      if (ps[i].dims[d] != p->dims[d]) return WZ_EINVAL;
  }
  wz_ctx* c = new (std::nothrow) wz_ctx();
  if (!c) return WZ_ENOMEM;
  c->p = *p;
  c->nm = nm;
  c->mp.assign(ps, ps + nm);
  const double m2 = p->m_re * p->m_re + p->m_im * p->m_im;
  for (int i = 0; i < nm; ++i) {
    c->same_mass &= (ps[i].m_re * ps[i].m_re + ps[i].m_im * ps[i].m_im) == m2;
    c->same_mass &= ps[i].r == p->r && ps[i].M0 == p->M0;
  }
  c->T = T;
  c->Z = Z;
  c->Y = Y;
  c->X = X;
  c->V = (long)T * Z * Y * X;
  c->stream = (cudaStream_t)stream;
  cudaGetDevice(&c->device);
  for (DevBuf* b : {&c->ws_apply, &c->ws_stage, &c->ws_solver, &c->ws_red, &c->ws_force, &c->ws_rat}) {
    b->used = &c->ws_used;
    b->cap = &c->ws_cap;
  }
  // WZ_NO_GRAPHS=1 in the environment makes the solver launch its chunks
  // eagerly instead of through the cached CUDA graph (same kernels, same results)
  const char* ng = getenv("WZ_NO_GRAPHS");
  c->use_graphs = !(ng && ng[0] == '1');
  int rc = build_tables(c);
  if (rc == WZ_OK) {
    std::vector<SiteCoef<double>> kd(nm);
    std::vector<SiteCoef<float>> kf(nm);
    for (int i = 0; i < nm; ++i) {
      kd[i] = site_coef_of<double>(ps[i]);
      kf[i] = site_coef_of<float>(ps[i]);
    }
    const size_t nphi = (size_t)nm * c->V;
    cudaError_t e = cudaMalloc(&c->phi64, sizeof(cplx<double>) * nphi);
    if (e == cudaSuccess) e = cudaMalloc(&c->phi32, sizeof(cplx<float>) * nphi);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->phi64, 0, sizeof(cplx<double>) * nphi, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->phi32, 0, sizeof(cplx<float>) * nphi, c->stream);
    if (e == cudaSuccess) e = cudaMalloc(&c->k64, sizeof(SiteCoef<double>) * nm);
    if (e == cudaSuccess) e = cudaMalloc(&c->k32, sizeof(SiteCoef<float>) * nm);
    if (e == cudaSuccess) e = cudaMemcpy(c->k64, kd.data(), sizeof(SiteCoef<double>) * nm, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->k32, kf.data(), sizeof(SiteCoef<float>) * nm, cudaMemcpyHostToDevice);
    std::vector<int> ids(nm);
    for (int i = 0; i < nm; ++i) ids[i] = i;
    if (e == cudaSuccess) e = cudaMalloc(&c->mid, sizeof(int) * nm);
    if (e == cudaSuccess) e = cudaMemcpy(c->mid, ids.data(), sizeof(int) * nm, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMallocHost(&c->host_pinned, WZ_PINNED_BYTES);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    for (int i = 0; i < wz_ctx::kMaxBranches - 1; ++i) {
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->branch_stream[i], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaMalloc(&c->counters, WZ_NCOUNTERS * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(c->counters, 0, WZ_NCOUNTERS * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) rc = cuda_error(c, e, "create");
  }
  if (rc != WZ_OK) {
    wz_destroy(c);
    return rc;
  }
  *out = c;
  return WZ_OK;
}

// phi of member i (complex128 [T][Z][Y][X], host or device) -> FP64 and FP32 copies
int set_member_phi(wz_ctx* c, int i, const void* phi) {
  if (!c || !phi || i < 0 || i >= c->nm) return set_error(c, WZ_EINVAL, "set_phi: bad argument");
  const size_t n = sizeof(cplx<double>) * c->V;
  WZ_CUDA_TRY(c, cudaMemcpyAsync(c->phi64 + (long)i * c->V, phi, n, cudaMemcpyDefault, c->stream));
  count_launch();
  phi_to_f32_kernel<<<(unsigned)((c->V + 255) / 256 < 2048 ? (c->V + 255) / 256 : 2048), 256, 0, c->stream>>>(
      c->phi64 + (long)i * c->V, c->phi32 + (long)i * c->V, c->V);
  WZ_CUDA_TRY(c, cudaGetLastError());
  if (!is_device_pointer(phi)) WZ_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->phi_set = true;
  return WZ_OK;
}

}  // namespace wz

extern "C" {

int wz_create(const wz_params* p, void* stream, wz_ctx** out) { return create_ctx(p, 1, stream, out); }

int wz_destroy(wz_ctx* c) {
  if (!c) return WZ_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  if (c->t64.block) cudaFree(c->t64.block);
  if (c->t32.block) cudaFree(c->t32.block);
  if (c->phi64) cudaFree(c->phi64);
  if (c->phi32) cudaFree(c->phi32);
  if (c->k64) cudaFree(c->k64);
  if (c->k32) cudaFree(c->k32);
  if (c->mid) cudaFree(c->mid);
  if (c->host_pinned) cudaFreeHost(c->host_pinned);
  for (auto& g : c->solver_graph) g.release();
  c->traj_graph.release();
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->cap_stream2) cudaStreamDestroy(c->cap_stream2);
  for (int i = 0; i < wz_ctx::kMaxBranches - 1; ++i) {
    if (c->branch_stream[i]) cudaStreamDestroy(c->branch_stream[i]);
    if (c->ev_join[i]) cudaEventDestroy(c->ev_join[i]);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->counters) cudaFree(c->counters);
  c->ws_apply.release();
  c->ws_stage.release();
  c->ws_solver.release();
  c->ws_red.release();
  c->ws_force.release();
  c->ws_rat.release();
  delete c;
  return WZ_OK;
}

const char* wz_last_error(const wz_ctx* c) { return c ? c->err.c_str() : "null context"; }

int wz_set_workspace_limit(wz_ctx* c, size_t bytes) {
  if (!c) return WZ_EINVAL;
  c->ws_cap = bytes;
  return WZ_OK;
}

size_t wz_workspace_bytes(const wz_ctx* c) { return c ? c->ws_used : 0; }

int wz_set_phi(wz_ctx* c, const void* phi) { return set_member_phi(c, 0, phi); }

int wz_apply(wz_ctx* c, int op, int dtype, const void* in, void* out, int nrhs, double shift) {
  if (!c) return WZ_EINVAL;
  if (!in || !out || nrhs < 0) return set_error(c, WZ_EINVAL, "wz_apply: bad argument");
  if (op < WZ_OP_M || op > WZ_OP_D) return set_error(c, WZ_EINVAL, "wz_apply: unknown op");
  if (nrhs == 0) return WZ_OK;
  if (c->nm > 1 && nrhs % c->nm) return set_error(c, WZ_EINVAL, "wz_apply: nrhs must be a multiple of the members");
  if (!c->same_mass && op >= WZ_OP_M0INV && op != WZ_OP_DSLASH && op != WZ_OP_D1 && op != WZ_OP_D)
    return set_error(c, WZ_EINVAL, "wz_apply: M0^-1 operators need one mass for all members");
  if (dtype == WZ_C128) return apply_typed<double>(c, op, in, out, nrhs, shift);
  if (dtype == WZ_C64) return apply_typed<float>(c, op, in, out, nrhs, shift);
  return set_error(c, WZ_EINVAL, "wz_apply: unknown dtype");
}

int wz_solve(wz_ctx* c, const void* b, void* x, int nrhs, double shift, double tol, int maxiter, unsigned flags,
             wz_solve_stats* stats, double* resid) {
  if (!c) return WZ_EINVAL;
  if (shift < 0.0) return set_error(c, WZ_EINVAL, "wz_solve: bad argument");
  return solve_common(c, b, nrhs, x, single_shift(shift), nrhs, tol, maxiter, flags, stats, resid, "wz_solve");
}

int wz_solve_multishift(wz_ctx* c, const void* b, void* x, int nrhs, int nshift, const double* shifts, double tol,
                        int maxiter, unsigned flags, wz_solve_stats* stats, double* resid) {
  if (!c) return WZ_EINVAL;
  if (nshift < 1 || nshift > WZ_SHIFT_MAX || !shifts)
    return set_error(c, WZ_EINVAL, "wz_solve_multishift: 1 <= nshift <= 64 shifts expected");
  if (c->nm > 1 && nrhs % c->nm)
    return set_error(c, WZ_EINVAL, "wz_solve_multishift: nrhs must be a multiple of the members");
  ShiftSpec sh;
  sh.d = nshift;
  sh.inner = c->nm > 1 ? nrhs / c->nm : nrhs;
  for (int i = 0; i < nshift; ++i) {
    if (!(shifts[i] >= 0.0)) return set_error(c, WZ_EINVAL, "wz_solve_multishift: shifts must be >= 0");
    sh.beta[i] = shifts[i];
  }
  if (nrhs == 0) sh.inner = 1;
  return solve_common(c, b, nrhs, x, sh, nrhs * nshift, tol, maxiter, flags, stats, resid, "wz_solve_multishift");
}

unsigned long long wz_kernel_launches(void) { return g_launches.load(); }

int wz_probe_begin(int kind, int real_bytes) {
  Probe& p = g_probe;
  if (kind < PK_ZT || kind > PK_RU_P5 || (real_bytes != 4 && real_bytes != 8)) return WZ_EINVAL;
  if (!p.d_blocks && cudaMalloc(&p.d_blocks, sizeof(unsigned long long)) != cudaSuccess) return WZ_ENOMEM;
  if (p.ev.empty()) {
    // enough pairs for every launch of a kernel class in one 16^4 x 12 RHS
    // solve (about 24k zt launches); launches past the pool are not timed
    p.ev.resize(2 * 32768);
    for (auto& e : p.ev)
      if (cudaEventCreate(&e) != cudaSuccess) return WZ_ECUDA;
  }
  if (cudaMemset(p.d_blocks, 0, sizeof(unsigned long long)) != cudaSuccess) return WZ_ECUDA;
  p.kind = kind;
  p.real_bytes = real_bytes;
  p.recorded = 0;
  p.launches = 0;
  p.bytes_per_block = 0.0;
  p.active = 1;
  return WZ_OK;
}

int wz_probe_end(wz_probe_result* out) {
  Probe& p = g_probe;
  if (!p.active) return WZ_EINVAL;
  p.active = 0;
  if (cudaDeviceSynchronize() != cudaSuccess) return WZ_ECUDA;
  double ms = 0.0;
  for (int i = 0; i < p.recorded; ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p.ev[2 * i], p.ev[2 * i + 1]) != cudaSuccess) return WZ_ECUDA;
    ms += t;
  }
  unsigned long long bytes = 0;
  if (cudaMemcpy(&bytes, p.d_blocks, sizeof(bytes), cudaMemcpyDeviceToHost) != cudaSuccess) return WZ_ECUDA;
  if (out) {
    out->launches = p.launches;
    out->timed_launches = p.recorded;
    out->total_ms = ms;
    out->bytes = (double)bytes;
  }
  return WZ_OK;
}

}  // extern "C"
