// Internal context of the library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/wz.h"
#include "wz_kernels.cuh"

namespace wz {

// Momentum-space tables of one precision (a0 of the hot path, Sec. 3.1):
//   hV  = h(p)/V, hdV = h(p)/(den(p) V), dV = 1/(den(p) V),
//   h = 2/(omega + b), den = h^2 sum sin^2 p + |m|^2  (Sec. 7.3)
// plus per-axis sin p tables and the antiperiodic twist cos/sin(pi t/T).
template <typename R> struct Tables {
  R* hV = nullptr;
  R* hdV = nullptr;
  R* dV = nullptr;
  R* d2sV = nullptr;  // scalar D2(p)/V, periodic grid (Eq. acws)
  R* ksV = nullptr;   // scalar K(p)/V = (1 - D2/2)/V
  R* w1V = nullptr;   // 1/(omega(p) V), fermion grid: D1(p) = i gamma.sin p / omega
  R* w1sV = nullptr;  // 1/(omega(p) V), periodic (scalar) grid
  R* d2fV = nullptr;  // D2(p)/V = (1 - b/omega)/V, fermion grid: overlap D = D1 + D2
  R* sinT = nullptr;
  R* sinZ = nullptr;
  R* sinY = nullptr;
  R* sinX = nullptr;
  R* twc = nullptr;
  R* tws = nullptr;
  R* twc1 = nullptr;  // identity twist (cos = 1, sin = 0): xy passes of periodic scalar fields
  R* tws0 = nullptr;
  void* block = nullptr;  // single allocation holding everything above
};

// A device buffer that only grows.  The buffers of one context share a byte
// count and an optional cap on it (wz_set_workspace_limit): a growth beyond
// the cap is refused as cudaMalloc refuses one beyond free memory, before the
// old buffer is released.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  size_t* used = nullptr;       // the context's workspace bytes (may be null)
  const size_t* cap = nullptr;  // the context's cap, 0 = none (may be null)
  cudaError_t reserve(size_t n) {
    if (n <= bytes) return cudaSuccess;
    if (used && cap && *cap && *used - bytes + n > *cap) return cudaErrorMemoryAllocation;
    if (ptr) cudaFree(ptr);
    if (used) *used -= bytes;
    ptr = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&ptr, n);
    if (e == cudaSuccess) {
      bytes = n;
      if (used) *used += n;
    } else {
      cudaGetLastError();  // an allocation failure is not sticky: keep it out of later launch checks
    }
    return e;
  }
  void release() {
    if (ptr) cudaFree(ptr);
    if (used) *used -= bytes;
    ptr = nullptr;
    bytes = 0;
  }
};

// Cached CUDA graph of the solver's chunk loop and what it was captured for.
struct SolverGraphKey {
  int nrhs;
  int pc;
  int maxiter;
  double delta2;
  void* ws;
  size_t ws_bytes;
  const void* phi64;
  const void* phi32;
  int gsz;      // right-hand sides per group
  int nbranch;  // streams the groups alternate between
  int pdl;      // kernels launched with programmatic stream serialization
  int tpb;      // tiles per block of the FP32 zt passes (0: resident blocks)
};
struct SolverGraph {
  SolverGraphKey key{};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned long long body_launches = 0;
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    key = SolverGraphKey{};
  }
};

// Cached CUDA graph of a whole HMC trajectory and what it was captured for.
struct TrajGraphKey {
  double tau, tol;
  int nsteps, integrator, npf, maxiter;
  unsigned flags;
  unsigned long long seed;
  unsigned long long rational;  // hash of the rational action and heatbath (RHMC), else of none
  void *ws_force, *ws_solver, *ws_apply;
  size_t b_force, b_solver, b_apply;
};
struct TrajGraph {
  TrajGraphKey key{};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned long long outer_launches = 0, body_launches = 0, body_launches_h = 0;
  int force_evals = 0;
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    key = TrajGraphKey{};
  }
};

}  // namespace wz

struct wz_ctx {
  wz_params p{};                 // member 0 (the lattice of a single-lattice context)
  int nm = 1;                    // members: lattices of the same extent sharing the tables
  std::vector<wz_params> mp;     // parameters per member
  bool same_mass = true;         // all members share |m| (the M0^-1 tables depend on it)
  wz::SiteCoef<double>* k64 = nullptr;  // couplings per member (device)
  wz::SiteCoef<float>* k32 = nullptr;
  int* mid = nullptr;            // Philox key offset of each member (device; 0..nm-1, batch: lattice index)
  int T = 0, Z = 0, Y = 0, X = 0;
  long V = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  std::string err;

  wz::Tables<double> t64;
  wz::Tables<float> t32;
  wz::cplx<double>* phi64 = nullptr;  // [member][T][Z][Y][X]
  wz::cplx<float>* phi32 = nullptr;
  bool phi_set = false;

  wz::DevBuf ws_apply;    // momentum / M psi intermediates of the apply
  wz::DevBuf ws_stage;    // staging of host buffers
  wz::DevBuf ws_solver;   // solver vectors
  wz::DevBuf ws_red;      // reduction partials and per-RHS scalars
  wz::DevBuf ws_force;    // force / HMC fields
  wz::DevBuf ws_rat;      // shifted solutions of a rational apply
  size_t ws_used = 0;     // bytes held by the six workspaces above
  size_t ws_cap = 0;      // cap on ws_used (wz_set_workspace_limit), 0 = none
  // small pinned block for scalar read-back: [0, WZ_PINNED_SCRATCH_OFFSET) holds
  // the solver's per-RHS state, the rest is scratch for other reductions
  void* host_pinned = nullptr;
  // solver graphs and their capture stream
  bool use_graphs = true;
  bool pdl_capture_failed = false;             // a graph capture with dependent launches failed: plain launches
  cudaStream_t cap_stream = nullptr;
  cudaStream_t cap_stream2 = nullptr;          // body of solver loops inside a trajectory capture
  // extra branches of a solver chunk (RHS groups on concurrent streams)
  static const int kMaxBranches = 4;
  cudaStream_t branch_stream[kMaxBranches - 1] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[kMaxBranches - 1] = {};
  // device counters: [0] iterations, [1] reliable updates, [2] trips of solver
  // loops, [3] trajectory number, [4] trips of the heatbath solver loop of an
  // RHMC trajectory, [7] sticky device error word (a bounded wait ran out)
  unsigned long long* counters = nullptr;
  int trip_slot = 2;                           // counter of the trips of an inline solver loop
  unsigned long long inline_body_launches = 0; // kernels per trip of an inline solver loop
  wz::SolverGraph solver_graph[4];             // [mixed, FP64] x [plain, preconditioned]
  wz::TrajGraph traj_graph;
};

#define WZ_PINNED_BYTES (256 * 1024)
#define WZ_NCOUNTERS 8
#define WZ_COUNTER_DEVICE_ERROR 7
#define WZ_PINNED_SCRATCH_OFFSET (128 * 1024)

namespace wz {

int set_error(wz_ctx* c, int code, const std::string& msg);
int cuda_error(wz_ctx* c, cudaError_t e, const char* where);
bool is_device_pointer(const void* p);

// apply entry (templated on precision), defined in apply_impl.cuh
template <typename R>
int apply_op(wz_ctx* c, int op, const cplx<R>* in, cplx<R>* out, int nrhs, R shift, cplx<R>* ws);
template <typename R> size_t apply_ws_bytes(const wz_ctx* c, int op, int nrhs);

template <typename R> const Tables<R>& tables(const wz_ctx* c);
template <> inline const Tables<double>& tables<double>(const wz_ctx* c) { return c->t64; }
template <> inline const Tables<float>& tables<float>(const wz_ctx* c) { return c->t32; }
template <typename R> const SiteCoef<R>* karr_of(const wz_ctx* c);
template <> inline const SiteCoef<double>* karr_of<double>(const wz_ctx* c) { return c->k64; }
template <> inline const SiteCoef<float>* karr_of<float>(const wz_ctx* c) { return c->k32; }
template <typename R> const cplx<R>* phi_of(const wz_ctx* c);
template <> inline const cplx<double>* phi_of<double>(const wz_ctx* c) { return c->phi64; }
template <> inline const cplx<float>* phi_of<float>(const wz_ctx* c) { return c->phi32; }

bool extent_supported(int n);
bool zt_supported(int nz, int nt);
int create_ctx(const wz_params* ps, int nm, void* stream, wz_ctx** out);
int set_member_phi(wz_ctx* c, int i, const void* phi);

}  // namespace wz

#define WZ_CUDA_TRY(c, expr)                                  \
  do {                                                        \
    cudaError_t _e = (expr);                                  \
    if (_e != cudaSuccess) return wz::cuda_error(c, _e, #expr); \
  } while (0)
