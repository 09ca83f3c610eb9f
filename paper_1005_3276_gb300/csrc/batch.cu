// Batches of independent lattices (replicas of uneven extent and coupling).
//
// The lattices of a batch are grouped by extent.  Each group is one context
// whose "members" share the momentum tables and whose fields carry the member
// index outermost, so one kernel launch per pass covers every right-hand side
// of every lattice of the group (couplings and phi are looked up per member
// inside the kernels).  Groups run concurrently, each on its own stream with
// its own cached solver graph, driven by one host thread per group.
#include <algorithm>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "apply_impl.cuh"
#include "hmc.h"
#include "solver.h"
#include "wz_ctx.h"


using namespace wz;

struct wz_batch {
  int n = 0;
  std::vector<wz_ctx*> groups;
  std::vector<cudaStream_t> streams;
  std::vector<std::vector<int>> members;  // lattice indices of each group, in member order
  std::vector<int> group_of, member_of;   // per lattice
  std::string err;
};

static int batch_error(wz_batch* b, int code, const std::string& m) {
  if (b) b->err = m;
  return code;
}

extern "C" {

int wz_batch_create(const wz_params* ps, int n, void* stream, wz_batch** out) {
  (void)stream;
  if (!ps || n < 1 || !out) return WZ_EINVAL;
  *out = nullptr;
  wz_batch* b = new (std::nothrow) wz_batch();
  if (!b) return WZ_ENOMEM;
  b->n = n;
  b->group_of.assign(n, -1);
  b->member_of.assign(n, -1);
  std::map<std::vector<int>, int> key;
  for (int i = 0; i < n; ++i) {
    std::vector<int> d(ps[i].dims, ps[i].dims + 4);
    auto it = key.find(d);
    int gi;
    if (it == key.end()) {
      gi = (int)b->members.size();
      key[d] = gi;
      b->members.emplace_back();
    } else {
      gi = it->second;
    }
    b->group_of[i] = gi;
    b->member_of[i] = (int)b->members[gi].size();
    b->members[gi].push_back(i);
  }
  for (size_t gi = 0; gi < b->members.size(); ++gi) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      wz_batch_destroy(b);
      return WZ_ECUDA;
    }
    b->streams.push_back(s);
    std::vector<wz_params> gp;
    for (int i : b->members[gi]) gp.push_back(ps[i]);
    wz_ctx* c = nullptr;
    int rc = create_ctx(gp.data(), (int)gp.size(), s, &c);
    if (rc) {
      wz_batch_destroy(b);
      return rc;
    }
    // Philox key offsets: every lattice draws as lattice i of the batch
    cudaMemcpy(c->mid, b->members[gi].data(), sizeof(int) * gp.size(), cudaMemcpyHostToDevice);
    b->groups.push_back(c);
  }
  *out = b;
  return WZ_OK;
}

int wz_batch_destroy(wz_batch* b) {
  if (!b) return WZ_OK;
  for (wz_ctx* c : b->groups) wz_destroy(c);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  delete b;
  return WZ_OK;
}

const char* wz_batch_last_error(const wz_batch* b) { return b ? b->err.c_str() : "null batch"; }

int wz_batch_size(const wz_batch* b) { return b ? b->n : 0; }

int wz_batch_groups(const wz_batch* b) { return b ? (int)b->groups.size() : 0; }

int wz_batch_set_phi(wz_batch* b, int i, const void* phi) {
  if (!b || i < 0 || i >= b->n || !phi) return batch_error(b, WZ_EINVAL, "wz_batch_set_phi: bad argument");
  wz_ctx* c = b->groups[b->group_of[i]];
  int rc = set_member_phi(c, b->member_of[i], phi);
  if (rc) return batch_error(b, rc, c->err);
  cudaStreamSynchronize(c->stream);
  return WZ_OK;
}

int wz_batch_get_phi(wz_batch* b, int i, void* phi) {
  if (!b || i < 0 || i >= b->n || !phi) return batch_error(b, WZ_EINVAL, "wz_batch_get_phi: bad argument");
  wz_ctx* c = b->groups[b->group_of[i]];
  if (cudaMemcpyAsync(phi, c->phi64 + (long)b->member_of[i] * c->V, sizeof(cplx<double>) * c->V, cudaMemcpyDefault,
                      c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return batch_error(b, WZ_ECUDA, "wz_batch_get_phi: copy failed");
  return WZ_OK;
}

int wz_batch_solve(wz_batch* b, const void* const* bs, void* const* xs, int nrhs, double tol, int maxiter,
                   unsigned flags, wz_solve_stats* st) {
  if (!b || !bs || !xs || nrhs < 1 || tol <= 0.0 || maxiter < 1)
    return batch_error(b, WZ_EINVAL, "wz_batch_solve: bad argument");
  if (flags & WZ_SOLVE_PC) return batch_error(b, WZ_EINVAL, "wz_batch_solve: no M0^-1 preconditioning in batches");
  const int ng = (int)b->groups.size();
  std::vector<int> rcs(ng, WZ_OK);
  std::vector<SolveOut> outs(ng);
  auto run = [&](int gi) {
    wz_ctx* c = b->groups[gi];
    const int nm = c->nm;
    const size_t f = sizeof(cplx<double>) * 4 * (size_t)c->V * nrhs;  // one lattice's nrhs fields
    int rc = c->ws_stage.reserve(2 * f * nm) == cudaSuccess ? WZ_OK : WZ_ENOMEM;
    if (rc) {
      rcs[gi] = rc;
      return;
    }
    char* sb = (char*)c->ws_stage.ptr;
    char* sx = sb + f * nm;
    for (int j = 0; j < nm; ++j) {
      const int i = b->members[gi][j];
      if (cudaMemcpyAsync(sb + f * j, bs[i], f, cudaMemcpyDefault, c->stream) != cudaSuccess) rc = WZ_ECUDA;
    }
    if (!rc)
      rc = (flags & WZ_SOLVE_MIXED)
               ? solve_impl<float>(c, (const cplx<double>*)sb, (cplx<double>*)sx, nrhs * nm, single_shift(0.0), tol,
                                   maxiter,
                                   false, 0.1, &outs[gi])
               : solve_impl<double>(c, (const cplx<double>*)sb, (cplx<double>*)sx, nrhs * nm, single_shift(0.0), tol,
                                   maxiter,
                                    false, 0.0, &outs[gi]);
    if (rc == WZ_OK || rc == WZ_NOT_CONVERGED) {
      for (int j = 0; j < nm; ++j) {
        const int i = b->members[gi][j];
        if (cudaMemcpyAsync(xs[i], sx + f * j, f, cudaMemcpyDefault, c->stream) != cudaSuccess) rc = WZ_ECUDA;
      }
      if (cudaStreamSynchronize(c->stream) != cudaSuccess) rc = WZ_ECUDA;
    }
    rcs[gi] = rc;
  };
  std::vector<std::thread> th;
  for (int gi = 1; gi < ng; ++gi) th.emplace_back(run, gi);
  run(0);
  for (auto& t : th) t.join();
  SolveOut tot;
  int worst = WZ_OK;
  double site_applies = 0.0;
  for (int gi = 0; gi < ng; ++gi) {
    if (rcs[gi] != WZ_OK && rcs[gi] != WZ_NOT_CONVERGED) return batch_error(b, rcs[gi], b->groups[gi]->err);
    if (rcs[gi] == WZ_NOT_CONVERGED) worst = WZ_NOT_CONVERGED;
    site_applies += (double)(outs[gi].total_iterations + outs[gi].reliable_updates) * (double)b->groups[gi]->V;
    tot.iterations = std::max(tot.iterations, outs[gi].iterations);
    tot.total_iterations += outs[gi].total_iterations;
    tot.reliable_updates += outs[gi].reliable_updates;
    tot.converged += outs[gi].converged;
    tot.max_true_residual = std::max(tot.max_true_residual, outs[gi].max_true_residual);
  }
  if (st) {
    st->iterations = tot.iterations;
    st->total_iterations = tot.total_iterations;
    st->reliable_updates = tot.reliable_updates;
    st->converged = tot.converged;
    st->max_true_residual = tot.max_true_residual;
    st->site_applies = site_applies;
    st->seconds = 0.0;
  }
  return worst;
}

int wz_batch_trajectory(wz_batch* b, const wz_hmc_params* h, wz_traj_stats* st) {
  if (!b || !h || h->npf < 0 || h->nsteps < 1 || h->tol <= 0.0 || h->tau <= 0.0)
    return batch_error(b, WZ_EINVAL, "wz_batch_trajectory: bad argument");
  const int ng = (int)b->groups.size();
  std::vector<int> rcs(ng, WZ_OK);
  std::vector<std::vector<wz_traj_stats>> gst(ng);
  auto run = [&](int gi) {
    wz_ctx* c = b->groups[gi];
    gst[gi].resize(c->nm);
    rcs[gi] = trajectory_impl(c, h, gst[gi].data());
  };
  std::vector<std::thread> th;
  for (int gi = 1; gi < ng; ++gi) th.emplace_back(run, gi);
  run(0);
  for (auto& t : th) t.join();
  for (int gi = 0; gi < ng; ++gi) {
    if (rcs[gi]) return batch_error(b, rcs[gi], b->groups[gi]->err);
    for (int j = 0; st && j < b->groups[gi]->nm; ++j) st[b->members[gi][j]] = gst[gi][j];
  }
  return WZ_OK;
}

}  // extern "C"
