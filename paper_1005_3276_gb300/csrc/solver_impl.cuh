// Host sequencing of the fused CG solver (see wz_cg.cuh for the algorithm).
//
// The iteration passes are issued in chunks of K iterations followed by one
// reliable-update block; every kernel gates itself per right-hand side on the
// device state, so a chunk is a fixed launch sequence and the host only reads
// the per-RHS state between chunks to see whether all have finished.
#pragma once
#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "apply_impl.cuh"
#include "solver.h"
#include "wz_cg.cuh"

namespace wz {

// Workspace layout (bytes) for a solve with iteration type RI.
template <typename RI> struct SolverWS {
  size_t field_ri, field64, off_xlo, off_r, off_p, off_A, off_C, off_A64, off_C64, off_bt, off_xt, off_part,
      off_st, off_trips, total;
  SolverWS(long V, int nrhs, int nblk, bool pc) {
    field_ri = sizeof(cplx<RI>) * 4 * (size_t)V * nrhs;
    field64 = sizeof(cplx<double>) * 4 * (size_t)V * nrhs;
    size_t o = 0;
    auto take = [&](size_t n) {
      size_t r = o;
      o += (n + 255) & ~size_t(255);
      return r;
    };
    off_xlo = take(field_ri);
    off_r = take(field_ri);
    off_p = take(field_ri);
    off_A = take(field_ri);
    off_C = take(field_ri);
    off_A64 = take(field64);
    off_C64 = take(field64);
    off_bt = take(field64);  // right-hand side of the recursion (b, or b~ when preconditioned)
    off_xt = take(field64);  // FP64 solution of the recursion (x, or x~)
    off_part = take(sizeof(double) * 3 * (size_t)nrhs * (nblk > 64 ? nblk : 64));
    off_st = take(sizeof(RhsState) * nrhs);
    off_trips = take(sizeof(int));
    total = o;
  }
};

// b, x: FP64 device fields.  RI: iteration precision (float: mixed, double: FP64).
// nrhs systems; system q solves (M^dag M + sh.of(q)) x_q = b[sh.src(q)].
template <typename RI>
int solve_impl(wz_ctx* c, const cplx<double>* b, cplx<double>* x, int nrhs, const ShiftSpec& sh, double tol,
               int maxiter, bool pc, double delta, SolveOut* out, bool inline_capture) {
  if (inline_capture && pc) return set_error(c, WZ_EINVAL, "preconditioned solves cannot be captured inline");
  const int L = c->X;
  const int TZ = c->T * c->Z;
  const int nblk = xy_nblk(L, TZ);
  SolverWS<RI> W(c->V, nrhs, nblk, pc);
  WZ_CUDA_TRY(c, c->ws_solver.reserve(W.total));
  char* base = (char*)c->ws_solver.ptr;
  cplx<RI>* xlo = (cplx<RI>*)(base + W.off_xlo);
  cplx<RI>* r = (cplx<RI>*)(base + W.off_r);
  cplx<RI>* p = (cplx<RI>*)(base + W.off_p);
  cplx<RI>* A = (cplx<RI>*)(base + W.off_A);
  cplx<RI>* Cb = (cplx<RI>*)(base + W.off_C);
  cplx<double>* A64 = (cplx<double>*)(base + W.off_A64);
  cplx<double>* C64 = (cplx<double>*)(base + W.off_C64);
  const int npart = nblk > 64 ? nblk : 64;
  double* part3 = (double*)(base + W.off_part);
  double* part5 = part3 + (size_t)nrhs * npart;
  double* partR = part5 + (size_t)nrhs * npart;
  RhsState* st = (RhsState*)(base + W.off_st);
  cudaStream_t s = c->stream;
  const long n_per_rhs = 4L * c->V;

  // preconditioned problem: b~ = (M0^-1)^dag b, solve for x~ = M0 x
  cplx<double>* bs = (cplx<double>*)(base + W.off_bt);
  cplx<double>* xs = (cplx<double>*)(base + W.off_xt);
  count_launch();
  gather_rhs<<<dim3(64, nrhs), 256, 0, s>>>(b, bs, n_per_rhs, sh);
  WZ_CUDA_TRY(c, cudaGetLastError());
  if (pc) {
    int rc = apply_op<double>(c, WZ_OP_M0INV_DAG, bs, bs, nrhs, 0.0, A64);
    if (rc) return rc;
  }

  WZ_CUDA_TRY(c, cudaMemsetAsync(xs, 0, W.field64, s));
  count_launch(2);
  cg_init<RI><<<dim3(64, nrhs), 256, 0, s>>>(bs, r, xlo, p, n_per_rhs, partR, 64);
  WZ_CUDA_TRY(c, cudaGetLastError());
  cg_scalar_init<<<nrhs, 32, 0, s>>>(st, partR, 64, tol * tol, sh);
  WZ_CUDA_TRY(c, cudaGetLastError());

  const int gate_stride = sizeof(RhsState) / sizeof(int);
  const int* gate_run = &st->run;
  const int* gate_ru = &st->ru;

  CGArgs<RI, RI> ga{};
  ga.A = A;
  ga.Cb = Cb;
  ga.p = p;
  ga.r = r;
  ga.x = xlo;
  ga.phi = phi_of<RI>(c);
  ga.kArr = karr_of<RI>(c);
  ga.rpm = rhs_per_member(c, nrhs);
  ga.Z = c->Z;
  ga.twc = tables<RI>(c).twc;
  ga.tws = tables<RI>(c).tws;
  ga.shifted = sh.any();
  ga.st = st;
  ga.nblk = nblk;
  ga.TZ = TZ;
  ga.gate_ru = 0;

  CGArgs<double, RI> ra{};
  ra.A = A64;
  ra.Cb = C64;
  ra.p = xs;  // x_hi
  ra.lo_x = xlo;
  ra.lo_p = p;
  ra.lo_r = r;
  ra.b = bs;
  ra.phi = c->phi64;
  ra.kArr = c->k64;
  ra.rpm = ga.rpm;
  ra.Z = c->Z;
  ra.twc = c->t64.twc;
  ra.tws = c->t64.tws;
  ra.shifted = ga.shifted;
  ra.st = st;
  ra.nblk = nblk;
  ra.TZ = TZ;
  ra.gate_ru = 1;

  ZTArgs<RI> z1 = zt_args<RI>(c, RI(1)), z2 = zt_args<RI>(c, RI(-1));
  z1.A = z2.A = A;
  z1.gate = z2.gate = gate_run;
  z1.gate_stride = z2.gate_stride = gate_stride;
  z1.fail = z2.fail = &st->status;
  z1.fail_stride = z2.fail_stride = gate_stride;
  ZTArgs<double> y1 = zt_args<double>(c, 1.0), y2 = zt_args<double>(c, -1.0);
  y1.A = y2.A = A64;
  y1.gate = y2.gate = gate_ru;
  y1.gate_stride = y2.gate_stride = gate_stride;
  y1.fail = y2.fail = &st->status;
  y1.fail_stride = y2.fail_stride = gate_stride;
  const int mul1 = pc ? ZT_M0INV : ZT_DSLASH, mul2 = pc ? ZT_M0INV_DAG : ZT_DSLASH;

  const double delta2 = delta * delta;
  const int K = 8;
  RhsState* hst = (RhsState*)c->host_pinned;
  if (sizeof(RhsState) * nrhs > WZ_PINNED_SCRATCH_OFFSET - 64) return set_error(c, WZ_EINVAL, "too many right-hand sides");
  cudaError_t e;
#define WZ_RUN(...)                                                 \
  do {                                                              \
    e = (__VA_ARGS__);                                              \
    if (e != cudaSuccess) return cuda_error(c, e, #__VA_ARGS__);    \
  } while (0)
  const int max_chunks = maxiter / K + 64;

  // Right-hand sides are iterated in groups of gsz: the five passes of one
  // group run back to back, so its working set (five spinor fields per RHS)
  // can stay in L2 between producer and consumer passes.  The group size is
  // chosen per solve shape by timing the candidates (autotune_group below).
  int gsz = nrhs;
  // With nbranch > 1 the groups alternate between nbranch streams (parallel
  // branches of the graph), each group with its own scalar and reliable-update
  // kernels, so that the passes of one group overlap those of the others.
  int nbranch = 1;
  // Programmatic dependent launch of the chain's kernels (each kernel's launch
  // and block set-up overlap the tail of the one before it on its stream);
  // chosen with the groups, never while the probe brackets single launches.
  bool pdl = false;
  auto set_pdl = [&](bool on) {
    pdl = on && !g_probe.active;
    ga.pdl = ra.pdl = z1.pdl = z2.pdl = y1.pdl = y2.pdl = pdl ? 1 : 0;
  };
  // Tiles per block of the FP32 zt passes of the mixed solver (their persistent
  // grid: 0 starts as many blocks as are resident; k > 0 at most ceil(tiles / k)
  // blocks, which leaves SMs to the concurrent groups).  The FP64 passes are
  // bound by arithmetic and keep every resident block.
  auto set_ztpb = [&](int k) { z1.tpb = z2.tpb = sizeof(RI) == 4 ? k : 0; };

  // iteration counters of the chunks (off while the tuner times candidates)
  unsigned long long* cnt = c->counters;

  // K iterations and one reliable-update block of the right-hand sides [r0, r0 + ng)
  auto issue_group_chunk = [&](int r0, int ng, cudaStream_t q) -> cudaError_t {
    cudaError_t e2;
#define WZ_Q(...)                          \
  do {                                     \
    e2 = (__VA_ARGS__);                    \
    if (e2 != cudaSuccess) return e2;      \
  } while (0)
    for (int k = 0; k < K; ++k) {
      CGArgs<RI, RI> a1 = ga;
      a1.rhs0 = r0;
      WZ_Q(launch_cg<RI, RI>(L, pc, CG_P1, a1, ng, q));
      ZTArgs<RI> zz1 = z1;
      zz1.rhs0 = r0;
      WZ_Q(launch_zt<RI>(c->Z, c->T, mul1, zz1, ng, q));
      CGArgs<RI, RI> a3 = ga;
      a3.rhs0 = r0;
      a3.part_out = part3;
      WZ_Q(launch_cg<RI, RI>(L, pc, CG_P3, a3, ng, q));
      ZTArgs<RI> zz2 = z2;
      zz2.rhs0 = r0;
      WZ_Q(launch_zt<RI>(c->Z, c->T, mul2, zz2, ng, q));
      CGArgs<RI, RI> a5 = ga;
      a5.rhs0 = r0;
      a5.part_in = part3;
      a5.part_out = part5;
      WZ_Q(launch_cg<RI, RI>(L, pc, CG_P5, a5, ng, q));
      count_launch();
      WZ_Q(launch_k(pdl, cg_scalar_iter, dim3(ng), dim3(32), 0, q, st + r0, part5 + (long)r0 * nblk,
                    part3 + (long)r0 * nblk, nblk, delta2, maxiter, cnt));
    }
    CGArgs<double, RI> u1 = ra;
    u1.rhs0 = r0;
    WZ_Q(launch_cg<double, RI>(L, pc, RU_P1, u1, ng, q));
    ZTArgs<double> w1 = y1;
    w1.rhs0 = r0;
    WZ_Q(launch_zt<double>(c->Z, c->T, mul1, w1, ng, q));
    CGArgs<double, double> u3{};
    u3.A = A64;
    u3.Cb = C64;
    u3.p = xs;
    u3.phi = c->phi64;
    u3.kArr = c->k64;
    u3.rpm = ga.rpm;
    u3.Z = c->Z;
    u3.twc = c->t64.twc;
    u3.tws = c->t64.tws;
    u3.shifted = ga.shifted;
    u3.st = st;
    u3.nblk = nblk;
    u3.TZ = TZ;
    u3.gate_ru = 1;
    u3.rhs0 = r0;
    u3.pdl = ra.pdl;
    WZ_Q(launch_cg<double, double>(L, pc, CG_P3, u3, ng, q));
    ZTArgs<double> w2 = y2;
    w2.rhs0 = r0;
    WZ_Q(launch_zt<double>(c->Z, c->T, mul2, w2, ng, q));
    CGArgs<double, RI> u5 = ra;
    u5.rhs0 = r0;
    u5.part_out = partR;
    WZ_Q(launch_cg<double, RI>(L, pc, RU_P5, u5, ng, q));
    count_launch();
    WZ_Q(launch_k(pdl, cg_scalar_ru, dim3(ng), dim3(32), 0, q, st + r0, partR + (long)r0 * nblk, nblk, maxiter,
                  cnt));
#undef WZ_Q
    return cudaSuccess;
  };

  // one chunk: K iterations and one reliable-update block, all gated on the device
  auto issue_chunk = [&](cudaStream_t q) -> cudaError_t {
    cudaError_t e2;
    if (nbranch > 1 && gsz < nrhs) {
      // The kernel probe times launches one at a time: the same per-group
      // launches (each group with its own scalar and reliable-update kernels)
      // in the same order, all on q, so that every launch of a class is
      // bracketed alone and the class counts are those of the timed solve.
      if (g_probe.active) {
        for (int r0 = 0; r0 < nrhs; r0 += gsz) {
          const int ng = nrhs - r0 < gsz ? nrhs - r0 : gsz;
          if ((e2 = issue_group_chunk(r0, ng, q)) != cudaSuccess) return e2;
        }
        return cudaSuccess;
      }
      // fork the branch streams off q, deal the groups round robin, join
      const int nb = nbranch;
      if ((e2 = cudaEventRecord(c->ev_fork, q)) != cudaSuccess) return e2;
      for (int b = 0; b < nb - 1; ++b)
        if ((e2 = cudaStreamWaitEvent(c->branch_stream[b], c->ev_fork, 0)) != cudaSuccess) return e2;
      int g = 0;
      for (int r0 = 0; r0 < nrhs; r0 += gsz, ++g) {
        const int ng = nrhs - r0 < gsz ? nrhs - r0 : gsz;
        const int b = g % nb;
        if ((e2 = issue_group_chunk(r0, ng, b ? c->branch_stream[b - 1] : q)) != cudaSuccess) return e2;
      }
      for (int b = 0; b < nb - 1; ++b) {
        if ((e2 = cudaEventRecord(c->ev_join[b], c->branch_stream[b])) != cudaSuccess) return e2;
        if ((e2 = cudaStreamWaitEvent(q, c->ev_join[b], 0)) != cudaSuccess) return e2;
      }
      return cudaSuccess;
    }
#define WZ_Q(...)                          \
  do {                                     \
    e2 = (__VA_ARGS__);                    \
    if (e2 != cudaSuccess) return e2;      \
  } while (0)
    for (int k = 0; k < K; ++k) {
      for (int r0 = 0; r0 < nrhs; r0 += gsz) {
        const int ng = nrhs - r0 < gsz ? nrhs - r0 : gsz;
        CGArgs<RI, RI> a1 = ga;
        a1.rhs0 = r0;
        WZ_Q(launch_cg<RI, RI>(L, pc, CG_P1, a1, ng, q));
        ZTArgs<RI> zz1 = z1;
        zz1.rhs0 = r0;
        WZ_Q(launch_zt<RI>(c->Z, c->T, mul1, zz1, ng, q));
        CGArgs<RI, RI> a3 = ga;
        a3.rhs0 = r0;
        a3.part_out = part3;
        WZ_Q(launch_cg<RI, RI>(L, pc, CG_P3, a3, ng, q));
        ZTArgs<RI> zz2 = z2;
        zz2.rhs0 = r0;
        WZ_Q(launch_zt<RI>(c->Z, c->T, mul2, zz2, ng, q));
        CGArgs<RI, RI> a5 = ga;
        a5.rhs0 = r0;
        a5.part_in = part3;
        a5.part_out = part5;
        WZ_Q(launch_cg<RI, RI>(L, pc, CG_P5, a5, ng, q));
      }
      count_launch();
      WZ_Q(launch_k(pdl, cg_scalar_iter, dim3(nrhs), dim3(32), 0, q, st, part5, part3, nblk, delta2, maxiter, cnt));
    }
    WZ_Q(launch_cg<double, RI>(L, pc, RU_P1, ra, nrhs, q));
    WZ_Q(launch_zt<double>(c->Z, c->T, mul1, y1, nrhs, q));
    CGArgs<double, double> r3{};
    r3.A = A64;
    r3.Cb = C64;
    r3.p = xs;
    r3.phi = c->phi64;
    r3.kArr = c->k64;
    r3.rpm = ga.rpm;
    r3.Z = c->Z;
    r3.twc = c->t64.twc;
    r3.tws = c->t64.tws;
    r3.shifted = ga.shifted;
    r3.st = st;
    r3.nblk = nblk;
    r3.TZ = TZ;
    r3.gate_ru = 1;
    r3.pdl = ra.pdl;
    WZ_Q(launch_cg<double, double>(L, pc, CG_P3, r3, nrhs, q));
    WZ_Q(launch_zt<double>(c->Z, c->T, mul2, y2, nrhs, q));
    CGArgs<double, RI> r5 = ra;
    r5.part_out = partR;
    WZ_Q(launch_cg<double, RI>(L, pc, RU_P5, r5, nrhs, q));
    count_launch();
    WZ_Q(launch_k(pdl, cg_scalar_ru, dim3(nrhs), dim3(32), 0, q, st, partR, nblk, maxiter, cnt));
#undef WZ_Q
    return cudaSuccess;
  };

  // Autotune the RHS group size, the branch count, dependent launch and the zt
  // passes' tiles per block once per solve shape: for each candidate,
  // re-initialise and time three chunks (24 iterations) with CUDA events,
  // twice, keeping the better round.  The first three are searched jointly
  // (with the zt grid at the resident blocks), the tiles per block for the
  // winner.
  {
    struct Choice {
      int g, nb, pdl, tpb;
    };
    static std::mutex mu;
    static std::map<std::vector<long>, Choice> cache;
    const std::vector<long> tkey{(long)sizeof(RI), (long)pc, (long)c->T, (long)c->Z, (long)c->X, (long)nrhs,
                                 (long)c->nm};
    bool found = false;
    Choice fc{};
    {
      std::lock_guard<std::mutex> lk(mu);
      auto it = cache.find(tkey);
      if (it != cache.end()) {
        found = true;
        fc = it->second;
      }
    }
    const char* forced = getenv("WZ_RHS_GROUP");  // a fixed group size overrides the tuner
    const char* forced_b = getenv("WZ_RHS_BRANCHES");
    const char* forced_pdl = getenv("WZ_PDL");     // 0 or 1 overrides the tuner's dependent-launch choice
    const char* forced_tpb = getenv("WZ_ZT_TPB");  // zt tiles per block (0: resident blocks)
    const bool pdl_forced = forced_pdl && (forced_pdl[0] == '0' || forced_pdl[0] == '1');
    const bool tpb_forced = forced_tpb && forced_tpb[0] >= '0' && forced_tpb[0] <= '9';
    // dependent launch by default (a solve that cannot be timed), unless a
    // graph capture with it has failed on this context
    bool pdl_pick = pdl_forced ? forced_pdl[0] == '1' : !c->pdl_capture_failed;
    int tpb_pick = tpb_forced ? atoi(forced_tpb) : 0;
    if (forced && atoi(forced) > 0) {
      gsz = atoi(forced) < nrhs ? atoi(forced) : nrhs;
      nbranch = forced_b ? atoi(forced_b) : 1;
      nbranch = nbranch < 1 ? 1 : (nbranch > wz_ctx::kMaxBranches ? wz_ctx::kMaxBranches : nbranch);
    } else if (found) {
      gsz = fc.g;
      nbranch = fc.nb;
      if (!pdl_forced) pdl_pick = fc.pdl != 0 && !c->pdl_capture_failed;
      if (!tpb_forced) tpb_pick = fc.tpb;
    } else if (inline_capture && nrhs >= 8) {
      // no timing inside a capture: four groups on four branches (the choice the
      // tuner makes for 12 right-hand sides at 16^4)
      gsz = (nrhs + 3) / 4;
      nbranch = (nrhs + gsz - 1) / gsz;
    } else if (!inline_capture && !g_probe.active) {
      std::vector<Choice> cand;
      for (int d : {1, 2, 3, 4, 6, 8})
        if (nrhs / d >= 1) {
          const int g = (nrhs + d - 1) / d;
          const int ngroups = (nrhs + g - 1) / g;
          for (int nb = 1; nb <= (ngroups < wz_ctx::kMaxBranches ? ngroups : wz_ctx::kMaxBranches); ++nb)
            for (int pd = 0; pd < 2; ++pd) {
              if (pdl_forced && pd != (pdl_pick ? 1 : 0)) continue;
              bool dup = false;
              for (const Choice& k : cand) dup |= (k.g == g && k.nb == nb && k.pdl == pd);
              if (!dup) cand.push_back(Choice{g, nb, pd, tpb_pick});
            }
        }
      cudaEvent_t e0, e1;
      cnt = nullptr;
      WZ_RUN(cudaEventCreate(&e0));
      WZ_RUN(cudaEventCreate(&e1));
      auto time_choice = [&](const Choice& cb, float* out_ms) -> cudaError_t {
        cudaError_t e2;
        gsz = cb.g;
        nbranch = cb.nb;
        set_pdl(cb.pdl != 0);
        set_ztpb(cb.tpb);
        if ((e2 = issue_chunk(s)) != cudaSuccess) return e2;  // warm-up on whatever state the recursion is in
        // the better of two timed rounds of three chunks (candidates a few
        // percent apart are otherwise ordered by noise)
        float ms = 1e30f;
        for (int round = 0; round < 2; ++round) {
          if ((e2 = cudaEventRecord(e0, s)) != cudaSuccess) return e2;
          for (int rep = 0; rep < 3; ++rep)
            if ((e2 = issue_chunk(s)) != cudaSuccess) return e2;
          if ((e2 = cudaEventRecord(e1, s)) != cudaSuccess) return e2;
          if ((e2 = cudaEventSynchronize(e1)) != cudaSuccess) return e2;
          float t = 0.f;
          if ((e2 = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess) return e2;
          ms = t < ms ? t : ms;
        }
        *out_ms = ms;
        // back to the initial state of the solve
        if ((e2 = cudaMemsetAsync(xs, 0, W.field64, s)) != cudaSuccess) return e2;
        count_launch(2);
        cg_init<RI><<<dim3(64, nrhs), 256, 0, s>>>(bs, r, xlo, p, n_per_rhs, partR, 64);
        if ((e2 = cudaGetLastError()) != cudaSuccess) return e2;
        cg_scalar_init<<<nrhs, 32, 0, s>>>(st, partR, 64, tol * tol, sh);
        return cudaGetLastError();
      };
      float best = 1e30f;
      Choice bestc{nrhs, 1, 0, tpb_pick};
      for (const Choice& cb : cand) {
        float ms = 0.f;
        WZ_RUN(time_choice(cb, &ms));
        if (ms < best) {
          best = ms;
          bestc = cb;
        }
      }
      if (!tpb_forced && sizeof(RI) == 4)
        for (int k : {2, 4}) {
          Choice cb = bestc;
          cb.tpb = k;
          float ms = 0.f;
          WZ_RUN(time_choice(cb, &ms));
          if (ms < best) {
            best = ms;
            bestc = cb;
          }
        }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      cnt = c->counters;
      gsz = bestc.g;
      nbranch = bestc.nb;
      pdl_pick = bestc.pdl != 0;
      tpb_pick = bestc.tpb;
      std::lock_guard<std::mutex> lk(mu);
      cache[tkey] = bestc;
    }
    set_pdl(pdl_pick);
    set_ztpb(tpb_pick);
  }


  // Graph mode: the whole chunk loop is one CUDA graph whose body sits in a
  // WHILE conditional node; a one-thread kernel at the end of the body keeps
  // the loop going while some RHS is active, and stops it after max_chunks
  // trips in any case.  The graph only references workspace buffers, so it is
  // cached on the context and replayed by every solve of the same shape.
  // The kernel probe needs eager launches (it brackets each launch).
  const bool use_graph = c->use_graphs && !g_probe.active;
  SolverGraph& G = c->solver_graph[(sizeof(RI) == 4 ? 0 : 1) + (pc ? 2 : 0)];
  int* trips = (int*)(base + W.off_trips);

  // Inline capture: the caller is capturing stream s into a larger graph (a
  // whole HMC trajectory).  The chunk loop becomes a WHILE conditional node of
  // that graph; its body is captured on a second stream.  No host interaction.
  if (inline_capture) {
    WZ_RUN(cudaMemsetAsync(trips, 0, sizeof(int), s));
    cudaStreamCaptureStatus cs;
    cudaGraph_t capg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    WZ_RUN(cudaStreamGetCaptureInfo(s, &cs, nullptr, &capg, &deps, nullptr, &ndeps));
    if (cs != cudaStreamCaptureStatusActive) return set_error(c, WZ_EINVAL, "inline solve outside a capture");
    cudaGraphConditionalHandle h;
    WZ_RUN(cudaGraphConditionalHandleCreate(&h, capg, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    WZ_RUN(cudaGraphAddNode(&node, capg, deps, nullptr, ndeps, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    WZ_RUN(cudaStreamBeginCaptureToGraph(c->cap_stream2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    const unsigned long long l0 = tl_launches;
    cudaError_t ce = issue_chunk(c->cap_stream2);
    if (ce == cudaSuccess) {
      count_launch();
      cg_loop_cond<<<1, 32, 0, c->cap_stream2>>>(h, st, nrhs, trips, max_chunks, c->counters, c->trip_slot);
      ce = cudaGetLastError();
    }
    c->inline_body_launches = tl_launches - l0;
    g_launches -= c->inline_body_launches;
    tl_launches = l0;
    cudaGraph_t captured = nullptr;
    cudaError_t ee = cudaStreamEndCapture(c->cap_stream2, &captured);
    if (ce != cudaSuccess) return cuda_error(c, ce, "inline solver capture");
    if (ee != cudaSuccess) return cuda_error(c, ee, "cudaStreamEndCapture (body)");
    WZ_RUN(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    WZ_RUN(cudaMemcpyAsync(x, xs, W.field64, cudaMemcpyDeviceToDevice, s));
    if (out) *out = SolveOut{};
    return WZ_OK;
  }
  if (use_graph) {
    SolverGraphKey key{};
    key.nrhs = nrhs;
    key.pc = pc;
    key.maxiter = maxiter;
    key.delta2 = delta2;
    key.ws = c->ws_solver.ptr;
    key.ws_bytes = c->ws_solver.bytes;
    key.phi64 = c->phi64;
    key.phi32 = c->phi32;
    key.gsz = gsz;
    key.nbranch = nbranch;
    key.pdl = pdl ? 1 : 0;
    key.tpb = z1.tpb;
    // a capture or instantiation that fails with dependent launches is
    // repeated once with plain launches (and the context keeps to them)
    for (int attempt = 0; attempt < 2 && (!G.exec || memcmp(&key, &G.key, sizeof(key)) != 0); ++attempt) {
      G.release();
      WZ_CUDA_TRY(c, cudaGraphCreate(&G.graph, 0));
      cudaGraphConditionalHandle h;
      WZ_CUDA_TRY(c, cudaGraphConditionalHandleCreate(&h, G.graph, 1, cudaGraphCondAssignDefault));
      cudaGraphNodeParams np{};
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = h;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      cudaGraphNode_t node;
      WZ_CUDA_TRY(c, cudaGraphAddNode(&node, G.graph, nullptr, nullptr, 0, &np));
      cudaGraph_t body = np.conditional.phGraph_out[0];
      WZ_CUDA_TRY(c, cudaStreamBeginCaptureToGraph(c->cap_stream, body, nullptr, nullptr, 0,
                                                   cudaStreamCaptureModeRelaxed));
      const unsigned long long l0 = tl_launches;
      cudaError_t ce = issue_chunk(c->cap_stream);
      if (ce == cudaSuccess) {
        count_launch();
        cg_loop_cond<<<1, 32, 0, c->cap_stream>>>(h, st, nrhs, trips, max_chunks, c->counters, 2);
        ce = cudaGetLastError();
      }
      G.body_launches = tl_launches - l0;  // kernels per trip of the WHILE body
      g_launches -= G.body_launches;       // capturing launches nothing
      tl_launches = l0;
      cudaGraph_t captured = nullptr;
      cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &captured);
      cudaError_t ei = (ce == cudaSuccess && ee == cudaSuccess) ? cudaGraphInstantiate(&G.exec, G.graph, 0) : ce;
      if (ce == cudaSuccess && ee == cudaSuccess && ei == cudaSuccess) {
        G.key = key;
        break;
      }
      if (pdl && attempt == 0) {
        cudaGetLastError();
        G.release();
        c->pdl_capture_failed = true;
        set_pdl(false);
        key.pdl = 0;
        continue;
      }
      if (ce != cudaSuccess) return cuda_error(c, ce, "solver graph capture");
      if (ee != cudaSuccess) return cuda_error(c, ee, "cudaStreamEndCapture");
      return cuda_error(c, ei, "cudaGraphInstantiate (solver)");
    }
  }

  // The preconditioned recursion stops on the residual of M~^dag M~ x~ = b~;
  // the original residual b - M^dag M x = M0^dag (b~ - M~^dag M~ x~) is then
  // checked in FP64 and RHS that miss tol resume with a tighter tolerance.
  std::vector<double> rel(nrhs);
  for (int outer = 0; outer < 8; ++outer) {
  if (use_graph) {
    WZ_RUN(cudaMemsetAsync(trips, 0, sizeof(int), s));
    WZ_RUN(cudaGraphLaunch(G.exec, s));
    WZ_RUN(cudaMemcpyAsync(hst, st, sizeof(RhsState) * nrhs, cudaMemcpyDeviceToHost, s));
    int* htrips = (int*)((char*)c->host_pinned + WZ_PINNED_SCRATCH_OFFSET - 64);
    WZ_RUN(cudaMemcpyAsync(htrips, trips, sizeof(int), cudaMemcpyDeviceToHost, s));
    WZ_RUN(cudaStreamSynchronize(s));
    count_launch((unsigned long long)(*htrips) * G.body_launches);
  } else {
    for (int chunk = 0; chunk < max_chunks; ++chunk) {
      WZ_RUN(issue_chunk(s));
      WZ_RUN(cudaMemcpyAsync(hst, st, sizeof(RhsState) * nrhs, cudaMemcpyDeviceToHost, s));
      WZ_RUN(cudaStreamSynchronize(s));
      bool any = false;
      for (int j = 0; j < nrhs; ++j) any |= hst[j].active != 0;
      if (!any) break;
    }
  }
  if (!pc) {
    WZ_RUN(cudaMemcpyAsync(x, xs, W.field64, cudaMemcpyDeviceToDevice, s));
    break;
  }
  {
    int rc = apply_op<double>(c, WZ_OP_M0INV, xs, x, nrhs, 0.0, A64);
    if (rc) return rc;
    rc = true_residuals(c, b, x, nrhs, sh, rel.data());
    if (rc) return rc;
  }
  bool again = false;
  for (int j = 0; j < nrhs; ++j) {
    if (hst[j].status == WZ_OK && hst[j].bnorm2 > 0.0 && rel[j] > tol) {
      const double f = 0.5 * tol / rel[j];
      hst[j].tol2 *= f * f;
      hst[j].active = 1;
      hst[j].run = 1;
      hst[j].ru = 0;
      again = true;
    }
  }
  if (!again) break;
  WZ_RUN(cudaMemcpyAsync(st, hst, sizeof(RhsState) * nrhs, cudaMemcpyHostToDevice, s));
  }
#undef WZ_RUN

  for (int j = 0; j < nrhs; ++j) {
    if (hst[j].status == WZ_ETIMEOUT || hst[j].status == WZ_ECUDA)
      return set_error(c, hst[j].status, hst[j].status == WZ_ETIMEOUT ? "solver: a staged copy wait ran out"
                                                                       : "solver: a staged copy was misaligned");
    if (hst[j].status == WZ_ENONFINITE)
      return set_error(c, WZ_ENONFINITE, "solver: a residual norm became NaN or Inf (non-finite input)");
  }
  SolveOut o;
  for (int j = 0; j < nrhs; ++j) {
    o.iterations = hst[j].iters > o.iterations ? hst[j].iters : o.iterations;
    o.total_iterations += hst[j].iters;
    o.reliable_updates += hst[j].ru_count;
    const bool ok = hst[j].active == 0 && hst[j].status == WZ_OK;
    o.converged += ok ? 1 : 0;
    const double rj = pc ? rel[j] : (hst[j].bnorm2 > 0 ? sqrt(hst[j].rtrue2 / hst[j].bnorm2) : 0.0);
    o.max_true_residual = rj > o.max_true_residual ? rj : o.max_true_residual;
  }
  *out = o;
  return o.converged == nrhs ? WZ_OK : WZ_NOT_CONVERGED;
}

}  // namespace wz
