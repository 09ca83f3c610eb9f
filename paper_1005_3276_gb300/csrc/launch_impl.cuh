// Launch wrappers of every kernel template: grid sizes, dynamic shared memory,
// algorithmic bytes for the probe.  Included only by the kern_L*.cu and
// zt_*.cu translation units, which instantiate them once per extent.
#pragma once
#include <cudaTypedefs.h>  // PFN_cuTensorMapEncodeTiled

#include "launch.h"

namespace wz {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool looked = false;
  if (!looked) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    looked = true;
  }
  return fn;
}

// Tensor map of a zt-pass field A [rhs][t][z][XY][4] for nrhs right-hand sides:
// 3D in 8-byte elements, (XY * 4 * U, Z, T * nrhs), box (C * 4 * U, Z, T) = one tile.
template <typename R, int NZ, int NT>
static cudaError_t zt_tensor_map(const ZTArgs<R>& a, int nrhs, CUtensorMap* m) {
  constexpr int U = sizeof(cplx<R>) / 8;
  constexpr int C = ZTShape<R, NZ, NT>::C;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t row = (cuuint64_t)a.XY * 4 * U;  // elements of one (t, z) row
  cuuint64_t dims[3] = {row, (cuuint64_t)NZ, (cuuint64_t)NT * nrhs};
  cuuint64_t strides[2] = {row * 8, row * 8 * NZ};  // bytes, dimensions 1 and 2
  cuuint32_t box[3] = {(cuuint32_t)(C * 4 * U), (cuuint32_t)NZ, (cuuint32_t)NT};
  cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, (void*)a.A, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Tensor map of a momentum table [p_t][p_z][column] (R), box (CB, Z, T): the
// slice of one tile (CB >= C columns, see ZTSmem).
template <typename R, int NZ, int NT, int MUL>
static cudaError_t zt_table_map(const R* tab, int XY, CUtensorMap* m) {
  constexpr int C = ZTSmem<R, NZ, NT, MUL>::CB;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  cuuint64_t dims[3] = {(cuuint64_t)XY, (cuuint64_t)NZ, (cuuint64_t)NT};
  cuuint64_t strides[2] = {(cuuint64_t)XY * sizeof(R), (cuuint64_t)XY * NZ * sizeof(R)};
  cuuint32_t box[3] = {(cuuint32_t)C, (cuuint32_t)NZ, (cuuint32_t)NT};
  cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(m, sizeof(R) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                         (void*)tab, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}


template <typename R, int L, int MODE, bool STAGE>
static cudaError_t launch_xy_s(const XYArgs<R>& a, int grid, double blk_bytes, cudaStream_t st) {
  using S = XYShape<L>;
  const size_t smem = XYSmem<R, L, MODE, STAGE>::total;
  static SmemAttrDone attr;  // one attribute call per instantiation and device
  {
    cudaError_t e = set_smem_once(xy_pass<R, L, MODE, STAGE>, smem, attr);
    if (e != cudaSuccess) return e;
  }
  return probed(PK_XY, (int)sizeof(R), blk_bytes, st, [&](unsigned long long* cnt) {
    XYArgs<R> b = a;
    b.blk_count = cnt;
    b.probe_inc = (unsigned long long)blk_bytes;
    xy_pass<R, L, MODE, STAGE><<<grid, S::THREADS, smem, st>>>(b);
    return cudaGetLastError();
  });
}

template <typename R, int L, int MODE>
static cudaError_t launch_xy_t(const XYArgs<R>& a, cudaStream_t st) {
  using S = XYShape<L>;
  using XS = XYSmem<R, L, MODE, true>;
  const int grid = (a.nplanes + S::PPC - 1) / S::PPC;
  if (grid == 0) return cudaSuccess;
  // algorithmic bytes of one block: the spinor fields it reads and writes,
  // plus phi where the site term needs it
  using I = XYModeInfo<MODE>;
  int fields = (I::inv ? 1 : 0) + (I::fwd ? 1 : 0) + (a.psi ? 1 : 0) + (a.psi2 ? 1 : 0) + (a.v_out ? 1 : 0);
  const bool uses_phi = !(MODE == XY_FWD || MODE == XY_INV || MODE == XY_INV_ADD);
  const double site = 4.0 * sizeof(cplx<R>) * fields + (uses_phi ? sizeof(cplx<R>) : 0);
  const double blk_bytes = site * L * L * S::PPC;
  // staged form: FP32, extents up to 32, 16-byte aligned operands (the user's
  // fields may be views at any offset) and blocks of planes within one RHS
  auto al = [](const void* p) { return ((unsigned long long)p & 15ull) == 0; };
  const bool stage = sizeof(R) == 4 && L <= 32 && a.TZ % S::PPC == 0 && (!I::inv || al(a.A_in)) &&
                     (!XS::USES_PSI || al(a.psi)) && (!XS::USES_PHI || al(a.phi));
  if constexpr (sizeof(R) == 4 && L <= 32) {
    if (stage) return launch_xy_s<R, L, MODE, true>(a, grid, blk_bytes, st);
  }
  return launch_xy_s<R, L, MODE, false>(a, grid, blk_bytes, st);
}

template <typename R, int L>
cudaError_t launch_xy_L(int mode, const XYArgs<R>& a, cudaStream_t st) {
  switch (mode) {
    case XY_FWD: return launch_xy_t<R, L, XY_FWD>(a, st);
    case XY_FWD_YINTDAG: return launch_xy_t<R, L, XY_FWD_YINTDAG>(a, st);
    case XY_INV: return launch_xy_t<R, L, XY_INV>(a, st);
    case XY_INV_Y: return launch_xy_t<R, L, XY_INV_Y>(a, st);
    case XY_INV_YDAG: return launch_xy_t<R, L, XY_INV_YDAG>(a, st);
    case XY_INV_Y_FWD: return launch_xy_t<R, L, XY_INV_Y_FWD>(a, st);
    case XY_INV_PC: return launch_xy_t<R, L, XY_INV_PC>(a, st);
    case XY_INV_PC_FWD: return launch_xy_t<R, L, XY_INV_PC_FWD>(a, st);
    case XY_INV_ADD: return launch_xy_t<R, L, XY_INV_ADD>(a, st);
  }
  return cudaErrorInvalidValue;
}

template <typename R, int NZ, int NT, int MUL>
static cudaError_t launch_zt_t(const ZTArgs<R>& a, int nrhs, cudaStream_t st) {
  using S = ZTShape<R, NZ, NT>;
  constexpr int C = S::C;
  using ZS = ZTSmem<R, NZ, NT, MUL>;
  const size_t smem = ZS::total;
  static SmemAttrDone attr;
  {
    cudaError_t e = set_smem_once(zt_pass<R, NZ, NT, MUL>, smem, attr);
    if (e != cudaSuccess) return e;
  }
  const long ntot = (long)nrhs * a.ntiles;
  if (ntot == 0) return cudaSuccess;
  // persistent grid: at most the blocks resident on the device (fewer when the
  // caller asks for at least a.tpb tiles a block), balanced so that every
  // block takes the same number of tiles (ceil(ntot / grid))
  static ResidentBlocks resident;
  int gmax = 0;
  {
    cudaError_t e = resident.get(zt_pass<R, NZ, NT, MUL>, S::THREADS, smem, &gmax);
    if (e != cudaSuccess) return e;
  }
  long per = (ntot + gmax - 1) / gmax;
  if (a.tpb > per) per = a.tpb;
  const long grid = (ntot + per - 1) / per;
  // the map covers right-hand sides 0 .. rhs0 + nrhs - 1 of A; the last one is reused
  const R* t0 = (MUL == ZT_DSLASH || MUL == ZT_GRAD || MUL == ZT_OVERLAP) ? a.hV : (MUL == ZT_SCALAR ? a.d2sV : a.hdV);
  const R* t1 = (MUL == ZT_DSLASH || MUL == ZT_GRAD) ? nullptr : (MUL == ZT_SCALAR ? a.ksV : a.dV);
  struct MapCache {
    const void* A = nullptr;
    const void* t0 = nullptr;
    const void* t1 = nullptr;
    int XY = 0, n = 0;
    CUtensorMap m, m0, m1;
  };
  static thread_local MapCache mc;
  if (mc.A != (const void*)a.A || mc.XY != a.XY || mc.n != a.rhs0 + nrhs || mc.t0 != t0 || mc.t1 != t1) {
    cudaError_t e = zt_tensor_map<R, NZ, NT>(a, a.rhs0 + nrhs, &mc.m);
    if (e == cudaSuccess && ZS::NTAB >= 1) e = zt_table_map<R, NZ, NT, MUL>(t0, a.XY, &mc.m0);
    if (e == cudaSuccess && ZS::NTAB >= 2) e = zt_table_map<R, NZ, NT, MUL>(t1, a.XY, &mc.m1);
    if (e != cudaSuccess) {
      mc.A = nullptr;
      return e;
    }
    if (ZS::NTAB < 1) mc.m0 = mc.m;  // unused parameters
    if (ZS::NTAB < 2) mc.m1 = mc.m;
    mc.A = a.A;
    mc.t0 = t0;
    mc.t1 = t1;
    mc.XY = a.XY;
    mc.n = a.rhs0 + nrhs;
  }
  const CUtensorMap tm = mc.m, tm0 = mc.m0, tm1 = mc.m1;
  // one tile reads and writes C columns x NZ x NT sites of 4 spins and reads
  // the momentum tables it needs (1 for Dslash and D1 on scalars, 2 for
  // M0^-1 and the scalar pair)
  const int ntab = (MUL == ZT_DSLASH || MUL == ZT_GRAD) ? 1 : 2;
  const double bytes = (double)C * NZ * NT * (2.0 * 4 * sizeof(cplx<R>) + ntab * sizeof(R));
  return probed(PK_ZT, (int)sizeof(R), bytes, st, [&](unsigned long long* cnt) {
    ZTArgs<R> b = a;
    b.ntot = (int)ntot;
    b.blk_count = cnt;
    b.probe_inc = (unsigned long long)bytes;
    return launch_k(b.pdl != 0, zt_pass<R, NZ, NT, MUL>, dim3((unsigned)grid), dim3(S::THREADS), smem, st, b, tm,
                    tm0, tm1);
  });
}

template <typename R, int NZ, int NT>
cudaError_t launch_zt_p(int mul, const ZTArgs<R>& a, int nrhs, cudaStream_t st) {
  switch (mul) {
    case ZT_DSLASH: return launch_zt_t<R, NZ, NT, ZT_DSLASH>(a, nrhs, st);
    case ZT_M0INV: return launch_zt_t<R, NZ, NT, ZT_M0INV>(a, nrhs, st);
    case ZT_M0INV_DAG: return launch_zt_t<R, NZ, NT, ZT_M0INV_DAG>(a, nrhs, st);
    case ZT_OVERLAP: return launch_zt_t<R, NZ, NT, ZT_OVERLAP>(a, nrhs, st);
    case ZT_SCALAR:
      if constexpr (sizeof(R) == 8) return launch_zt_t<R, NZ, NT, ZT_SCALAR>(a, nrhs, st);
      break;
    case ZT_GRAD:
      if constexpr (sizeof(R) == 8) return launch_zt_t<R, NZ, NT, ZT_GRAD>(a, nrhs, st);
      break;
  }
  return cudaErrorInvalidValue;
}

template <typename R, typename LO, int L, int MODE, bool PC>
static cudaError_t launch_cg_t(const CGArgs<R, LO>& a, int nrhs, cudaStream_t st) {
  using S = XYShape<L>;
  const size_t smem = CGSmem<R, L, MODE, PC>::total;
  static SmemAttrDone attr;
  {
    cudaError_t e = set_smem_once(xy_cg<R, LO, L, MODE, PC>, smem, attr);
    if (e != cudaSuccess) return e;
  }
  dim3 grid(a.nblk, nrhs);
  // algorithmic bytes of one block (PPC planes of L x L sites, 4 spins)
  const double f = 4.0 * sizeof(cplx<R>), lo = 4.0 * sizeof(cplx<LO>), ph = sizeof(cplx<R>);
  double site = 0.0;
  int kind = PK_CG_P1;
  switch (MODE) {
    case CG_P1: site = 6 * f; kind = PK_CG_P1; break;                 // r, p, x in; p, A, x out
    case CG_P3: site = 4 * f + ph; kind = PK_CG_P3; break;            // A, p in; C, A out; phi
    case CG_P5: site = (a.shifted && !PC ? 5 : 4) * f + (PC ? 0 : ph); kind = PK_CG_P5; break;  // A, C, r (p) in; r out
    case RU_P1: site = 3 * f + 3 * lo; kind = PK_RU_P1; break;        // x_hi, x_lo, p in; x_hi, x_lo, A out
    case RU_P5: site = 4 * f + lo + (PC ? 0 : ph); kind = PK_RU_P5; break;  // A, x_hi, C, b in; r out
  }
  const double blk_bytes = site * L * L * S::PPC;
  return probed(kind, (int)sizeof(R), blk_bytes, st, [&](unsigned long long* cnt) {
    CGArgs<R, LO> b = a;
    b.blk_count = cnt;
    b.probe_inc = (unsigned long long)blk_bytes;
    return launch_k(b.pdl != 0, xy_cg<R, LO, L, MODE, PC>, grid, dim3(S::THREADS), smem, st, b);
  });
}

template <typename R, typename LO, int L, bool PC>
static cudaError_t launch_cg_m(int mode, const CGArgs<R, LO>& a, int nrhs, cudaStream_t st) {
  switch (mode) {
    case CG_P1: return launch_cg_t<R, LO, L, CG_P1, PC>(a, nrhs, st);
    case CG_P3: return launch_cg_t<R, LO, L, CG_P3, PC>(a, nrhs, st);
    case CG_P5: return launch_cg_t<R, LO, L, CG_P5, PC>(a, nrhs, st);
    case RU_P1: return launch_cg_t<R, LO, L, RU_P1, PC>(a, nrhs, st);
    case RU_P5: return launch_cg_t<R, LO, L, RU_P5, PC>(a, nrhs, st);
  }
  return cudaErrorInvalidValue;
}

template <typename R, typename LO, int L>
cudaError_t launch_cg_L(bool pc, int mode, const CGArgs<R, LO>& a, int nrhs, cudaStream_t st) {
  return pc ? launch_cg_m<R, LO, L, true>(mode, a, nrhs, st) : launch_cg_m<R, LO, L, false>(mode, a, nrhs, st);
}

template <int L>
cudaError_t launch_fk_L(int which, const ForceArgs<double>& a, dim3 grid, cudaStream_t st) {
  using S = XYShape<L>;
  const size_t smem = sizeof(cplx<double>) * S::PLANE * S::PPC + 33 * sizeof(double);
  static SmemAttrDone done[3];
  cudaError_t e = cudaSuccess;
  if (which == FK_FORCE) e = set_smem_once(xy_force<L>, smem, done[0]);
  if (which == FK_BOSON_FWD) e = set_smem_once(xy_boson_fwd<L>, smem, done[1]);
  if (which == FK_BOSON_INV) e = set_smem_once(xy_boson_inv<L>, smem, done[2]);
  if (e != cudaSuccess) return e;
  count_launch();
  if (which == FK_FORCE) xy_force<L><<<grid, S::THREADS, smem, st>>>(a);
  if (which == FK_BOSON_FWD) xy_boson_fwd<L><<<grid, S::THREADS, smem, st>>>(a);
  if (which == FK_BOSON_INV) xy_boson_inv<L><<<grid, S::THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace wz
