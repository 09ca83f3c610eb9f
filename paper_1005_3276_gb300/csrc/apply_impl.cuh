// Pass sequencing of the operators of wz_op, templated on precision.
//
//   M        : xy_fwd(psi) -> zt(+Dslash) -> xy_inv(+ Y psi)
//   M^dag    : xy_fwd(psi) -> zt(-Dslash) -> xy_inv(+ Y^dag psi)
//   M^dag M  : xy_fwd(psi) -> zt(+Dslash) -> xy_inv_fwd(C = M psi) -> zt(-Dslash)
//              -> xy_inv(+ Y^dag C + shift psi)
//   M~ = 1 + Y_int M0^-1,  M~^dag = 1 + (M0^-1)^dag Y_int^dag   (Sec. 7.3, M0 M0^-1 = 1)
#pragma once
#include "wz_ctx.h"
#include "launch.h"

namespace wz {


template <typename R> static SiteCoef<R> site_coef_of(const wz_params& p) {
  SiteCoef<R> k;
  k.m_re = (R)p.m_re;
  k.m_im = (R)p.m_im;
  k.cg_re = (R)(p.yukawa * p.g_re);
  k.cg_im = (R)(p.yukawa * p.g_im);
  k.g_re = (R)p.g_re;
  k.g_im = (R)p.g_im;
  return k;
}

// right-hand sides per member for a launch over nrhs right-hand sides in total
static inline int rhs_per_member(const wz_ctx* c, int nrhs) { return c->nm > 1 ? nrhs / c->nm : (nrhs > 0 ? nrhs : 1); }

template <typename R> static XYArgs<R> xy_args(const wz_ctx* c, int nrhs) {
  XYArgs<R> a{};
  a.phi = phi_of<R>(c);
  a.kArr = karr_of<R>(c);
  a.rpm = rhs_per_member(c, nrhs);
  a.nplanes = nrhs * c->T * c->Z;
  a.TZ = c->T * c->Z;
  a.Z = c->Z;
  a.twc = tables<R>(c).twc;
  a.tws = tables<R>(c).tws;
  a.fail = (int*)(c->counters + WZ_COUNTER_DEVICE_ERROR);  // sticky device error word of the context
  return a;
}

// the column tile of zt_pass<R, nz, nt> (ZTShape::C), from the runtime extents
template <typename R> static int zt_cols(int nz, int nt) { return zt_cols_of<R>(nz, nt); }

template <typename R> static ZTArgs<R> zt_args(const wz_ctx* c, R sign) {
  const Tables<R>& t = tables<R>(c);
  ZTArgs<R> a{};
  a.hV = t.hV;
  a.hdV = t.hdV;
  a.dV = t.dV;
  a.d2sV = t.d2sV;
  a.ksV = t.ksV;
  a.sinT = t.sinT;
  a.sinZ = t.sinZ;
  a.sinY = t.sinY;
  a.sinX = t.sinX;
  a.twc = t.twc;
  a.tws = t.tws;
  a.sign = sign;
  a.m_re = (R)c->p.m_re;
  a.m_im = (R)c->p.m_im;
  a.X = c->X;
  a.XY = c->X * c->Y;
  const int C = zt_cols<R>(c->Z, c->T);
  a.ntiles = (a.XY + C - 1) / C;
  a.fail = (int*)(c->counters + WZ_COUNTER_DEVICE_ERROR);  // sticky device error word of the context
  a.fail_stride = 0;
  return a;
}

template <typename R> size_t apply_ws_bytes(const wz_ctx* c, int op, int nrhs) {
  const size_t field = sizeof(cplx<R>) * 4 * (size_t)c->V * nrhs;
  const bool two = (op == WZ_OP_MDAGM || op == WZ_OP_MTILDE_DAGM);
  return two ? 2 * field : field;
}

// ws must hold apply_ws_bytes(c, op, nrhs) bytes.
template <typename R>
int apply_op(wz_ctx* c, int op, const cplx<R>* in, cplx<R>* out, int nrhs, R shift, cplx<R>* ws) {
  const int L = c->X;
  const long field = 4L * c->V * nrhs;
  cplx<R>* A = ws;
  cplx<R>* Cb = ws + field;
  cudaStream_t st = c->stream;
  XYArgs<R> xa = xy_args<R>(c, nrhs);
  cudaError_t e = cudaSuccess;
#define WZ_RUN(expr)                                    \
  do {                                                  \
    e = (expr);                                         \
    if (e != cudaSuccess) return cuda_error(c, e, #expr); \
  } while (0)

  auto fwd = [&](int mode, const cplx<R>* src) {
    XYArgs<R> a = xa;
    a.psi = src;
    a.A_out = A;
    return launch_xy<R>(L, mode, a, st);
  };
  auto zt = [&](int mul, R sign) {
    ZTArgs<R> a = zt_args<R>(c, sign);
    a.A = A;
    return launch_zt<R>(c->Z, c->T, mul, a, nrhs, st);
  };
  auto inv = [&](int mode, const cplx<R>* psi, const cplx<R>* psi2, cplx<R>* vout, cplx<R>* aout) {
    XYArgs<R> a = xa;
    a.A_in = A;
    a.A_out = aout;
    a.psi = psi;
    a.psi2 = psi2;
    a.shift = shift;
    a.v_out = vout;
    return launch_xy<R>(L, mode, a, st);
  };

  switch (op) {
    case WZ_OP_M:
      WZ_RUN(fwd(XY_FWD, in));
      WZ_RUN(zt(ZT_DSLASH, R(1)));
      WZ_RUN(inv(XY_INV_Y, in, nullptr, out, nullptr));
      break;
    case WZ_OP_MDAG:
      WZ_RUN(fwd(XY_FWD, in));
      WZ_RUN(zt(ZT_DSLASH, R(-1)));
      WZ_RUN(inv(XY_INV_YDAG, in, nullptr, out, nullptr));
      break;
    case WZ_OP_MDAGM:
      WZ_RUN(fwd(XY_FWD, in));
      WZ_RUN(zt(ZT_DSLASH, R(1)));
      WZ_RUN(inv(XY_INV_Y_FWD, in, nullptr, Cb, A));
      WZ_RUN(zt(ZT_DSLASH, R(-1)));
      WZ_RUN(inv(XY_INV_YDAG, Cb, shift != R(0) ? in : nullptr, out, nullptr));
      break;
    case WZ_OP_DSLASH:
      WZ_RUN(fwd(XY_FWD, in));
      WZ_RUN(zt(ZT_DSLASH, R(1)));
      WZ_RUN(inv(XY_INV, nullptr, nullptr, out, nullptr));
      break;
    case WZ_OP_D1: {
      // the Dslash multiply with 1/omega in place of h: D1(p) = i gamma.sin p / omega
      WZ_RUN(fwd(XY_FWD, in));
      ZTArgs<R> za = zt_args<R>(c, R(1));
      za.A = A;
      za.hV = tables<R>(c).w1V;
      WZ_RUN(launch_zt<R>(c->Z, c->T, ZT_DSLASH, za, nrhs, st));
      WZ_RUN(inv(XY_INV, nullptr, nullptr, out, nullptr));
      break;
    }
    case WZ_OP_D: {
      // the overlap operator D = D1 + D2 = 1 - V (Sec. 2.2): i gamma.sin p / omega + (1 - b/omega)
      WZ_RUN(fwd(XY_FWD, in));
      ZTArgs<R> za = zt_args<R>(c, R(1));
      za.A = A;
      za.hV = tables<R>(c).w1V;
      za.dV = tables<R>(c).d2fV;
      WZ_RUN(launch_zt<R>(c->Z, c->T, ZT_OVERLAP, za, nrhs, st));
      WZ_RUN(inv(XY_INV, nullptr, nullptr, out, nullptr));
      break;
    }
    case WZ_OP_M0INV:
    case WZ_OP_M0INV_DAG:
      WZ_RUN(fwd(XY_FWD, in));
      WZ_RUN(zt(op == WZ_OP_M0INV ? ZT_M0INV : ZT_M0INV_DAG, R(1)));
      WZ_RUN(inv(XY_INV, nullptr, nullptr, out, nullptr));
      break;
    case WZ_OP_MTILDE:
      WZ_RUN(fwd(XY_FWD, in));
      WZ_RUN(zt(ZT_M0INV, R(1)));
      WZ_RUN(inv(XY_INV_PC, in, nullptr, out, nullptr));
      break;
    case WZ_OP_MTILDE_DAG:
      WZ_RUN(fwd(XY_FWD_YINTDAG, in));
      WZ_RUN(zt(ZT_M0INV_DAG, R(1)));
      WZ_RUN(inv(XY_INV_ADD, in, nullptr, out, nullptr));
      break;
    case WZ_OP_MTILDE_DAGM:
      WZ_RUN(fwd(XY_FWD, in));
      WZ_RUN(zt(ZT_M0INV, R(1)));
      WZ_RUN(inv(XY_INV_PC_FWD, in, nullptr, Cb, A));
      WZ_RUN(zt(ZT_M0INV_DAG, R(1)));
      WZ_RUN(inv(XY_INV_ADD, Cb, shift != R(0) ? in : nullptr, out, nullptr));
      break;
    default:
      return set_error(c, WZ_EINVAL, "unknown operator");
  }
#undef WZ_RUN
  return WZ_OK;
}

}  // namespace wz
