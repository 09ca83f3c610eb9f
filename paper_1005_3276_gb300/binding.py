"""ctypes binding of the C ABI declared in include/wz.h (argument marshalling only).

Every function here forwards to the entry point of the same name in libwz.so;
all arithmetic runs in the library's CUDA kernels.  Fields may be torch
tensors (device or host) or numpy arrays (host); both must be C-contiguous
with dtype complex64 (WZ_C64) or complex128 (WZ_C128).  There is no fallback:
if libwz.so is missing or fails to load, importing this module raises.
"""

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libwz.so")

WZ_OK, WZ_EINVAL, WZ_ENOMEM, WZ_ECUDA, WZ_NOT_CONVERGED, WZ_EUNSUPPORTED, WZ_ETIMEOUT, WZ_ENONFINITE = range(8)
WZ_C64, WZ_C128 = 0, 1
(WZ_OP_M, WZ_OP_MDAG, WZ_OP_MDAGM, WZ_OP_DSLASH, WZ_OP_M0INV, WZ_OP_M0INV_DAG,
 WZ_OP_MTILDE, WZ_OP_MTILDE_DAG, WZ_OP_MTILDE_DAGM, WZ_OP_D1, WZ_OP_D) = range(11)
OPS = {"M": WZ_OP_M, "Mdag": WZ_OP_MDAG, "MdagM": WZ_OP_MDAGM, "Dslash": WZ_OP_DSLASH,
       "M0inv": WZ_OP_M0INV, "M0inv_dag": WZ_OP_M0INV_DAG, "Mtilde": WZ_OP_MTILDE,
       "Mtilde_dag": WZ_OP_MTILDE_DAG, "Mtilde_dagM": WZ_OP_MTILDE_DAGM, "D1": WZ_OP_D1, "D": WZ_OP_D}


class WzParams(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("m_re", ctypes.c_double), ("m_im", ctypes.c_double),
                ("g_re", ctypes.c_double), ("g_im", ctypes.c_double), ("r", ctypes.c_double),
                ("M0", ctypes.c_double), ("yukawa", ctypes.c_double)]


class WzSolveStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("total_iterations", ctypes.c_int),
                ("reliable_updates", ctypes.c_int), ("converged", ctypes.c_int),
                ("max_true_residual", ctypes.c_double), ("seconds", ctypes.c_double),
                ("site_applies", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


WZ_SOLVE_MIXED, WZ_SOLVE_PC = 1, 2


class WzProbeResult(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_long), ("timed_launches", ctypes.c_long),
                ("total_ms", ctypes.c_double), ("bytes", ctypes.c_double)]


class WzHmcParams(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("nsteps", ctypes.c_int), ("integrator", ctypes.c_int),
                ("npf", ctypes.c_int), ("tol", ctypes.c_double), ("maxiter", ctypes.c_int),
                ("flags", ctypes.c_uint), ("seed", ctypes.c_ulonglong), ("traj_index", ctypes.c_uint)]


class WzTrajStats(ctypes.Structure):
    _fields_ = [("H0", ctypes.c_double), ("H1", ctypes.c_double), ("dH", ctypes.c_double),
                ("u", ctypes.c_double), ("accept", ctypes.c_int), ("force_evals", ctypes.c_int),
                ("cg_iterations", ctypes.c_longlong), ("reliable_updates", ctypes.c_int),
                ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


WZ_RATIONAL_MAX = 64


class WzRational(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("a0", ctypes.c_double), ("alpha", ctypes.c_double * WZ_RATIONAL_MAX),
                ("beta", ctypes.c_double * WZ_RATIONAL_MAX), ("power", ctypes.c_double), ("lo", ctypes.c_double),
                ("hi", ctypes.c_double), ("build_lo", ctypes.c_double), ("build_hi", ctypes.c_double),
                ("err", ctypes.c_double)]

    def as_dict(self):
        d = int(self.d)
        return {"d": d, "a0": self.a0, "alpha": np.array(self.alpha[:d]), "beta": np.array(self.beta[:d]),
                "gamma": self.power, "lo": self.lo, "hi": self.hi, "build_lo": self.build_lo,
                "build_hi": self.build_hi, "err": self.err}


def rational_struct(coef):
    """WzRational from a mapping with a0, alpha, beta (and optional gamma, lo, hi, err)."""
    r = WzRational()
    alpha, beta = list(coef["alpha"]), list(coef["beta"])
    if len(alpha) != len(beta) or len(alpha) > WZ_RATIONAL_MAX:
        raise ValueError("alpha and beta need the same length <= 64")
    r.d = len(alpha)
    r.a0 = float(coef["a0"])
    for i, (a, b) in enumerate(zip(alpha, beta)):
        r.alpha[i], r.beta[i] = float(a), float(b)
    r.power = float(coef.get("gamma", 0.0))
    r.lo, r.hi = float(coef.get("lo", 0.0)), float(coef.get("hi", 0.0))
    r.err = float(coef.get("err", 0.0))
    return r


WZ_FORCE_FERMION, WZ_FORCE_BOSON = 1, 2
WZ_HMC_FP64_SOLVES, WZ_HMC_NO_METROPOLIS = 1, 2
INTEGRATORS = {"leapfrog": 0, "omelyan": 1}

PROBE_KINDS = {"zt": 0, "xy": 1, "cg_p1": 2, "cg_p3": 3, "cg_p5": 4, "ru_p1": 5, "ru_p5": 6}


class WzError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"wz status {code}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIBPATH):
        raise ImportError(f"{LIBPATH} is missing: run __graft_entry__.build() (nvcc, sm_103a) first")
    lib = ctypes.CDLL(LIBPATH)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "wz_create": ([ctypes.POINTER(WzParams), P, ctypes.POINTER(P)], I),
        "wz_destroy": ([P], I),
        "wz_last_error": ([P], ctypes.c_char_p),
        "wz_supported_extent": ([I], I),
        "wz_set_phi": ([P, P], I),
        "wz_apply": ([P, I, I, P, P, I, D], I),
        "wz_solve": ([P, P, P, I, D, D, I, ctypes.c_uint, ctypes.POINTER(WzSolveStats),
                      ctypes.POINTER(ctypes.c_double)], I),
        "wz_apply_mdagm_noalloc": ([P, I, P, P, I, D], I),
        "wz_get_phi": ([P, P], I),
        "wz_force": ([P, P, I, D, ctypes.c_uint, P, ctypes.POINTER(D), ctypes.POINTER(D),
                      ctypes.POINTER(WzSolveStats)], I),
        "wz_action": ([P, P, I, D, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(WzSolveStats)], I),
        "wz_md_integrate": ([P, P, P, I, ctypes.POINTER(WzHmcParams), ctypes.POINTER(WzTrajStats)], I),
        "wz_trajectory": ([P, ctypes.POINTER(WzHmcParams), ctypes.POINTER(WzTrajStats)], I),
        "wz_batch_create": ([ctypes.POINTER(WzParams), I, P, ctypes.POINTER(P)], I),
        "wz_batch_destroy": ([P], I),
        "wz_batch_last_error": ([P], ctypes.c_char_p),
        "wz_batch_size": ([P], I),
        "wz_batch_groups": ([P], I),
        "wz_batch_set_phi": ([P, I, P], I),
        "wz_batch_get_phi": ([P, I, P], I),
        "wz_batch_solve": ([P, ctypes.POINTER(P), ctypes.POINTER(P), I, D, I, ctypes.c_uint,
                            ctypes.POINTER(WzSolveStats)], I),
        "wz_batch_trajectory": ([P, ctypes.POINTER(WzHmcParams), ctypes.POINTER(WzTrajStats)], I),
        "wz_solve_multishift": ([P, P, P, I, I, ctypes.POINTER(D), D, I, ctypes.c_uint,
                                 ctypes.POINTER(WzSolveStats), ctypes.POINTER(D)], I),
        "wz_rational_minimax": ([D, D, D, I, ctypes.POINTER(WzRational)], I),
        "wz_spectral_bounds": ([P, ctypes.POINTER(D), ctypes.POINTER(D)], I),
        "wz_rational_apply": ([P, ctypes.POINTER(WzRational), P, P, I, D, I, ctypes.c_uint, D,
                               ctypes.POINTER(WzSolveStats)], I),
        "wz_rhmc_force": ([P, P, I, ctypes.POINTER(WzRational), D, ctypes.c_uint, P, ctypes.POINTER(D),
                           ctypes.POINTER(D), ctypes.POINTER(WzSolveStats)], I),
        "wz_rhmc_trajectory": ([P, ctypes.POINTER(WzHmcParams), ctypes.POINTER(WzRational),
                                ctypes.POINTER(WzRational), ctypes.POINTER(WzTrajStats)], I),
        "wz_ward_identity": ([P, D, I, ctypes.c_uint, ctypes.POINTER(D), ctypes.POINTER(D),
                              ctypes.POINTER(WzSolveStats)], I),
        "wz_supercurrent": ([P, P, D, I, ctypes.c_uint, ctypes.POINTER(D), ctypes.POINTER(WzSolveStats)], I),
        "wz_one_loop": ([I, D, ctypes.POINTER(D)], I),
        "wz_aux_vev": ([P, ctypes.POINTER(D)], I),
        "wz_locality": ([P, ctypes.POINTER(D), I], I),
        "wz_locality_op": ([P, I, ctypes.POINTER(D), I], I),
        "wz_kernel_launches": ([], ctypes.c_ulonglong),
        "wz_set_workspace_limit": ([P, ctypes.c_size_t], I),
        "wz_workspace_bytes": ([P], ctypes.c_size_t),
        "wz_selftest_wait_timeout": ([I, ctypes.POINTER(I), ctypes.POINTER(ctypes.c_longlong)], I),
        "wz_fma_peak": ([I, I, ctypes.POINTER(D), ctypes.POINTER(D)], I),
        "wz_probe_begin": ([I, I], I),
        "wz_probe_end": ([ctypes.POINTER(WzProbeResult)], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


LIB = _load()

EXPORTS = ("wz_create", "wz_destroy", "wz_last_error", "wz_supported_extent", "wz_set_phi", "wz_apply",
           "wz_solve", "wz_apply_mdagm_noalloc", "wz_get_phi", "wz_force", "wz_action", "wz_md_integrate",
           "wz_trajectory", "wz_batch_create", "wz_batch_destroy", "wz_batch_last_error", "wz_batch_size",
           "wz_batch_groups", "wz_batch_set_phi", "wz_batch_get_phi", "wz_batch_solve", "wz_batch_trajectory",
           "wz_solve_multishift", "wz_rational_minimax", "wz_spectral_bounds", "wz_rational_apply",
           "wz_rhmc_force", "wz_rhmc_trajectory", "wz_ward_identity", "wz_supercurrent", "wz_one_loop",
           "wz_aux_vev", "wz_locality", "wz_kernel_launches", "wz_probe_begin", "wz_probe_end",
           "wz_selftest_wait_timeout", "wz_set_workspace_limit", "wz_workspace_bytes", "wz_locality_op", "wz_fma_peak")


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def field_ptr(x, dtype=None):
    """(pointer, wz dtype) of a contiguous complex field (torch tensor or numpy array)."""
    if _is_torch(x):
        import torch
        if not x.is_contiguous():
            raise ValueError("field must be contiguous")
        dt = {torch.complex64: WZ_C64, torch.complex128: WZ_C128}.get(x.dtype)
        ptr = x.data_ptr()
    else:
        if not (isinstance(x, np.ndarray) and x.flags["C_CONTIGUOUS"]):
            raise ValueError("field must be a C-contiguous numpy array or torch tensor")
        dt = {np.dtype(np.complex64): WZ_C64, np.dtype(np.complex128): WZ_C128}.get(x.dtype)
        ptr = x.ctypes.data
    if dt is None:
        raise ValueError(f"unsupported dtype {x.dtype}")
    if dtype is not None and dt != dtype:
        raise ValueError("dtype mismatch")
    return ctypes.c_void_p(ptr), dt


def check(ctx, rc):
    if rc != WZ_OK:
        msg = LIB.wz_last_error(ctx).decode() if ctx else ""
        raise WzError(rc, msg)
    return rc


def make_params(dims, m=0.1, g=0.1, r=1.0, M0=1.0, yukawa=2.0):
    p = WzParams()
    for i in range(4):
        p.dims[i] = int(dims[i])
    m, g = complex(m), complex(g)
    p.m_re, p.m_im, p.g_re, p.g_im = m.real, m.imag, g.real, g.imag
    p.r, p.M0, p.yukawa = float(r), float(M0), float(yukawa)
    return p


def wz_create(params, stream=None):
    h = ctypes.c_void_p()
    check(None, LIB.wz_create(ctypes.byref(params), ctypes.c_void_p(stream or 0), ctypes.byref(h)))
    return h


def wz_destroy(ctx):
    return LIB.wz_destroy(ctx)


def wz_last_error(ctx):
    return LIB.wz_last_error(ctx).decode()


def wz_supported_extent(n):
    return bool(LIB.wz_supported_extent(int(n)))


def wz_set_phi(ctx, phi):
    ptr, dt = field_ptr(phi)
    if dt != WZ_C128:
        raise ValueError("phi must be complex128")
    return check(ctx, LIB.wz_set_phi(ctx, ptr))


def wz_apply(ctx, op, inp, out, nrhs, shift=0.0):
    pin, dt = field_ptr(inp)
    pout, _ = field_ptr(out, dt)
    op = OPS.get(op, op)
    return check(ctx, LIB.wz_apply(ctx, int(op), dt, pin, pout, int(nrhs), float(shift)))


def wz_solve(ctx, b, x, nrhs, shift=0.0, tol=1e-10, maxiter=100000, flags=WZ_SOLVE_MIXED, resid=False,
             raise_on_nonconvergence=True):
    """Returns (status, stats dict, per-RHS true residuals or None)."""
    pb, dt = field_ptr(b, WZ_C128)
    px, _ = field_ptr(x, WZ_C128)
    st = WzSolveStats()
    res = (ctypes.c_double * max(int(nrhs), 1))() if resid else None
    rc = LIB.wz_solve(ctx, pb, px, int(nrhs), float(shift), float(tol), int(maxiter), int(flags),
                      ctypes.byref(st), res)
    if rc not in (WZ_OK, WZ_NOT_CONVERGED) or (rc == WZ_NOT_CONVERGED and raise_on_nonconvergence):
        check(ctx, rc)
    return rc, st.as_dict(), (list(res)[:nrhs] if resid else None)


def wz_apply_mdagm_noalloc(ctx, inp, out, nrhs, shift=0.0):
    """(M^dag M + shift) inp with the static device scratch (no allocation)."""
    pin, dt = field_ptr(inp)
    pout, _ = field_ptr(out, dt)
    return check(ctx, LIB.wz_apply_mdagm_noalloc(ctx, dt, pin, pout, int(nrhs), float(shift)))


def wz_get_phi(ctx, phi):
    ptr, dt = field_ptr(phi, WZ_C128)
    return check(ctx, LIB.wz_get_phi(ctx, ptr))


def wz_force(ctx, eta, npf, grad, tol=1e-10, parts=WZ_FORCE_FERMION | WZ_FORCE_BOSON):
    """grad <- dS/dphi; returns (S_B, S_pf, solve stats)."""
    pe = field_ptr(eta, WZ_C128)[0] if npf > 0 else ctypes.c_void_p(0)
    pg, _ = field_ptr(grad, WZ_C128)
    sb, spf, st = ctypes.c_double(), ctypes.c_double(), WzSolveStats()
    check(ctx, LIB.wz_force(ctx, pe, int(npf), float(tol), int(parts), pg, ctypes.byref(sb),
                            ctypes.byref(spf), ctypes.byref(st)))
    return sb.value, spf.value, st.as_dict()


def wz_action(ctx, eta, npf, tol=1e-10):
    """(S_B, S_pf, solve stats) at the context's phi."""
    pe = field_ptr(eta, WZ_C128)[0] if npf > 0 else ctypes.c_void_p(0)
    sb, spf, st = ctypes.c_double(), ctypes.c_double(), WzSolveStats()
    check(ctx, LIB.wz_action(ctx, pe, int(npf), float(tol), ctypes.byref(sb), ctypes.byref(spf), ctypes.byref(st)))
    return sb.value, spf.value, st.as_dict()


def hmc_params(tau=1.0, nsteps=10, integrator="leapfrog", npf=1, tol=1e-10, maxiter=0, flags=0, seed=0,
               traj_index=0):
    return WzHmcParams(float(tau), int(nsteps), INTEGRATORS.get(integrator, integrator), int(npf), float(tol),
                       int(maxiter), int(flags), int(seed), int(traj_index))


def wz_md_integrate(ctx, pi, eta, npf, params):
    pp, _ = field_ptr(pi, WZ_C128)
    pe = field_ptr(eta, WZ_C128)[0] if npf > 0 else ctypes.c_void_p(0)
    st = WzTrajStats()
    check(ctx, LIB.wz_md_integrate(ctx, pp, pe, int(npf), ctypes.byref(params), ctypes.byref(st)))
    return st.as_dict()


def wz_trajectory(ctx, params):
    st = WzTrajStats()
    check(ctx, LIB.wz_trajectory(ctx, ctypes.byref(params), ctypes.byref(st)))
    return st.as_dict()


def wz_solve_multishift(ctx, b, x, nrhs, shifts, tol=1e-10, maxiter=100000, flags=WZ_SOLVE_MIXED, resid=False,
                        raise_on_nonconvergence=True):
    """x[i * nrhs + j] = (M^dag M + shifts[i])^-1 b[j]; returns (status, stats, residuals or None)."""
    pb, _ = field_ptr(b, WZ_C128)
    px, _ = field_ptr(x, WZ_C128)
    sh = (ctypes.c_double * len(shifts))(*[float(v) for v in shifts])
    st = WzSolveStats()
    nsys = int(nrhs) * len(shifts)
    res = (ctypes.c_double * max(nsys, 1))() if resid else None
    rc = LIB.wz_solve_multishift(ctx, pb, px, int(nrhs), len(shifts), sh, float(tol), int(maxiter), int(flags),
                                 ctypes.byref(st), res)
    if rc not in (WZ_OK, WZ_NOT_CONVERGED) or (rc == WZ_NOT_CONVERGED and raise_on_nonconvergence):
        check(ctx, rc)
    return rc, st.as_dict(), (list(res)[:nsys] if resid else None)


def wz_rational_minimax(power, lo, hi, d):
    """Minimax relative approximation of x^power on [lo, hi] (host computation)."""
    r = WzRational()
    rc = LIB.wz_rational_minimax(float(power), float(lo), float(hi), int(d), ctypes.byref(r))
    if rc != WZ_OK:
        raise WzError(rc, "wz_rational_minimax failed")
    return r


def wz_spectral_bounds(ctx):
    lo, hi = ctypes.c_double(), ctypes.c_double()
    check(ctx, LIB.wz_spectral_bounds(ctx, ctypes.byref(lo), ctypes.byref(hi)))
    return lo.value, hi.value


def _as_rational(r):
    return r if isinstance(r, WzRational) else rational_struct(r)


def wz_rational_apply(ctx, r, inp, out, nrhs, tol=1e-10, maxiter=100000, flags=WZ_SOLVE_MIXED, pc_cutoff=100.0):
    pin, _ = field_ptr(inp, WZ_C128)
    pout, _ = field_ptr(out, WZ_C128)
    st = WzSolveStats()
    rr = _as_rational(r)
    check(ctx, LIB.wz_rational_apply(ctx, ctypes.byref(rr), pin, pout, int(nrhs), float(tol), int(maxiter),
                                     int(flags), float(pc_cutoff), ctypes.byref(st)))
    return st.as_dict()


def wz_rhmc_force(ctx, eta, npf, action, grad, tol=1e-10, parts=WZ_FORCE_FERMION | WZ_FORCE_BOSON):
    """grad <- dS/dphi with the rational action; returns (S_B, S_pf, solve stats)."""
    pe = field_ptr(eta, WZ_C128)[0] if npf > 0 else ctypes.c_void_p(0)
    pg, _ = field_ptr(grad, WZ_C128)
    sb, spf, st = ctypes.c_double(), ctypes.c_double(), WzSolveStats()
    ra = _as_rational(action)
    check(ctx, LIB.wz_rhmc_force(ctx, pe, int(npf), ctypes.byref(ra), float(tol), int(parts), pg,
                                 ctypes.byref(sb), ctypes.byref(spf), ctypes.byref(st)))
    return sb.value, spf.value, st.as_dict()


def wz_rhmc_trajectory(ctx, params, action, heatbath):
    st = WzTrajStats()
    ra, rh = _as_rational(action), _as_rational(heatbath)
    check(ctx, LIB.wz_rhmc_trajectory(ctx, ctypes.byref(params), ctypes.byref(ra), ctypes.byref(rh),
                                      ctypes.byref(st)))
    return st.as_dict()


def wz_ward_identity(ctx, tol=1e-12, maxiter=100000, mixed=False):
    """(W_R, W_L) of Eq. exid at the context's phi, 4 x 4 complex numpy arrays, and solve stats."""
    wr, wl = (ctypes.c_double * 32)(), (ctypes.c_double * 32)()
    st = WzSolveStats()
    check(ctx, LIB.wz_ward_identity(ctx, float(tol), int(maxiter), WZ_SOLVE_MIXED if mixed else 0, wr, wl,
                                    ctypes.byref(st)))
    to = lambda a: (np.array(a[0::2]) + 1j * np.array(a[1::2])).reshape(4, 4)
    return to(wr), to(wl), st.as_dict()


def wz_supercurrent(ctx, w, T, tol=1e-12, maxiter=100000, mixed=False):
    """R[s, mu, dx, dy, a, b] of the supercurrent correlators (Eq. sitre) for the
    source weight w (complex128 (T, Z, Y, X), numpy or device tensor), and solve stats."""
    ptr, dt = field_ptr(w)
    if dt != WZ_C128:
        raise ValueError("w must be complex128")
    n = 2 * 4 * T * T * 16
    buf = (ctypes.c_double * (2 * n))()
    st = WzSolveStats()
    check(ctx, LIB.wz_supercurrent(ctx, ptr, float(tol), int(maxiter),
                                   WZ_SOLVE_MIXED if mixed else 0, buf, ctypes.byref(st)))
    out = np.ctypeslib.as_array(buf)
    R = (out[0::2] + 1j * out[1::2]).reshape(2, 4, T, T, 4, 4)
    return R, st.as_dict()


def wz_one_loop(N, ma):
    """(Z_phi - 1, Z_chi - 1, Z_F - 1) / |g|^2 of the one-loop sums on N^4 momenta."""
    z = (ctypes.c_double * 3)()
    rc = LIB.wz_one_loop(int(N), float(ma), z)
    if rc != WZ_OK:
        raise WzError(rc, "wz_one_loop failed")
    return tuple(z)


def wz_aux_vev(ctx, nm=1):
    """(1/V) sum_x F~(x) per member, as a list of complex numbers."""
    out = (ctypes.c_double * (2 * nm))()
    check(ctx, LIB.wz_aux_vev(ctx, out))
    return [complex(out[2 * j], out[2 * j + 1]) for j in range(nm)]


def wz_locality(ctx, dims, op=WZ_OP_DSLASH):
    """f(r), r = 0 .. T/2 + Z/2 + Y/2 + X/2, of Dslash (or the overlap D) on a point source."""
    n = sum(int(d) // 2 for d in dims) + 1
    out = (ctypes.c_double * n)()
    check(ctx, LIB.wz_locality_op(ctx, OPS.get(op, op), out, n))
    return np.array(list(out))


def wz_fma_peak(real_bytes, iters):
    """(TFLOP/s, ms) of the FMA throughput microkernel in FP64 (8) or FP32 (4)."""
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    check(None, LIB.wz_fma_peak(int(real_bytes), int(iters), ctypes.byref(tf), ctypes.byref(ms)))
    return tf.value, ms.value


def wz_selftest_wait_timeout(polls):
    """(status, cycles) of the bounded-wait self-test: WZ_ETIMEOUT when the wait ran out."""
    st, cyc = ctypes.c_int(-1), ctypes.c_longlong(0)
    check(None, LIB.wz_selftest_wait_timeout(int(polls), ctypes.byref(st), ctypes.byref(cyc)))
    return st.value, cyc.value


def wz_kernel_launches():
    return int(LIB.wz_kernel_launches())


def wz_probe_begin(kind, real_bytes):
    return check(None, LIB.wz_probe_begin(PROBE_KINDS.get(kind, kind), int(real_bytes)))


def wz_probe_end():
    r = WzProbeResult()
    check(None, LIB.wz_probe_end(ctypes.byref(r)))
    return {k: getattr(r, k) for k, _ in r._fields_}


class Lattice:
    """Owns one wz_ctx; methods forward to the C entry points of the same name."""

    def __init__(self, dims, m=0.1, g=0.1, r=1.0, M0=1.0, yukawa=2.0, stream=None):
        self.dims = tuple(int(d) for d in dims)
        self.params = make_params(dims, m, g, r, M0, yukawa)
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except ImportError:
                stream = None
        self.ctx = wz_create(self.params, stream)

    def close(self):
        if self.ctx:
            wz_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_phi(self, phi):
        return wz_set_phi(self.ctx, phi)

    def set_workspace_limit(self, nbytes):
        return check(self.ctx, LIB.wz_set_workspace_limit(self.ctx, int(nbytes)))

    def workspace_bytes(self):
        return int(LIB.wz_workspace_bytes(self.ctx))

    def _nrhs(self, f):
        n = f.numel() if _is_torch(f) else f.size
        return n // (4 * int(np.prod(self.dims)))

    def solve(self, b, x, shift=0.0, tol=1e-10, maxiter=100000, mixed=True, pc=False, resid=False,
              raise_on_nonconvergence=True):
        flags = (WZ_SOLVE_MIXED if mixed else 0) | (WZ_SOLVE_PC if pc else 0)
        return wz_solve(self.ctx, b, x, self._nrhs(b), shift, tol, maxiter, flags, resid,
                        raise_on_nonconvergence)

    def get_phi(self, phi):
        return wz_get_phi(self.ctx, phi)

    def solve_multishift(self, b, x, shifts, tol=1e-10, maxiter=100000, mixed=True, pc=False, resid=False):
        flags = (WZ_SOLVE_MIXED if mixed else 0) | (WZ_SOLVE_PC if pc else 0)
        return wz_solve_multishift(self.ctx, b, x, self._nrhs(b), shifts, tol, maxiter, flags, resid)

    def spectral_bounds(self):
        return wz_spectral_bounds(self.ctx)

    def rational_apply(self, r, inp, out, tol=1e-10, maxiter=100000, mixed=True, pc=False, pc_cutoff=100.0):
        flags = (WZ_SOLVE_MIXED if mixed else 0) | (WZ_SOLVE_PC if pc else 0)
        return wz_rational_apply(self.ctx, r, inp, out, self._nrhs(inp), tol, maxiter, flags, pc_cutoff)

    def rhmc_force(self, eta, npf, action, grad, tol=1e-10, parts=WZ_FORCE_FERMION | WZ_FORCE_BOSON):
        return wz_rhmc_force(self.ctx, eta, npf, action, grad, tol, parts)

    def rhmc_trajectory(self, action, heatbath, **kw):
        return wz_rhmc_trajectory(self.ctx, hmc_params(**kw), action, heatbath)

    def action(self, eta, npf, tol=1e-10):
        return wz_action(self.ctx, eta, npf, tol)

    def ward_identity(self, tol=1e-12, maxiter=100000, mixed=False):
        return wz_ward_identity(self.ctx, tol, maxiter, mixed)

    def supercurrent(self, w, tol=1e-12, maxiter=100000, mixed=False):
        return wz_supercurrent(self.ctx, w, self.dims[0], tol, maxiter, mixed)

    def aux_vev(self):
        return wz_aux_vev(self.ctx)[0]

    def locality(self, op="Dslash"):
        return wz_locality(self.ctx, self.dims, op)

    def force(self, eta, grad, tol=1e-10, parts=WZ_FORCE_FERMION | WZ_FORCE_BOSON):
        npf = 0 if eta is None else self._nrhs(eta)
        return wz_force(self.ctx, eta, npf, grad, tol, parts)

    def md_integrate(self, pi, eta, **kw):
        npf = 0 if eta is None else self._nrhs(eta)
        return wz_md_integrate(self.ctx, pi, eta, npf, hmc_params(npf=npf, **kw))

    def trajectory(self, **kw):
        return wz_trajectory(self.ctx, hmc_params(**kw))

    def apply(self, op, inp, out, nrhs=None, shift=0.0):
        if nrhs is None:
            nrhs = inp.numel() // (4 * int(np.prod(self.dims))) if _is_torch(inp) else inp.size // (4 * int(np.prod(self.dims)))
        return wz_apply(self.ctx, op, inp, out, nrhs, shift)


def _bcheck(b, rc, ok=(WZ_OK,)):
    if rc not in ok:
        raise WzError(rc, LIB.wz_batch_last_error(b).decode() if b else "")
    return rc


class Batch:
    """Independent lattices of uneven extent and coupling; forwards to wz_batch_*."""

    def __init__(self, lattices):
        """lattices: list of dicts with dims, m, g (and optionally r, M0, yukawa)."""
        self.n = len(lattices)
        self.dims = [tuple(int(d) for d in l["dims"]) for l in lattices]
        arr = (WzParams * self.n)()
        for i, l in enumerate(lattices):
            arr[i] = make_params(l["dims"], l.get("m", 0.1), l.get("g", 0.1), l.get("r", 1.0), l.get("M0", 1.0),
                                 l.get("yukawa", 2.0))
        h = ctypes.c_void_p()
        rc = LIB.wz_batch_create(arr, self.n, None, ctypes.byref(h))
        if rc != WZ_OK:
            raise WzError(rc, "wz_batch_create failed")
        self.h = h

    def close(self):
        if self.h:
            LIB.wz_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def groups(self):
        return LIB.wz_batch_groups(self.h)

    def set_phi(self, i, phi):
        return _bcheck(self.h, LIB.wz_batch_set_phi(self.h, int(i), field_ptr(phi, WZ_C128)[0]))

    def get_phi(self, i, phi):
        return _bcheck(self.h, LIB.wz_batch_get_phi(self.h, int(i), field_ptr(phi, WZ_C128)[0]))

    def solve(self, bs, xs, nrhs, tol=1e-10, maxiter=100000, mixed=True):
        pb = (ctypes.c_void_p * self.n)(*[field_ptr(b, WZ_C128)[0].value for b in bs])
        px = (ctypes.c_void_p * self.n)(*[field_ptr(x, WZ_C128)[0].value for x in xs])
        st = WzSolveStats()
        rc = LIB.wz_batch_solve(self.h, pb, px, int(nrhs), float(tol), int(maxiter),
                                WZ_SOLVE_MIXED if mixed else 0, ctypes.byref(st))
        _bcheck(self.h, rc)
        return st.as_dict()

    def trajectory(self, **kw):
        p = hmc_params(**kw)
        st = (WzTrajStats * self.n)()
        _bcheck(self.h, LIB.wz_batch_trajectory(self.h, ctypes.byref(p), st))
        return [x.as_dict() for x in st]
