"""Plain conjugate gradient on M^dagger M + beta (Sec. 7.2, Eqs. theprob, yuier).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Textbook Hestenes-Stiefel CG for a Hermitian positive-definite operator, FP64,
x0 = 0, stopped when the recursive relative residual drops below tol; the true
relative residual ||b - A x|| / ||b|| is recomputed at the end.  The
preconditioned variant solves M~^dagger M~ x~ = b~ with M~ = M M0^-1,
x~ = M0 x, b~ = (M0^-1)^dagger b and returns x = M0^-1 x~ (Sec. 7.3).
"""

import numpy as np

from . import fftops


def vdot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def cg(apply_A, b, tol=1e-12, maxiter=100000):
    """Return (x, iterations, true_relative_residual)."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = vdot(r, r).real
    bnorm = np.sqrt(vdot(b, b).real)
    it = 0
    if bnorm == 0.0:
        return x, 0, 0.0
    while np.sqrt(rr) > tol * bnorm and it < maxiter:
        Ap = apply_A(p)
        alpha = rr / vdot(p, Ap).real
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    res = b - apply_A(x)
    return x, it, float(np.sqrt(vdot(res, res).real) / bnorm)


def solve_MdagM(params, phi, b, shift=0.0, tol=1e-12, maxiter=100000):
    """Unpreconditioned CG on (M^dagger M + shift) x = b."""
    return cg(lambda v: fftops.apply_MdagM(params, phi, v, shift), b, tol, maxiter)


def solve_MdagM_pc(params, phi, b, tol=1e-12, maxiter=100000):
    """M0^-1 preconditioned CG (Sec. 7.3); returns x of the original problem.

    The stopping test is on the preconditioned residual; the returned residual
    is the true one of M^dagger M x = b.
    """
    bt = fftops.apply_M0inv(params, b, dagger=True)

    def A(v):
        return fftops.apply_Mtilde_dag(params, phi, fftops.apply_Mtilde(params, phi, v))

    xt, it, _ = cg(A, bt, tol, maxiter)
    x = fftops.apply_M0inv(params, xt)
    res = b - fftops.apply_MdagM(params, phi, x)
    return x, it, float(np.sqrt(vdot(res, res).real / vdot(b, b).real))


def true_residual(params, phi, b, x, shift=0.0):
    res = b - fftops.apply_MdagM(params, phi, x, shift)
    return float(np.sqrt(vdot(res, res).real / vdot(b, b).real))
