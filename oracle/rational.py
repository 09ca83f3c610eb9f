"""Rational approximation of powers of M^dagger M (Eq. jkjk, Eq. hbeq, Sec. 7.4).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The pseudofermion action needs (M^dagger M)^-1/4 and the heatbath (M^dagger M)^1/8;
both are replaced by a rational function of degree d in partial fractions,

    x^gamma  ~  r(x) = alpha_0 + sum_{i=1}^d alpha_i / (x + beta_i),    x in [lo, hi],

so that r(M^dagger M) eta needs the d shifted solves (M^dagger M + beta_i) X_i = eta
of Eq. yuier.  The paper wants the coefficients that make the error smallest over
the eigenvalue range (taken from the free operator M0^dagger M0 at weak coupling)
and prints none.  Reading taken here: the minimax RELATIVE error
max_x |r(x) / x^gamma - 1| over [lo, hi], type (d, d).

``minimax`` is the classical Remez exchange written in the coefficient form
r = P/Q (P, Q polynomials of degree d in y = x / sqrt(lo hi)), in mpmath with
enough digits for the monomial basis:

  1. P/Q interpolates y^gamma at 2d+1 points spread in log y (a linear solve);
  2. the reference is 2d+2 alternating extrema of e(y) = P/(Q y^gamma) - 1;
  3. Newton on P(y_j) - y_j^gamma (1 + s_j h) Q(y_j) = 0 (j = 0..2d+1,
     s_j = +-1 alternating) for the coefficients and the level h;
  4. 2-3 repeat until the extrema are level.
The poles -beta_i are the roots of Q; the residues are P/Q' there.

``zolotarev_inverse_sqrt`` is Zolotarev's closed-form optimum for gamma = -1/2
(Jacobi elliptic functions from scipy), used only to pin ``minimax``.
"""

import math

import numpy as np

from . import cg as cg_mod


def _working_dps(d, kappa):
    # the Vandermonde matrices span kappa^(+-d/2); keep ~35 digits beyond that
    return int(40 + d * math.log10(max(kappa, 10.0)) * 0.75)


def minimax(gamma, lo, hi, d, level_tol=1e-10, max_exchanges=60):
    """Coefficients {a0, alpha, beta, err} of the minimax relative approximation.

    err is the levelled error |h| of the final reference (the maximum relative
    error over [lo, hi] when the exchange has converged).
    """
    import mpmath as mp

    if not (0.0 < lo < hi) or d < 0:
        raise ValueError("need 0 < lo < hi and d >= 0")
    kappa = hi / lo
    mp.mp.dps = _working_dps(d, kappa)
    g = mp.mpf(gamma)
    s = mp.sqrt(mp.mpf(lo) * mp.mpf(hi))
    ylo, yhi = mp.mpf(lo) / s, mp.mpf(hi) / s
    Llo, Lhi = mp.log(ylo), mp.log(yhi)
    n = 2 * d + 2

    def P_of(c, y):
        return mp.polyval(list(reversed(c[: d + 1])), y)

    def Q_of(c, y):
        return mp.polyval(list(reversed([mp.mpf(1)] + list(c[d + 1: 2 * d + 1]))), y)

    def err(c, y):
        return P_of(c, y) / (Q_of(c, y) * y ** g) - 1

    # 1. rational interpolation at 2d+1 points in log y (unknowns p_0..p_d, q_1..q_d)
    mid, half = (Llo + Lhi) / 2, (Lhi - Llo) / 2
    nodes = [mp.exp(mid + half * mp.cos(mp.pi * (k + mp.mpf(1) / 2) / (2 * d + 1))) for k in range(2 * d + 1)]
    A = mp.matrix(2 * d + 1, 2 * d + 1)
    rhs = mp.matrix(2 * d + 1, 1)
    for j, y in enumerate(nodes):
        f = y ** g
        for k in range(d + 1):
            A[j, k] = y ** k
        for k in range(1, d + 1):
            A[j, d + k] = -f * y ** k
        rhs[j] = f
    coef = list(mp.lu_solve(A, rhs)) if d > 0 else [mp.mpf(1)]  # d = 0: exact at y = 1

    # 2. alternating extrema of the relative error on a log grid refined by golden section
    def extrema(c):
        G = 24 * n
        grid = [mid - half * mp.cos(mp.pi * k / (G - 1)) for k in range(G)]  # ln y, dense at the ends
        e = [err(c, mp.exp(u)) for u in grid]
        idx = [0] + [k for k in range(1, G - 1) if (e[k] - e[k - 1]) * (e[k + 1] - e[k]) <= 0] + [G - 1]
        pts, vals = [], []
        for k in idx:
            if k in (0, G - 1):
                u = grid[k]
            else:
                sg = 1 if e[k] > 0 else -1
                a, b = grid[k - 1], grid[k + 1]
                gr = (mp.sqrt(5) - 1) / 2
                x1, x2 = b - gr * (b - a), a + gr * (b - a)
                f1, f2 = sg * err(c, mp.exp(x1)), sg * err(c, mp.exp(x2))
                for _ in range(40):
                    if f1 > f2:
                        b, x2, f2 = x2, x1, f1
                        x1 = b - gr * (b - a)
                        f1 = sg * err(c, mp.exp(x1))
                    else:
                        a, x1, f1 = x1, x2, f2
                        x2 = a + gr * (b - a)
                        f2 = sg * err(c, mp.exp(x2))
                u = (a + b) / 2
            v = err(c, mp.exp(u))
            if pts and (v > 0) == (vals[-1] > 0):
                if abs(v) > abs(vals[-1]):
                    pts[-1], vals[-1] = u, v
            else:
                pts.append(u)
                vals.append(v)
        while len(pts) > n:  # drop the smaller end
            if abs(vals[0]) < abs(vals[-1]):
                pts.pop(0)
                vals.pop(0)
            else:
                pts.pop()
                vals.pop()
        if len(pts) < n:
            raise RuntimeError("Remez: fewer than 2d+2 alternating extrema")
        return [mp.exp(u) for u in pts], vals

    ref, vals = extrema(coef)
    h = mp.mpf(0)
    for _ in range(max_exchanges):
        sig = [1 if vals[0] > 0 else -1]
        for _j in range(1, n):
            sig.append(-sig[-1])
        # 3. Newton on the levelled-error equations
        x = list(coef) + [abs(h)]
        for _it in range(50):
            F = mp.matrix(n, 1)
            J = mp.matrix(n, n)
            for j, y in enumerate(ref):
                f = y ** g
                Pv = P_of(x, y)
                Qv = Q_of(x, y)
                lev = 1 + sig[j] * x[n - 1]
                F[j] = (Pv - f * lev * Qv) / f
                for k in range(d + 1):
                    J[j, k] = y ** k / f
                for k in range(1, d + 1):
                    J[j, d + k] = -lev * y ** k
                J[j, n - 1] = -sig[j] * Qv
            dx = mp.lu_solve(J, -F)
            x = [x[k] + dx[k] for k in range(n)]
            if mp.norm(dx, mp.inf) < mp.mpf(10) ** (-(mp.mp.dps - 10)):
                break
        coef, h = x[: n - 1], x[n - 1]
        ref, vals = extrema(coef)
        mags = [abs(v) for v in vals]
        if (max(mags) - min(mags)) / max(mags) < level_tol:
            break
    else:
        raise RuntimeError("Remez: extrema did not level")

    # partial fractions in x: r(x) = s^gamma P(x/s) / Q(x/s)
    sg = s ** g
    if d == 0:
        return {"gamma": gamma, "lo": lo, "hi": hi, "d": 0, "a0": float(sg * coef[0]),
                "alpha": np.zeros(0), "beta": np.zeros(0), "err": float(max(mags))}
    qdesc = [coef[d + k] for k in range(d, 0, -1)] + [mp.mpf(1)]  # q_d .. q_1, 1
    roots = mp.polyroots(qdesc, maxsteps=400, extraprec=4 * mp.mp.dps)
    dq = [k * coef[d + k] for k in range(d, 0, -1)]  # Q' descending
    alpha, beta = [], []
    for yr in roots:
        if abs(mp.im(yr)) > mp.mpf(10) ** (-mp.mp.dps // 3) * abs(yr) or mp.re(yr) >= 0:
            raise RuntimeError("Remez: a pole is not on the negative real axis")
        yr = mp.re(yr)
        beta.append(-s * yr)
        alpha.append(sg * s * P_of(coef, yr) / mp.polyval(dq, yr))
    order = sorted(range(d), key=lambda i: beta[i])
    a0 = sg * coef[d] / coef[2 * d]
    return {
        "gamma": gamma,
        "lo": lo,
        "hi": hi,
        "d": d,
        "a0": float(a0),
        "alpha": np.array([float(alpha[i]) for i in order]),
        "beta": np.array([float(beta[i]) for i in order]),
        "err": float(max(mags)),
    }


def evaluate(coef, x):
    """r(x) = alpha_0 + sum_i alpha_i / (x + beta_i) (numpy, elementwise)."""
    x = np.asarray(x, dtype=float)
    out = np.full_like(x, coef["a0"])
    for a, b in zip(coef["alpha"], coef["beta"]):
        out = out + a / (x + b)
    return out


def relative_error(coef, gamma, x):
    x = np.asarray(x, dtype=float)
    return evaluate(coef, x) / x ** gamma - 1.0


def rational_apply(params, phi, eta, coef, tol=1e-13):
    """r(M^dagger M) eta = alpha_0 eta + sum_i alpha_i (M^dagger M + beta_i)^-1 eta (Eq. jkjk)."""
    out = coef["a0"] * eta
    for a, b in zip(coef["alpha"], coef["beta"]):
        X, _, _ = cg_mod.solve_MdagM(params, phi, eta, float(b), tol)
        out = out + a * X
    return out


def zolotarev_inverse_sqrt(lo, hi, d):
    """Zolotarev's best relative approximation of x^-1/2 on [lo, hi], type (d, d).

    r(x) = C prod_{l=1}^d (x + c_{2l}) / (x + c_{2l-1}),
    c_l = lo sn^2(u_l; k'^2) / cn^2(u_l; k'^2), u_l = l K(k'^2) / (2d + 1),
    k'^2 = 1 - lo/hi; C levels the error.  Returns (poles c_odd, zeros c_even,
    C, err) with err measured on a dense log grid.
    """
    from scipy.special import ellipj, ellipk

    m = 1.0 - lo / hi
    K = ellipk(m)
    l = np.arange(1, 2 * d + 1)
    sn, cn, _, _ = ellipj(l * K / (2 * d + 1), m)
    c = lo * sn ** 2 / cn ** 2
    poles, zeros = c[0::2], c[1::2]
    x = np.exp(np.linspace(np.log(lo), np.log(hi), 200001))
    prod = np.ones_like(x)
    for z, p in zip(zeros, poles):
        prod *= (x + z) / (x + p)
    g = prod * np.sqrt(x)
    C = 2.0 / (g.max() + g.min())
    err = (g.max() - g.min()) / (g.max() + g.min())
    return poles, zeros, C, err
