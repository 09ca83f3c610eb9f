"""Hybrid Monte Carlo trajectory (Sec. 7.2, molecular dynamics and Metropolis).

TEST INFRASTRUCTURE ONLY (see the package docstring).

One trajectory with npf pseudofermions and a single pole (beta = 0):

    eta_k = M^dagger(phi0) R_k                       (heatbath; R_k ~ exp(-|R|^2))
    H     = 1/2 sum |pi|^2 + S_B(phi) + sum_k eta_k^dagger (M^dagger M)^-1 eta_k
    MD    : d phi / d tau = pi,  d pi / d tau = -G(phi)   (G of ``force``)
    accept with probability min(1, exp(-(H1 - H0)))

RHMC (Secs. 7.2, 7.4): with rational approximations r_a ~ x^-gamma (action, Eq. jkjk)
and r_h ~ x^(gamma/2) (heatbath, Eq. hbeq),

    eta_k = r_h(M^dagger M(phi0)) R_k,   S_pf = sum_k eta_k^dagger r_a(M^dagger M) eta_k,

and the force of ``force.rational_pf_force``; the paper's phase-quenched
det(M^dagger M)^1/4 has gamma = 1/4.

Integrators: leapfrog (momentum half steps at both ends) and the
second-order minimum-norm scheme of Omelyan, Mryglod and Folk with
lambda = 0.1931833275037836.  phi and pi are complex arrays whose real and
imaginary parts are the two real fields.
"""

import numpy as np

from . import cg as cg_mod
from . import fftops
from . import force as force_mod
from . import rational

OMELYAN_LAMBDA = 0.1931833275037836


def total_force(params, phi, etas, tol):
    G = force_mod.bosonic_force(params, phi)
    for eta in etas:
        G = G + force_mod.pf_force(params, phi, eta, 0.0, tol)
    return G


def hamiltonian(params, phi, pi, etas, tol):
    H = 0.5 * float(np.vdot(pi, pi).real) + force_mod.bosonic_action(params, phi)
    for eta in etas:
        X, _, _ = cg_mod.solve_MdagM(params, phi, eta, 0.0, tol)
        H += float(np.vdot(eta, X).real)
    return H


def integrate(params, phi, pi, etas, tau, nsteps, integrator="leapfrog", tol=1e-13, force_fn=None):
    """Molecular-dynamics evolution; returns (phi, pi, n_force_evaluations).

    force_fn(params, phi, etas, tol) replaces ``total_force`` when given."""
    eps = tau / nsteps
    nforce = 0
    F = force_fn if force_fn is not None else total_force
    if integrator == "leapfrog":
        pi = pi - 0.5 * eps * F(params, phi, etas, tol)
        nforce += 1
        for step in range(nsteps):
            phi = phi + eps * pi
            w = eps if step < nsteps - 1 else 0.5 * eps
            pi = pi - w * F(params, phi, etas, tol)
            nforce += 1
        return phi, pi, nforce
    if integrator == "omelyan":
        lam = OMELYAN_LAMBDA
        for _ in range(nsteps):
            pi = pi - lam * eps * F(params, phi, etas, tol)
            phi = phi + 0.5 * eps * pi
            pi = pi - (1.0 - 2.0 * lam) * eps * F(params, phi, etas, tol)
            phi = phi + 0.5 * eps * pi
            pi = pi - lam * eps * F(params, phi, etas, tol)
            nforce += 3
        return phi, pi, nforce
    raise ValueError(integrator)


def trajectory(params, phi0, pi0, R, u, tau=1.0, nsteps=10, integrator="leapfrog", tol=1e-13):
    """Run one trajectory from given random draws.

    R has shape (npf,) + dims + (4,); u is the Metropolis uniform.
    Returns a dict with phi (accepted or restored), phi_md (end of MD), H0, H1,
    dH and accept.
    """
    etas = [fftops.apply_Mdag(params, phi0, Rk) for Rk in R]
    H0 = hamiltonian(params, phi0, pi0, etas, tol)
    phi1, pi1, _ = integrate(params, phi0, pi0, etas, tau, nsteps, integrator, tol)
    H1 = hamiltonian(params, phi1, pi1, etas, tol)
    dH = H1 - H0
    accept = bool(u <= np.exp(-dH)) if dH > 0 else True
    return {
        "phi": phi1 if accept else phi0,
        "phi_md": phi1,
        "pi_md": pi1,
        "H0": H0,
        "H1": H1,
        "dH": dH,
        "accept": accept,
        "etas": etas,
    }


def rational_total_force(coef_action):
    def f(params, phi, etas, tol):
        G = force_mod.bosonic_force(params, phi)
        for eta in etas:
            G = G + force_mod.rational_pf_force(params, phi, eta, coef_action, tol)
        return G

    return f


def rational_hamiltonian(params, phi, pi, etas, coef_action, tol):
    H = 0.5 * float(np.vdot(pi, pi).real) + force_mod.bosonic_action(params, phi)
    for eta in etas:
        H += force_mod.rational_pf_action(params, phi, eta, coef_action, tol)
    return H


def rhmc_trajectory(params, phi0, pi0, R, u, coef_action, coef_heat, tau=1.0, nsteps=10, integrator="leapfrog",
                    tol=1e-13):
    """One RHMC trajectory from given draws (R: (npf,) + dims + (4,), u: uniform)."""
    etas = [rational.rational_apply(params, phi0, Rk, coef_heat, tol) for Rk in R]
    H0 = rational_hamiltonian(params, phi0, pi0, etas, coef_action, tol)
    phi1, pi1, _ = integrate(params, phi0, pi0, etas, tau, nsteps, integrator, tol,
                             force_fn=rational_total_force(coef_action))
    H1 = rational_hamiltonian(params, phi1, pi1, etas, coef_action, tol)
    dH = H1 - H0
    accept = bool(u <= np.exp(-dH)) if dH > 0 else True
    return {
        "phi": phi1 if accept else phi0,
        "phi_md": phi1,
        "pi_md": pi1,
        "H0": H0,
        "H1": H1,
        "dH": dH,
        "accept": accept,
        "etas": etas,
    }
