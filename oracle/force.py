"""Actions and molecular-dynamics forces (Eq. acws, Secs. 7.2 and 7.4).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Bosonic action (Eq. acws with a = 1, F~ integrated out):

    S_B = sum_x [ 2 phi^* (D2 phi) + W'^* (K W') ],  W' = m phi + g phi^2,
    K = 1 - D2/2,  scalar fields periodic in all directions.

Pseudofermion action with one pole (the single-pole form of Eq. jkjk, alpha=1):

    S_pf = eta^dagger (M^dagger M + beta)^-1 eta.

With the rational approximation of Eq. jkjk, r(x) = alpha_0 + sum_i alpha_i/(x + beta_i)
(``rational``), the pseudofermion action is eta^dagger r(M^dagger M) eta; alpha_0 eta^dagger eta
does not depend on phi, so its force is the alpha_i-weighted sum of single-pole forces
with shifts beta_i.

Forces are returned as the complex array G = dS/dphi_R + i dS/dphi_I, i.e. the
gradient with respect to the real and imaginary parts of phi at every site.

    G_B  = 4 (D2 phi) + 2 conj(m + 2 g phi) (K W')
    G_pf = -2 Re[Z^dagger dM/dphi_R X] - 2 i Re[Z^dagger dM/dphi_I X],
           X = (M^dagger M + beta)^-1 eta,  Z = M X,
           dM/dphi_R = c g P_+ + c g^* P_-,  dM/dphi_I = i c g P_+ - i c g^* P_-
"""

import numpy as np

from . import cg as cg_mod
from . import fftops
from . import rational


def superpotential_derivative(params, phi):
    """W'(phi) = m phi + g phi^2."""
    return params.m * phi + params.g * phi * phi


def bosonic_action(params, phi):
    D2phi = fftops.apply_D2_scalar(params, phi)
    W = superpotential_derivative(params, phi)
    KW = fftops.apply_K_scalar(params, W)
    return float((2.0 * np.vdot(phi, D2phi) + np.vdot(W, KW)).real)


def bosonic_force(params, phi):
    D2phi = fftops.apply_D2_scalar(params, phi)
    KW = fftops.apply_K_scalar(params, superpotential_derivative(params, phi))
    return 4.0 * D2phi + 2.0 * np.conj(params.m + 2.0 * params.g * phi) * KW


def pf_action(params, phi, eta, shift=0.0, tol=1e-13):
    X, _, _ = cg_mod.solve_MdagM(params, phi, eta, shift, tol)
    return float(np.vdot(eta, X).real)


def pf_force_from_solution(params, phi, X):
    """Site-local contraction -2 Re[Z^dagger dM X] with Z = M X."""
    c = params.yukawa
    g = params.g
    Z = fftops.apply_M(params, phi, X)
    cplus = np.sum(np.conj(Z[..., 2:4]) * X[..., 2:4], axis=-1)
    cminus = np.sum(np.conj(Z[..., 0:2]) * X[..., 0:2], axis=-1)
    dR = -2.0 * np.real(c * g * cplus + c * np.conj(g) * cminus)
    dI = -2.0 * np.real(1j * c * g * cplus - 1j * c * np.conj(g) * cminus)
    return dR + 1j * dI


def pf_force(params, phi, eta, shift=0.0, tol=1e-13):
    X, _, _ = cg_mod.solve_MdagM(params, phi, eta, shift, tol)
    return pf_force_from_solution(params, phi, X)


def auxiliary_vev(params, phi):
    """(1/V) sum_x F~(x) on the equation of motion of Eq. lata.

    Varying Eq. lata with respect to F~^* gives
    F~ = -(1 - D2/2)(m^* phi^* + g^* phi^*2); K(p=0) = 1 so the volume average
    reduces to -(1/V) sum_x (m^* phi^* + g^* phi^*2).
    """
    w = np.conj(params.m) * np.conj(phi) + np.conj(params.g) * np.conj(phi) ** 2
    return complex(-np.mean(fftops.apply_K_scalar(params, w)))


def rational_pf_action(params, phi, eta, coef, tol=1e-13):
    """eta^dagger r(M^dagger M) eta with r of Eq. jkjk (coefficients ``coef``)."""
    return float(np.vdot(eta, rational.rational_apply(params, phi, eta, coef, tol)).real)


def rational_pf_force(params, phi, eta, coef, tol=1e-13):
    """Gradient of ``rational_pf_action``: sum_i alpha_i G_pf(beta_i)."""
    G = np.zeros(phi.shape, dtype=complex)
    for a, b in zip(coef["alpha"], coef["beta"]):
        G = G + a * pf_force(params, phi, eta, float(b), tol)
    return G
