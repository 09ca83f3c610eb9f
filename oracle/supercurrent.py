"""Naive lattice supercurrent (Eq. latsuc) and its correlators of Eq. sitre.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The current in tilded fields, with W' = m phi + g phi^2, is

    S_mu(x) = sqrt2 [ (D1 phi) gamma_mu P_+ + (D1 phi^*) gamma_mu P_-
                      + W' gamma_mu P_- + W'^* gamma_mu P_+ ] chi(x) = Gamma_mu(x) chi(x)

where D1 on the scalar is the gamma-matrix valued field sum_nu gamma_nu f_nu,
f_nu = F^-1[i sin p_nu / omega F f] (periodic grid), as in the Ward identity.
With the fermions integrated out at fixed phi, <chi(x) chi^T(z) C> = -M^-1(x, z)
(the propagator -M^-1 C^-1 of the action's sign, times C), so the correlators of
Eq. sitre are, per configuration, phi_s(y) Gamma_mu(x) (-M^-1)(x, z) with
phi_0 = phi, phi_1 = phi^*.

Measured form (readings, the paper gives only the tree-level result): both x and
y are projected on zero spatial momentum, and the source z is weighted by a
caller field w (a point, a wall or Gaussian noise):

    psi_b  = -M^-1 (w e_b),       xi(t) = sum_zvec w(t, zvec)
    Q_mu(t)[a][b]  = sum_xvec [Gamma_mu psi_b]_a(t, xvec)
    Phi_s(t)       = sum_yvec phi_s(t, yvec)
    R_s,mu(dx, dy)[a][b] = sum_t' xi(t')^* sgn(t', dx) Phi_s(t' + dy) Q_mu(t' + dx)[a][b]

with times mod T and sgn(t', dx) = -1 where t' + dx >= T (the antiperiodic
fermion propagator across the boundary), so dx and dy are the sink times
relative to the source.  For a point source R is the zero-momentum correlator of
that source; for noise with E[w(z) w^*(z')] = delta its mean is the sum over all
source positions.  At g = 0 its mean over the free scalar is the tree-level
expression the paper derives below Eq. sitre.
"""

import numpy as np

from . import cg as cg_mod
from . import fftops
from .conventions import GAMMA, P_MINUS, P_PLUS
from .ward import scalar_d1_components

SQRT2 = np.sqrt(2.0)


def current_columns(params, phi, psi, d1phi=None, d1phis=None):
    """Gamma_mu psi_b at every site, shape (4 mu, nb) + dims + (4,), psi of shape (nb,) + dims + (4,)."""
    if d1phi is None:
        d1phi = scalar_d1_components(params.dims, phi, params.r, params.M0)
    if d1phis is None:
        d1phis = scalar_d1_components(params.dims, np.conj(phi), params.r, params.M0)
    Wp = params.m * phi + params.g * phi ** 2
    out = []
    for mu in range(4):
        vp = psi @ (GAMMA[mu] @ P_PLUS).T  # gamma_mu P_+ psi
        vm = psi @ (GAMMA[mu] @ P_MINUS).T
        t = sum(d1phi[nu][..., None] * (vp @ GAMMA[nu].T) for nu in range(4))
        t = t + sum(d1phis[nu][..., None] * (vm @ GAMMA[nu].T) for nu in range(4))
        t = t + Wp[..., None] * vm + np.conj(Wp)[..., None] * vp
        out.append(SQRT2 * t)
    return np.stack(out)


def propagator_columns(params, phi, w, tol=1e-13):
    """psi_b = -M^-1 (w e_b) for b = 0..3, shape (4,) + dims + (4,)."""
    out = []
    for b in range(4):
        src = np.zeros(params.dims + (4,), np.complex128)
        src[..., b] = w
        x, _, _ = cg_mod.solve_MdagM(params, phi, fftops.apply_Mdag(params, phi, src), 0.0, tol)
        out.append(-x)
    return np.stack(out)


def correlators(params, phi, w, tol=1e-13):
    """R[s, mu, dx, dy, a, b] of the module docstring (complex, shape (2, 4, T, T, 4, 4))."""
    T = params.dims[0]
    psi = propagator_columns(params, phi, w, tol)
    cur = current_columns(params, phi, psi)  # (mu, b, T, Z, Y, X, a)
    Q = cur.sum(axis=(3, 4, 5))  # (mu, b, T, a)
    Q = np.transpose(Q, (0, 2, 3, 1))  # (mu, t, a, b)
    Phi = [phi.sum(axis=(1, 2, 3)), np.conj(phi).sum(axis=(1, 2, 3))]
    xi = w.sum(axis=(1, 2, 3))
    R = np.zeros((2, 4, T, T, 4, 4), np.complex128)
    for s in range(2):
        for dx in range(T):
            for dy in range(T):
                acc = np.zeros((4, 4, 4), np.complex128)
                for tp in range(T):
                    sgn = -1.0 if tp + dx >= T else 1.0
                    acc += np.conj(xi[tp]) * sgn * Phi[s][(tp + dy) % T] * Q[:, (tp + dx) % T]
                R[s, :, dx, dy] = acc
    return R
