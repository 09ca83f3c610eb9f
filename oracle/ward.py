"""Broken supersymmetric Ward-Takahashi identity of Eq. exid, per configuration.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The identity relates the volume sum of the auxiliary field to the correlation
of the variation density S(x) of the action (Eq. uity) with the fermion summed
over the lattice.  The sum over x of S is the cubic expression of Eq. nzav, so
that with the fermions integrated out at a fixed scalar field (Majorana
propagator <chi(z) chi^T(y)> = -(C M)^-1(z, y) = -M^-1 C^-1 for the action's sign,
see the readings) both sides are computable per configuration:

    W_L[a, b] = F_b C[a, b],   F_b = sum_x F~ for b in P_+ (2, 3), sum_x F~^* for b in P_- (0, 1),
                               F~ = -(1 - D2/2)(m^* phi^* + g^* phi^*2)
    W_R[a, b] = sum_x [ Kop psi_b ]_a(x),  psi_b = M^-1 C^-1 u_b,  u_b(x) = e_b at every x
    Kop psi   = g (2 phi (D1 phi) P_+ psi + phi^2 D1 P_+ psi)
              + g^* (2 phi^* (D1 phi^*) P_- psi + phi^*2 D1 P_- psi)

D1 is the gamma-odd part of the overlap operator: on spinors (antiperiodic time)
i gamma.sin p / omega in momentum space; on a scalar field f (periodic) it is the
gamma-matrix valued field (D1 f)(x) = sum_mu gamma_mu f_mu(x),
f_mu = F^-1[i sin p_mu / omega(p) F[f]].  The common factor of the
transformation (sqrt 2 on both sides) is left out.  The identity states
<W_R> = <W_L> over the measure; in the continuum both vanish.

Readings (the paper leaves them implicit): the sum over y of the fermion makes
the source uniform, so no stochastic estimate is needed.  The left side is the
contact term of the source derivative before the paper's abbreviation: the
variation of chi~_b carries F~ in the P_+ rows and F~^* in the P_- rows.  With
exp(-S) and S = -sum (1/2) chi^T C M chi + ..., <chi chi^T> = -M^-1 C^-1; that sign
and C_ba = -C_ab make the identity <W_R> = <W_L> with W_R as defined (propagator
M^-1 C^-1).  The printed Eq. exid carries the opposite sign; the pin below decides.

Pins (tests/test_oracle_ward.py): W_R against a dense position-space route, its
zero at g = 0, the scalar D1 of a plane wave, and the identity <W_R> = <W_L>
itself over the exact measure Pf(CM) exp(-S_B) on a lattice where the
reduction of Eq. nzav is exact (T = 3, periodic fermions), which fixes the
sign and the chirality structure of W_L.
"""

import numpy as np

from . import cg as cg_mod
from . import fftops, momentum
from .conventions import CCONJ, GAMMA, P_MINUS, P_PLUS


def scalar_d1_components(dims, f, r=1.0, M0=1.0):
    """f_mu(x) = F^-1[i sin p_mu / omega F[f]] on the periodic grid, shape (4,) + dims."""
    _, omega, s = momentum.symbol_parts(dims, r, M0, fermion=False)
    fh = np.fft.fftn(f)
    return np.stack([np.fft.ifftn(1j * s[mu] / omega * fh) for mu in range(4)])


def spinor_d1(params, psi):
    """D1 psi with antiperiodic time (i gamma.sin p / omega in momentum space)."""
    D1, _ = momentum.D1_D2(params.dims, params.r, params.M0, fermion=True)
    return fftops.ifft4_fermion(fftops.spin_mult(D1, fftops.fft4_fermion(psi)))


def propagator_columns(params, phi, tol=1e-13):
    """psi_b = M^-1 C^-1 u_b for b = 0..3 (four uniform sources), shape (4,) + dims + (4,)."""
    dims = params.dims
    Cinv = np.linalg.inv(CCONJ)
    out = []
    for b in range(4):
        src = np.broadcast_to(Cinv[:, b], dims + (4,)).astype(np.complex128)
        rhs = fftops.apply_Mdag(params, phi, src)
        x, _, _ = cg_mod.solve_MdagM(params, phi, rhs, 0.0, tol)
        out.append(x)
    return np.stack(out)


def kop(params, phi, psi, d1phi=None, d1phis=None):
    """Kop psi of the module docstring (site field, shape dims + (4,))."""
    g = params.g
    if d1phi is None:
        d1phi = scalar_d1_components(params.dims, phi, params.r, params.M0)
    if d1phis is None:
        d1phis = scalar_d1_components(params.dims, np.conj(phi), params.r, params.M0)
    pp = psi @ P_PLUS.T  # P_+ psi at every site
    pm = psi @ P_MINUS.T
    d1p = spinor_d1(params, pp)
    d1m = spinor_d1(params, pm)
    # (D1 f) P psi = sum_mu f_mu gamma_mu (P psi)
    gp = sum(d1phi[mu][..., None] * (pp @ GAMMA[mu].T) for mu in range(4))
    gm = sum(d1phis[mu][..., None] * (pm @ GAMMA[mu].T) for mu in range(4))
    ph = phi[..., None]
    return g * (2.0 * ph * gp + ph ** 2 * d1p) + np.conj(g) * (2.0 * np.conj(ph) * gm + np.conj(ph) ** 2 * d1m)


def ward_right(params, phi, tol=1e-13):
    """W_R[a, b] = sum_x [Kop psi_b]_a(x)."""
    cols = propagator_columns(params, phi, tol)
    d1phi = scalar_d1_components(params.dims, phi, params.r, params.M0)
    d1phis = scalar_d1_components(params.dims, np.conj(phi), params.r, params.M0)
    W = np.zeros((4, 4), dtype=np.complex128)
    for b in range(4):
        W[:, b] = kop(params, phi, cols[b], d1phi, d1phis).reshape(-1, 4).sum(axis=0)
    return W


def ward_left(params, phi):
    """W_L[a, b] = F_b C[a, b]; K(p = 0) = 1 makes sum_x F~ = -sum_x (m^* phi^* + g^* phi^*2)."""
    Fsum = -np.sum(np.conj(params.m) * np.conj(phi) + np.conj(params.g) * np.conj(phi) ** 2)
    Fb = np.array([np.conj(Fsum), np.conj(Fsum), Fsum, Fsum])
    return CCONJ * Fb[None, :]
