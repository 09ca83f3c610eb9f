"""Fermion matrix M(phi) applied through the 4D FFT (Sec. 7.2, Eq. fmat).

TEST INFRASTRUCTURE ONLY (see the package docstring).

    M      = Dslash + Y,        Y      = (m + c g phi) P_+ + (m^* + c g^* phi^*) P_-
    M^dag  = -Dslash + Y^dag,   Y^dag  = (m^* + c g^* phi^*) P_+ + (m + c g phi) P_-

Dslash is anti-Hermitian and diagonal in momentum space, so it is applied as
"FFT, multiply by Dslash(p), inverse FFT" (the paper's "FFT trick", Sec. 7.2).
The fermion field is antiperiodic in time: multiplying by exp(-i pi t / T)
before a plain DFT over t yields the momenta p_t = pi (2n + 1) / T.
"""

import numpy as np

from .conventions import P_MINUS, P_PLUS
from . import momentum


def _twist(dims, sign):
    T = dims[0]
    t = np.arange(T, dtype=np.float64)
    return np.exp(sign * 1j * np.pi * t / T)[:, None, None, None]


def fft4_fermion(psi):
    """psi(x) (T, Z, Y, X, 4) -> psi_hat(p) on the antiperiodic-time grid."""
    dims = psi.shape[:4]
    tw = _twist(dims, -1.0)[..., None]
    return np.fft.fftn(psi * tw, axes=(0, 1, 2, 3))


def ifft4_fermion(psi_hat):
    """Inverse of fft4_fermion (includes the 1/V normalisation)."""
    dims = psi_hat.shape[:4]
    tw = _twist(dims, +1.0)[..., None]
    return np.fft.ifftn(psi_hat, axes=(0, 1, 2, 3)) * tw


def spin_mult(Mp, v):
    """out[..., a] = sum_b Mp[..., a, b] v[..., b]."""
    return np.einsum("...ab,...b->...a", Mp, v)


def apply_dslash(psi, r=1.0, M0=1.0, sign=+1.0):
    """sign * Dslash psi via FFT -> multiply -> inverse FFT."""
    dims = psi.shape[:4]
    Dp = momentum.dslash_symbol(dims, r, M0)
    return ifft4_fermion(sign * spin_mult(Dp, fft4_fermion(psi)))


def apply_overlap(psi, r=1.0, M0=1.0):
    """D psi with the overlap operator D = 1 - V, V = A (A^dag A)^-1/2, applied as
    FFT -> multiply by D(p) = 1 - (b(p) - i gamma.sin p)/omega(p) -> inverse FFT
    (Sec. 2.2; the kernel of Sec. 3.1's Eq. d1mom in momentum space)."""
    dims = psi.shape[:4]
    Dp = momentum.overlap_D(dims, r, M0)
    return ifft4_fermion(spin_mult(Dp, fft4_fermion(psi)))


def site_terms(params, phi):
    """(y_plus, y_minus): coefficients of P_+ and P_- in Y(x) (Eq. fmat)."""
    c = params.yukawa
    y_plus = params.m + c * params.g * phi
    y_minus = np.conj(params.m) + c * np.conj(params.g) * np.conj(phi)
    return y_plus, y_minus


def apply_Y(params, phi, psi, dagger=False):
    y_plus, y_minus = site_terms(params, phi)
    if dagger:
        y_plus, y_minus = np.conj(y_plus), np.conj(y_minus)
    out = np.empty_like(psi)
    out[..., 0:2] = y_minus[..., None] * psi[..., 0:2]
    out[..., 2:4] = y_plus[..., None] * psi[..., 2:4]
    return out


def apply_M(params, phi, psi):
    """M psi (Eq. fmat)."""
    return apply_dslash(psi, params.r, params.M0, +1.0) + apply_Y(params, phi, psi)


def apply_Mdag(params, phi, psi):
    """M^dagger psi = -Dslash psi + Y^dagger psi."""
    return apply_dslash(psi, params.r, params.M0, -1.0) + apply_Y(params, phi, psi, True)


def apply_MdagM(params, phi, psi, shift=0.0):
    """(M^dagger M + shift) psi (Eq. theprob / Eq. yuier)."""
    out = apply_Mdag(params, phi, apply_M(params, phi, psi))
    if shift:
        out = out + shift * psi
    return out


# ---------------------------------------------------------------- free preconditioner


def M0_symbol(params):
    """Free fermion matrix M0(p) = Dslash(p) + m P_+ + m^* P_- (Sec. 3.1)."""
    dims = params.dims
    return momentum.dslash_symbol(dims, params.r, params.M0) + (
        params.m * P_PLUS + np.conj(params.m) * P_MINUS
    )


def M0inv_symbol(params):
    """M0^-1(p) = M0^dagger(p) / (D_mu^dagger D_mu + |m|^2) (Sec. 7.3)."""
    M0p = M0_symbol(params)
    M0dag = np.conj(np.swapaxes(M0p, -1, -2))
    den = momentum.free_norm(params.dims, params.m, params.r, params.M0)
    return M0dag / den[..., None, None]


def apply_M0inv(params, psi, dagger=False):
    """M0^-1 psi, or (M0^-1)^dagger psi; both diagonal in momentum space."""
    S = M0inv_symbol(params)
    if dagger:
        S = np.conj(np.swapaxes(S, -1, -2))
    return ifft4_fermion(spin_mult(S, fft4_fermion(psi)))


def apply_Mtilde(params, phi, psi):
    """M~ = M M0^-1 (Eq. theprob)."""
    return apply_M(params, phi, apply_M0inv(params, psi))


def apply_Mtilde_dag(params, phi, psi):
    """M~^dagger = (M0^-1)^dagger M^dagger."""
    return apply_M0inv(params, apply_Mdag(params, phi, psi), dagger=True)


# ---------------------------------------------------------------- scalar operators


def apply_scalar_symbol(sym, f):
    """Apply a real momentum-space symbol to a periodic scalar field."""
    return np.fft.ifftn(sym * np.fft.fftn(f))


def apply_D2_scalar(params, f):
    D2, _ = momentum.scalar_D2_K(params.dims, params.r, params.M0)
    return apply_scalar_symbol(D2, f)


def apply_K_scalar(params, f):
    _, K = momentum.scalar_D2_K(params.dims, params.r, params.M0)
    return apply_scalar_symbol(K, f)
