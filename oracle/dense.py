"""Dense position-space operators for small lattices (Sec. 2.2, Eqs. kisu, lata, fmat).

TEST INFRASTRUCTURE ONLY (see the package docstring).

These builders follow the position-space definitions of Sec. 2.2 and never use
the momentum-space closed forms, so they pin the FFT path independently:

    forward/backward differences  d_mu f(x) = f(x+mu) - f(x),  d*_mu f(x) = f(x) - f(x-mu)
    D_W  = 1/2 gamma_mu (d*_mu + d_mu) - (r/2) d*_mu d_mu
    A    = M0 - D_W
    D1   = 1/2 gamma_mu (d*_mu + d_mu) (A^dagger A)^-1/2
    D2   = 1 - (M0 + (r/2) d*_mu d_mu) (A^dagger A)^-1/2
    D    = D1 + D2 = 1 - A (A^dagger A)^-1/2
    Dslash = (1 - D2/2)^-1 D1,  M = Dslash + Y                       (Eq. fmat)

The Wilson term is written with the sign that makes the scalar part of A equal
to M0 - 2 r sum sin^2(p/2), as the momentum-space formulas of Secs. 3.1 and 4.1
require (the position-space formula of Sec. 2.2 prints the opposite sign).
(A^dagger A)^-1/2 is evaluated by Hermitian eigendecomposition.

Fermion fields are antiperiodic in time: a hop across the time boundary picks
up a factor -1.  Index order of a dense vector is the C order of a
(T, Z, Y, X, 4) array: ((((t Z + z) Y + y) X + x) 4 + spin).
"""

import numpy as np

from .conventions import CCONJ, GAMMA, GAMMA5, MU_AXIS


def shift_matrix(dims, mu, antiperiodic_time):
    """S with (S f)(x) = f(x + mu_hat), including the time-boundary sign."""
    V = int(np.prod(dims))
    idx = np.arange(V).reshape(dims)
    axis = MU_AXIS[mu]
    nbr = np.roll(idx, -1, axis=axis)  # nbr[x] = index of x + mu
    sign = np.ones(dims)
    if antiperiodic_time and axis == 0:
        sign[dims[0] - 1] = -1.0
    S = np.zeros((V, V), dtype=np.complex128)
    S[idx.ravel(), nbr.ravel()] = sign.ravel()
    return S


def _spin_kron(site_op, spin_op):
    return np.kron(site_op, spin_op)


def build_kernel_parts(dims, r=1.0, M0=1.0, fermion=True):
    """Return (A, Dsym, Wscalar): A = M0 - D_W, the symmetric difference part
    1/2 gamma_mu (d + d*) and the scalar part M0 + (r/2) d* d, all 4V x 4V."""
    V = int(np.prod(dims))
    I4 = np.eye(4, dtype=np.complex128)
    IV = np.eye(V, dtype=np.complex128)
    Dsym = np.zeros((4 * V, 4 * V), dtype=np.complex128)
    lap = np.zeros((V, V), dtype=np.complex128)
    for mu in range(4):
        Sp = shift_matrix(dims, mu, fermion)
        Sm = Sp.conj().T  # (S^dagger f)(x) = f(x - mu) with the same sign rule
        Dsym += 0.5 * _spin_kron(Sp - Sm, GAMMA[mu])
        lap += Sp + Sm - 2.0 * IV  # d*_mu d_mu
    Wscalar = _spin_kron(M0 * IV + 0.5 * r * lap, I4)
    A = Wscalar - Dsym
    return A, Dsym, Wscalar


def inv_sqrt_hermitian(H):
    w, U = np.linalg.eigh(H)
    if w.min() <= 0:
        raise np.linalg.LinAlgError("A^dagger A is not positive definite")
    return (U * (1.0 / np.sqrt(w))) @ U.conj().T


def build_overlap(dims, r=1.0, M0=1.0, fermion=True):
    """Dense (D1, D2, D) of Sec. 2.2."""
    A, Dsym, Wscalar = build_kernel_parts(dims, r, M0, fermion)
    B = inv_sqrt_hermitian(A.conj().T @ A)
    n = A.shape[0]
    D1 = Dsym @ B
    D2 = np.eye(n) - Wscalar @ B
    return D1, D2, D1 + D2


def build_dslash(dims, r=1.0, M0=1.0):
    """Dense Dslash = (1 - D2/2)^-1 D1 (Eq. fmat), antiperiodic time."""
    D1, D2, _ = build_overlap(dims, r, M0, fermion=True)
    n = D1.shape[0]
    return np.linalg.solve(np.eye(n) - 0.5 * D2, D1)


def build_Y(params, phi):
    """Dense site-local term Y = (m + c g phi) P_+ + (m^* + c g^* phi^*) P_-."""
    c = params.yukawa
    y_plus = (params.m + c * params.g * phi).ravel()
    y_minus = (np.conj(params.m) + c * np.conj(params.g) * np.conj(phi)).ravel()
    diag = np.stack([y_minus, y_minus, y_plus, y_plus], axis=1).ravel()
    return np.diag(diag)


def build_M(params, phi, dslash=None):
    """Dense fermion matrix M = Dslash + Y (Eq. fmat)."""
    if dslash is None:
        dslash = build_dslash(params.dims, params.r, params.M0)
    return dslash + build_Y(params, phi)


def build_aux_block(params, phi, D=None):
    """Dense fermion operator of Eq. kisu on (chi, X) before X is integrated out.

    With chi~ = chi + X, the fermion terms of Eq. kisu are
    -(1/2) (chi, X)^T C K (chi, X) with K = [[D + Y, Y], [Y, Y - 2]] (a = 1).
    """
    if D is None:
        _, _, D = build_overlap(params.dims, params.r, params.M0, fermion=True)
    Y = build_Y(params, phi)
    n = D.shape[0]
    return np.block([[D + Y, Y], [Y, Y - 2.0 * np.eye(n)]])


def gamma5_dense(V):
    return np.kron(np.eye(V), GAMMA5)


def cconj_dense(V):
    return np.kron(np.eye(V), CCONJ)


def build_scalar_D2(dims, r=1.0, M0=1.0):
    """Scalar D2 (periodic in all directions) as a V x V matrix.

    D2 built on spinors is spin-diagonal because A^dagger A is; the (0, 0)
    spin block is returned (the test checks the other blocks agree).
    """
    _, D2, _ = build_overlap(dims, r, M0, fermion=False)
    V = int(np.prod(dims))
    return D2.reshape(V, 4, V, 4)
