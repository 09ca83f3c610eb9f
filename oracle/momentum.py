"""Closed-form overlap operator in momentum space (Secs. 2.2, 3.1, 7.3).

TEST INFRASTRUCTURE ONLY (see the package docstring).

With a = 1, Wilson parameter r and constant M0, the kernel A = M0 - D_W has the
Fourier symbol A(p) = b(p) - i gamma_mu sin p_mu with

    b(p)     = M0 - r * sum_mu 2 sin^2(p_mu / 2)       (Eq. d1mom denominator)
    omega(p) = sqrt(b^2 + sum_mu sin^2 p_mu) = |A(p)|  ((A^dagger A)^1/2)

so that (Sec. 2.2, Eq. d1mom; sign of i fixed by the Fourier convention below)

    D1(p) = i gamma_mu sin p_mu / omega,   D2(p) = 1 - b / omega,
    1 - D2/2 = (omega + b) / (2 omega),
    Dslash(p) = (1 - D2/2)^-1 D1 = i h(p) gamma_mu sin p_mu,  h = 2 / (omega + b).

Fourier convention: f_hat(p) = sum_x exp(-i p.x) f(x) (numpy's forward FFT),
so a forward difference f(x + mu) - f(x) becomes (exp(i p_mu) - 1) f_hat.

Fermion momenta (antiperiodic time, Sec. 3.1): p_t = pi (2 n + 1) / T and
p_k = 2 pi n / L_k; scalar momenta are all periodic, p_mu = 2 pi n / L_mu.
"""

import numpy as np

from .conventions import GAMMA, MU_AXIS


def axis_momenta(n, antiperiodic):
    """Momenta along one axis, in numpy FFT index order (index n -> p)."""
    k = np.arange(n, dtype=np.float64)
    if antiperiodic:
        return np.pi * (2.0 * k + 1.0) / n
    return 2.0 * np.pi * k / n


def momentum_grid(dims, fermion=True):
    """Return a list p[mu] of arrays of shape dims (T, Z, Y, X)."""
    T, Z, Y, X = dims
    per_axis = [
        axis_momenta(T, fermion),
        axis_momenta(Z, False),
        axis_momenta(Y, False),
        axis_momenta(X, False),
    ]
    grids = np.meshgrid(*per_axis, indexing="ij")
    return [grids[MU_AXIS[mu]] for mu in range(4)]


def symbol_parts(dims, r=1.0, M0=1.0, fermion=True):
    """b(p), omega(p) and the list sin(p_mu) on the full momentum grid."""
    p = momentum_grid(dims, fermion)
    s = [np.sin(pm) for pm in p]
    b = M0 - r * sum(2.0 * np.sin(pm / 2.0) ** 2 for pm in p)
    omega = np.sqrt(b * b + sum(sm * sm for sm in s))
    return b, omega, s


def h_of_p(dims, r=1.0, M0=1.0):
    """h(p) = 2 / (omega + b) on the fermion (antiperiodic-time) grid."""
    b, omega, _ = symbol_parts(dims, r, M0, fermion=True)
    return 2.0 / (omega + b)


def D1_D2(dims, r=1.0, M0=1.0, fermion=True):
    """Return (D1(p), D2(p)) as arrays of shape dims + (4, 4) and dims."""
    b, omega, s = symbol_parts(dims, r, M0, fermion)
    slash = sum(s[mu][..., None, None] * GAMMA[mu] for mu in range(4))
    D1 = 1j * slash / omega[..., None, None]
    D2 = 1.0 - b / omega
    return D1, D2


def overlap_D(dims, r=1.0, M0=1.0, fermion=True):
    """D(p) = 1 - A(p) / omega(p) as dims + (4, 4) (Sec. 2.2)."""
    b, omega, s = symbol_parts(dims, r, M0, fermion)
    slash = sum(s[mu][..., None, None] * GAMMA[mu] for mu in range(4))
    A = b[..., None, None] * np.eye(4) - 1j * slash
    return np.eye(4) - A / omega[..., None, None]


def dslash_symbol(dims, r=1.0, M0=1.0):
    """Dslash(p) = i h(p) gamma_mu sin p_mu (Eq. fmat) as dims + (4, 4)."""
    b, omega, s = symbol_parts(dims, r, M0, fermion=True)
    h = 2.0 / (omega + b)
    slash = sum(s[mu][..., None, None] * GAMMA[mu] for mu in range(4))
    return 1j * h[..., None, None] * slash


def free_norm(dims, m, r=1.0, M0=1.0):
    """D_mu^dagger D_mu + |m|^2 = h^2 sum sin^2 p_mu + |m|^2 (Sec. 7.3)."""
    b, omega, s = symbol_parts(dims, r, M0, fermion=True)
    h = 2.0 / (omega + b)
    return h * h * sum(sm * sm for sm in s) + abs(m) ** 2


def scalar_D2_K(dims, r=1.0, M0=1.0):
    """Scalar (periodic) symbols D2(p) and K(p) = 1 - D2(p)/2 (Eq. acws).

    On the periodic grid sum sin^2 vanishes at the 16 corners of the Brillouin
    zone; there omega = |b| and D2 = 1 - sign(b).
    """
    b, omega, _ = symbol_parts(dims, r, M0, fermion=False)
    D2 = 1.0 - b / omega
    return D2, 1.0 - 0.5 * D2
