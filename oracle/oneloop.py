"""One-loop lattice sums of Sec. 5 (finite system size, a = 1).

TEST INFRASTRUCTURE ONLY (see the package docstring).

With P_mu(k) = sin k_mu, M(k) = 1 - 2 sum_mu sin^2(k_mu / 2), s(k) = sqrt(P^2 + M^2)
and r(k) = 2 (1 - M/s) + (|m|^2 / 2)(1 + M/s) (the scalar propagator
denominator), on an N^4 lattice (k_mu = 2 pi n_mu / N, periodic) with
(1/N^4) sum_k in place of int d^4k / (2 pi)^4:

    scalar     Sigma_phi(p) / |g|^2 = (1/N^4) sum_k N(k, p) / (r(k) r(k + p)),
               N = P(p + k).P(k) / (s(k) s(k + p)) - P^2(k) / s^2(k)
    fermion    Sigma_chi(p) / |g|^2 = (1/N^4) sum_k P-slash(p + k) / (r(k) r(p + k) s(p + k))
    auxiliary  Sigma_F(0) / |g|^2   = (1/N^4) sum_k 1 / r(k)^2

and the counterterms of Tables sse, fse, ase at p = (0, 0, 0, 2 pi / N):

    Z_phi - 1 = Sigma_phi(p) / P^2(p),   Z_chi - 1 = -[Sigma_chi(p)]_3 / P_3(p),   Z_F - 1 = Sigma_F(0).

Readings: the lattice momentum P^2(p) = sin^2(2 pi / N) divides the scalar
self-energy; the fermion sign is the one that makes Z_chi - 1 negative as in
Table fse (the printed prefactor -i multiplies P-slash, i.e. the slope of
-Sigma along gamma_3); all directions periodic.  m enters only as ma = mL / N.
"""

import numpy as np


def _parts(k):
    P2 = sum(np.sin(x) ** 2 for x in k)
    M = 1.0 - 2.0 * sum(np.sin(0.5 * x) ** 2 for x in k)
    s = np.sqrt(P2 + M * M)
    return P2, M, s


def _r(M, s, ma):
    return 2.0 * (1.0 - M / s) + 0.5 * ma * ma * (1.0 + M / s)


def _grid(N, slab):
    """The momenta k_mu = 2 pi n / N of the slab of n_0 values, as 4 arrays."""
    n = 2.0 * np.pi * np.arange(N) / N
    return np.meshgrid(n[slab], n, n, n, indexing="ij")


def sums(N, ma, slab_size=8):
    """(Z_phi - 1, Z_chi - 1, Z_F - 1) / |g|^2 on N^4 momenta (plain loops over slabs of k_0)."""
    p3 = 2.0 * np.pi / N
    acc = np.zeros(3)
    for a in range(0, N, slab_size):
        k = _grid(N, slice(a, min(N, a + slab_size)))
        kp = [k[0], k[1], k[2], k[3] + p3]
        P2, M, s = _parts(k)
        _, Mp, sp = _parts(kp)
        r, rp = _r(M, s, ma), _r(Mp, sp, ma)
        dot = sum(np.sin(k[mu]) * np.sin(kp[mu]) for mu in range(4))
        num = dot / (s * sp) - P2 / (s * s)
        acc[0] += np.sum(num / (r * rp))
        acc[1] += np.sum(np.sin(kp[3]) / (r * rp * sp))
        acc[2] += np.sum(1.0 / (r * r))
    acc /= float(N) ** 4
    return acc[0] / np.sin(p3) ** 2, -acc[1] / np.sin(p3), acc[2]


def self_energies_at(N, ma, p):
    """Sigma_phi(p) and the four components of Sigma_chi(p) (over |g|^2) at a general p."""
    n = 2.0 * np.pi * np.arange(N) / N
    k = np.meshgrid(n, n, n, n, indexing="ij")
    kp = [k[mu] + p[mu] for mu in range(4)]
    P2, M, s = _parts(k)
    _, Mp, sp = _parts(kp)
    r, rp = _r(M, s, ma), _r(Mp, sp, ma)
    dot = sum(np.sin(k[mu]) * np.sin(kp[mu]) for mu in range(4))
    num = dot / (s * sp) - P2 / (s * s)
    sig_phi = np.mean(num / (r * rp))
    sig_chi = [np.mean(np.sin(kp[mu]) / (r * rp * sp)) for mu in range(4)]
    return sig_phi, sig_chi
