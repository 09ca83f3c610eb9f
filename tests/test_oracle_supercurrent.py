"""Pins of the supercurrent correlators (Eqs. latsuc, sitre) in the oracle.

1. At g = 0 the per-configuration correlator is bilinear in the free scalar, so
   its exact mean over the Gaussian measure (taken by polarisation over the
   columns of G^1/2) must equal the tree-level expression derived below Eq. sitre,
   sqrt2 gamma_nu gamma_mu P_- S D1_nu G + sqrt2 m^* gamma_mu P_+ S G (and the
   conjugate channel), built here from dense momentum-space propagators.
2. A constant scalar has D1 phi = 0 and a free fermion of mass m + 2 g phi, so
   the correlator has a closed form at g != 0 (the W' = m phi + g phi^2 terms).
3. Translating the scalar and the point source together in time (across the
   antiperiodic boundary) or in space leaves the correlator unchanged.
4. A 90 degree rotation in the x-y plane of the scalar and the source turns the
   correlator as a vector in mu and by the spin rotation S on both spin indices
   (the y sum at zero momentum hides the spatial D1 components from pin 1; this
   one sees them).
"""

import numpy as np
import pytest

import oracle
from oracle import supercurrent
from oracle.conventions import CCONJ, GAMMA, P_MINUS, P_PLUS
from paper_1005_3276_gb300 import synth

SQRT2 = np.sqrt(2.0)


def momenta(n, antiperiodic):
    k = np.arange(n)
    return (2 * k + 1) * np.pi / n if antiperiodic else 2 * np.pi * k / n


def grid(dims, fermion):
    """Momentum components p_mu on the (T, Z, Y, X) grid, mu = (t, x, y, z)."""
    T, Z, Y, X = dims
    pt, pz, py, px = np.meshgrid(momenta(T, fermion), momenta(Z, False), momenta(Y, False), momenta(X, False),
                                 indexing="ij")
    return [pt, px, py, pz]


def symbol(p):
    b = 1.0 - 2.0 * sum(np.sin(0.5 * q) ** 2 for q in p)
    om = np.sqrt(b * b + sum(np.sin(q) ** 2 for q in p))
    return b, om


def sites(dims):
    return [tuple(s) for s in np.ndindex(*dims)]


def free_fermion_propagator(dims, meff):
    """S(x, z) = -M0^-1(x, z) for M0(p) = Dslash(p) + meff P_+ + meff^* P_-, dense (V, V, 4, 4)."""
    p = grid(dims, True)
    b, om = symbol(p)
    h = 2.0 / (om + b)
    Mp = sum(1j * (h * np.sin(p[mu]))[..., None, None] * GAMMA[mu] for mu in range(4))
    Mp = Mp + meff * P_PLUS + np.conj(meff) * P_MINUS
    Minv = np.linalg.inv(Mp.reshape(-1, 4, 4))
    P = np.stack([q.ravel() for q in p], axis=1)  # (V, 4) with mu order (t, x, y, z)
    X = np.array([[s[0], s[3], s[2], s[1]] for s in sites(dims)], float)  # coordinates in mu order
    V = len(X)
    S = np.zeros((V, V, 4, 4), np.complex128)
    for z in range(V):
        ph = np.exp(1j * (X - X[z]) @ P.T)  # (x, p)
        S[:, z] = -np.einsum("xp,pab->xab", ph, Minv) / V
    return S


def dense_scalar(dims, m):
    """G[y, z] = <phi(y) phi^*(z)> of the free bosonic action and D_nu[x, z] = d_nu(x - z)."""
    p = grid(dims, False)
    b, om = symbol(p)
    Ghat = 1.0 / (2.0 * (1.0 - b / om) + abs(m) ** 2 * 0.5 * (1.0 + b / om))
    P = np.stack([q.ravel() for q in p], axis=1)
    X = np.array([[s[0], s[3], s[2], s[1]] for s in sites(dims)], float)
    V = len(X)
    E = np.exp(1j * X @ P.T)  # (x, p)
    G = (E * Ghat.ravel()) @ E.conj().T / V
    D = [(E * (1j * np.sin(P[:, nu]) / om.ravel())) @ E.conj().T / V for nu in range(4)]
    return G, D


def test_tree_level_mean_at_g0():
    dims = (4, 3, 3, 3)  # extent 3: sin p != 0 on every spatial axis
    m = 0.4 + 0.2j
    P = oracle.Params(dims=dims, m=m, g=0.0)
    T, V3 = dims[0], int(np.prod(dims[1:]))
    V = T * V3
    z0 = (1, 0, 1, 0)
    w = np.zeros(dims, np.complex128)
    w[z0] = 1.0
    G, D = dense_scalar(dims, m)
    ev, U = np.linalg.eigh(G)
    assert ev.min() > 0
    U = U * np.sqrt(ev)  # U U^dag = G
    mean = np.zeros((2, 4, T, T, 4, 4), np.complex128)
    for j in range(V):
        u = U[:, j].reshape(dims)
        mean += 0.5 * (supercurrent.correlators(P, u, w, 1e-14) + supercurrent.correlators(P, 1j * u, w, 1e-14))
    S = free_fermion_propagator(dims, m)
    idx = {s: i for i, s in enumerate(sites(dims))}
    zi = idx[z0]
    H0 = [Dn @ G.T for Dn in D]  # <phi(y) (D1 phi^*)_nu(x)> as [x, y]
    H1 = [Dn @ G for Dn in D]  # <phi^*(y) (D1 phi)_nu(x)> as [x, y]
    tree = np.zeros_like(mean)
    for dx in range(T):
        tx = (z0[0] + dx) % T
        sgn = -1.0 if z0[0] + dx >= T else 1.0
        for dy in range(T):
            ty = (z0[0] + dy) % T
            for xs in np.ndindex(*dims[1:]):
                xi = idx[(tx,) + xs]
                Sx = S[xi, zi]
                for ys in np.ndindex(*dims[1:]):
                    yi = idx[(ty,) + ys]
                    for mu in range(4):
                        t0 = sum(H0[nu][xi, yi] * GAMMA[nu] for nu in range(4)) @ GAMMA[mu] @ P_MINUS
                        t0 = t0 + np.conj(m) * G[yi, xi] * GAMMA[mu] @ P_PLUS
                        t1 = sum(H1[nu][xi, yi] * GAMMA[nu] for nu in range(4)) @ GAMMA[mu] @ P_PLUS
                        t1 = t1 + m * G[xi, yi] * GAMMA[mu] @ P_MINUS
                        tree[0, mu, dx, dy] += sgn * SQRT2 * t0 @ Sx
                        tree[1, mu, dx, dy] += sgn * SQRT2 * t1 @ Sx
    scale = np.abs(tree).max()
    assert scale > 1e-3
    np.testing.assert_allclose(mean, tree, rtol=0, atol=1e-11 * scale)


def test_constant_scalar_closed_form():
    dims = (6, 2, 4, 2)
    m, g, c = 0.3 - 0.1j, 0.45 + 0.2j, 0.5 + 0.3j
    P = oracle.Params(dims=dims, m=m, g=g)
    T, V3 = dims[0], int(np.prod(dims[1:]))
    phi = np.full(dims, c, np.complex128)
    z0 = (4, 1, 2, 0)
    w = np.zeros(dims, np.complex128)
    w[z0] = 1.0
    R = supercurrent.correlators(P, phi, w, 1e-14)
    S = free_fermion_propagator(dims, m + 2.0 * g * c)
    idx = {s: i for i, s in enumerate(sites(dims))}
    Wp = m * c + g * c * c
    ref = np.zeros_like(R)
    for dx in range(T):
        tx = (z0[0] + dx) % T
        sgn = -1.0 if z0[0] + dx >= T else 1.0
        Ssum = sum(S[idx[(tx,) + xs], idx[z0]] for xs in np.ndindex(*dims[1:]))
        for mu in range(4):
            Gam = SQRT2 * (Wp * GAMMA[mu] @ P_MINUS + np.conj(Wp) * GAMMA[mu] @ P_PLUS)
            for s, Phi in enumerate((V3 * c, V3 * np.conj(c))):
                ref[s, mu, dx, :] = sgn * Phi * (Gam @ Ssum)
    np.testing.assert_allclose(R, ref, rtol=0, atol=1e-11 * np.abs(ref).max())


@pytest.mark.parametrize("shift,axis", [(2, 0), (3, 0), (1, 2)])
def test_translation_invariance(shift, axis):
    dims = (4, 2, 4, 2)
    P = oracle.Params(dims=dims, m=0.4, g=0.5 + 0.2j)
    phi = synth.scalar_field(dims, 0.4, 21)
    z0 = (1, 1, 2, 0)
    w = np.zeros(dims, np.complex128)
    w[z0] = 1.0
    R = supercurrent.correlators(P, phi, w, 1e-14)
    R2 = supercurrent.correlators(P, np.roll(phi, shift, axis), np.roll(w, shift, axis), 1e-14)
    np.testing.assert_allclose(R2, R, rtol=0, atol=1e-10 * np.abs(R).max())


def test_source_weight_is_sesquilinear_in_the_time_weight():
    """Scaling the source by a complex c scales R by |c|^2 (xi^* times the solution)."""
    dims = (4, 2, 2, 2)
    P = oracle.Params(dims=dims, m=0.3, g=0.4)
    phi = synth.scalar_field(dims, 0.5, 3)
    w = synth.scalar_field(dims, 1.0, 4)
    c = 0.7 - 1.1j
    R = supercurrent.correlators(P, phi, w, 1e-14)
    R2 = supercurrent.correlators(P, phi, c * w, 1e-14)
    np.testing.assert_allclose(R2, abs(c) ** 2 * R, rtol=0, atol=1e-11 * np.abs(R2).max())


def test_rotation_covariance():
    """x' = L x with L e_x = e_y, L e_y = -e_x; psi'(x') = S psi(x) with
    S^-1 gamma_mu S = L_mu_nu gamma_nu, so R'_mu = L_mu_nu S R_nu C^-1 S^T C."""
    dims = (4, 2, 3, 3)  # Y = X
    L = np.eye(4)
    L[1, 1] = L[2, 2] = 0.0
    L[1, 2], L[2, 1] = -1.0, 1.0
    found = []
    for sgn in (1.0, -1.0):
        S = (np.eye(4) + sgn * GAMMA[1] @ GAMMA[2]) / np.sqrt(2.0)
        Si = np.linalg.inv(S)
        if all(np.allclose(Si @ GAMMA[mu] @ S, sum(L[mu, nu] * GAMMA[nu] for nu in range(4))) for mu in range(4)):
            found.append(S)
    assert len(found) == 1
    S = found[0]
    right = np.linalg.inv(CCONJ) @ S.T @ CCONJ
    P = oracle.Params(dims=dims, m=0.35 + 0.1j, g=0.5 - 0.3j)
    phi = synth.scalar_field(dims, 0.5, 31)
    w = synth.scalar_field(dims, 1.0, 32)

    def rotate(f):
        # f'(t, z, y', x') = f(x = y', y = -x'): the array axes are (T, Z, Y, X)
        n = dims[3]
        out = np.empty_like(f)
        for j in range(n):
            for i in range(n):
                out[:, :, j, i] = f[:, :, (-i) % n, j]
        return out

    R = supercurrent.correlators(P, phi, w, 1e-14)
    R2 = supercurrent.correlators(P, rotate(phi), rotate(w), 1e-14)
    ref = np.einsum("mn,ab,sndebc,cf->smdeaf", L, S, R, right)
    np.testing.assert_allclose(R2, ref, rtol=0, atol=1e-10 * np.abs(R).max())
