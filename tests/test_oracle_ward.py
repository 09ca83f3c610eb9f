"""Pins of the oracle's Ward-identity observables (Eq. exid, Eq. nzav).

W_R is computed two independent ways at 4^4: the oracle's FFT route (momentum
space D1, CG solves) and a dense position-space route (the overlap of Sec. 2.2
built from shift matrices and a Hermitian inverse square root, dense LU for
M^-1, the scalar D1 kernels read off the dense overlap on the periodic grid as
Tr(gamma_mu D1) / 4).  A dropped term, a wrong axis or sign of D1, a misplaced
C or chirality projector in either route makes them disagree.
"""

import numpy as np
import pytest

import oracle
from oracle import dense, ward
from oracle.conventions import CCONJ, GAMMA, P_MINUS, P_PLUS
from paper_1005_3276_gb300 import synth


def dense_ward_right(P, phi):
    dims = P.dims
    V = int(np.prod(dims))
    M = dense.build_M(P, phi)
    D1f, _, _ = dense.build_overlap(dims, P.r, P.M0, fermion=True)
    D1s, _, _ = dense.build_overlap(dims, P.r, P.M0, fermion=False)
    blocks = D1s.reshape(V, 4, V, 4)
    K = [0.25 * np.einsum("ba,xayb->xy", GAMMA[mu], blocks) for mu in range(4)]
    f = [K[mu] @ phi.ravel() for mu in range(4)]
    fs = [K[mu] @ np.conj(phi).ravel() for mu in range(4)]
    Cinv = np.linalg.inv(CCONJ)
    ph = phi.ravel()[:, None]
    W = np.zeros((4, 4), complex)
    for b in range(4):
        src = np.tile(Cinv[:, b], V)
        psi = np.linalg.solve(M, src).reshape(V, 4)
        pp, pm = psi @ P_PLUS.T, psi @ P_MINUS.T
        d1p = (D1f @ pp.ravel()).reshape(V, 4)
        d1m = (D1f @ pm.ravel()).reshape(V, 4)
        gp = sum(f[mu][:, None] * (pp @ GAMMA[mu].T) for mu in range(4))
        gm = sum(fs[mu][:, None] * (pm @ GAMMA[mu].T) for mu in range(4))
        kv = P.g * (2 * ph * gp + ph ** 2 * d1p) + np.conj(P.g) * (2 * np.conj(ph) * gm + np.conj(ph) ** 2 * d1m)
        W[:, b] = kv.sum(axis=0)
    return W


def test_ward_right_fft_equals_dense_4():
    dims = (4, 4, 4, 4)
    P = oracle.Params(dims=dims, m=0.4 + 0.1j, g=0.3 - 0.2j)
    phi = synth.scalar_field(dims, 0.5, 3)
    W = ward.ward_right(P, phi, tol=1e-14)
    Wd = dense_ward_right(P, phi)
    assert np.abs(W - Wd).max() <= 1e-9 * np.abs(Wd).max()
    assert np.abs(Wd).max() > 1e-3  # not trivially zero


def test_ward_right_vanishes_at_zero_coupling():
    dims = (4, 4, 4, 4)
    P = oracle.Params(dims=dims, m=0.4, g=0.0)
    phi = synth.scalar_field(dims, 0.5, 4)
    assert np.abs(ward.ward_right(P, phi)).max() == 0.0


def test_scalar_d1_of_a_plane_wave():
    """D1 on the periodic plane wave exp(i q.x) multiplies it by i sin q_mu / omega(q)."""
    dims = (4, 6, 4, 8)
    T, Z, Y, X = dims
    t, z, y, x = np.meshgrid(*[np.arange(n) for n in dims], indexing="ij")
    q = (2 * np.pi / T, 2 * 2 * np.pi / Z, 0.0, 3 * 2 * np.pi / X)  # (t, z, y, x) momenta
    f = np.exp(1j * (q[0] * t + q[1] * z + q[2] * y + q[3] * x))
    comp = ward.scalar_d1_components(dims, f)
    qmu = (q[0], q[3], q[2], q[1])  # mu = t, x, y, z
    b = 1.0 - sum(2 * np.sin(v / 2) ** 2 for v in qmu)
    omega = np.sqrt(b * b + sum(np.sin(v) ** 2 for v in qmu))
    for mu in range(4):
        np.testing.assert_allclose(comp[mu], 1j * np.sin(qmu[mu]) / omega * f, atol=1e-13)


def test_ward_left_is_the_auxiliary_sum():
    dims = (4, 4, 4, 4)
    P = oracle.Params(dims=dims, m=0.4 + 0.1j, g=0.3 - 0.2j)
    phi = synth.scalar_field(dims, 0.5, 5)
    from oracle import force
    V = int(np.prod(dims))
    F = V * force.auxiliary_vev(P, phi)
    WL = ward.ward_left(P, phi)
    np.testing.assert_allclose(WL[:, 2:], F * CCONJ[:, 2:], rtol=1e-13)
    np.testing.assert_allclose(WL[:, :2], np.conj(F) * CCONJ[:, :2], rtol=1e-13)
