"""Pins of the oracle's Ward-identity observables (Eq. exid, Eq. nzav).

W_R is computed two independent ways at 4^4: the oracle's FFT route (momentum
space D1, CG solves) and a dense position-space route (the overlap of Sec. 2.2
built from shift matrices and a Hermitian inverse square root, dense LU for
M^-1, the scalar D1 kernels read off the dense overlap on the periodic grid as
Tr(gamma_mu D1) / 4).  A dropped term, a wrong axis or sign of D1, a misplaced
C or chirality projector in either route makes them disagree.

The identity itself, <W_R> = <W_L> over the exact measure Pf(CM) exp(-S_B), is
checked on a lattice where the derivation of Eq. nzav is exact: T = 3 with
periodic fermions (no antiperiodic/periodic mismatch in the lattice integration
by parts, and 1 - D2/2 has no zero), spatial extent 1, by importance-sampled
integration over the three complex scalars with the dense route's W_R.  It
fixes the sign of the identity and the chirality structure of W_L.
"""

import numpy as np
import pytest

import oracle
from oracle import dense, ward
from oracle.conventions import CCONJ, GAMMA, P_MINUS, P_PLUS
from paper_1005_3276_gb300 import synth


def dense_ward_right(P, phi, antiperiodic=True):
    dims = P.dims
    V = int(np.prod(dims))
    D1f, D2f, _ = dense.build_overlap(dims, P.r, P.M0, fermion=antiperiodic)
    M = np.linalg.solve(np.eye(4 * V) - 0.5 * D2f, D1f) + dense.build_Y(P, phi)
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


def pfaffian(A):
    """Pf of a batch of antisymmetric matrices (N, n, n) by Parlett-Reid elimination."""
    A = A.copy()
    N, n, _ = A.shape
    pf = np.ones(N, complex)
    rows = np.arange(N)
    for k in range(0, n - 1, 2):
        kp = k + 1 + np.argmax(np.abs(A[:, k, k + 1:]), axis=1)
        swap = kp != k + 1
        if swap.any():  # a simultaneous row and column swap flips the sign
            r1, r2 = A[rows, k + 1, :].copy(), A[rows, kp, :].copy()
            A[rows, k + 1, :], A[rows, kp, :] = r2, r1
            c1, c2 = A[rows, :, k + 1].copy(), A[rows, :, kp].copy()
            A[rows, :, k + 1], A[rows, :, kp] = c2, c1
            pf[swap] *= -1
        a = A[:, k, k + 1]
        pf *= a
        if k + 2 < n:  # Schur complement of the 2 x 2 pivot block
            tau, v = A[:, k, k + 2:] / a[:, None], A[:, k + 1, k + 2:]
            A[:, k + 2:, k + 2:] += v[:, :, None] * tau[:, None, :] - tau[:, :, None] * v[:, None, :]
    return pf


def test_pfaffian_squares_to_the_determinant():
    rng = np.random.default_rng(1)
    A = rng.normal(size=(5, 12, 12)) + 1j * rng.normal(size=(5, 12, 12))
    A = A - np.transpose(A, (0, 2, 1))
    assert np.abs(pfaffian(A) ** 2 / np.linalg.det(A) - 1).max() < 1e-12
    B = A[:, :4, :4]
    ref = B[:, 0, 1] * B[:, 2, 3] - B[:, 0, 2] * B[:, 1, 3] + B[:, 0, 3] * B[:, 1, 2]
    assert np.abs(pfaffian(B) - ref).max() < 1e-12


def batched_ward(P, phis):
    """(Pf(CM), S_B, W_R[0,1], W_R[2,3], sum_x F~) for configurations phis (N, V) of a
    T x 1 x 1 x 1 lattice with periodic fermions (the dense route, batched)."""
    dims = P.dims
    V = int(np.prod(dims))
    m, g = P.m, P.g
    D1f, D2f, _ = dense.build_overlap(dims, P.r, P.M0, fermion=False)
    Dsl = np.linalg.solve(np.eye(4 * V) - 0.5 * D2f, D1f)
    D1s, D2s, _ = dense.build_overlap(dims, P.r, P.M0, fermion=False)
    D2s = D2s.reshape(V, 4, V, 4)[:, 0, :, 0]
    Kt = 0.25 * np.einsum("ba,xayb->xy", GAMMA[0], D1s.reshape(V, 4, V, 4))  # time component of D1 on the scalar
    K = np.eye(V) - 0.5 * D2s
    C = dense.cconj_dense(V)
    N = phis.shape[0]
    yp, ym = m + 2 * g * phis, np.conj(m) + 2 * np.conj(g) * np.conj(phis)
    M = Dsl[None] + np.stack([ym, ym, yp, yp], axis=2).reshape(N, 4 * V)[:, :, None] * np.eye(4 * V)[None]
    pf = pfaffian(C[None] @ M)
    Wp = m * phis + g * phis ** 2
    SB = (2 * np.einsum("nx,xy,ny->n", np.conj(phis), D2s, phis) + np.einsum("nx,xy,ny->n", np.conj(Wp), K, Wp)).real
    src = np.stack([np.tile(np.linalg.inv(CCONJ)[:, b], V) for b in range(4)], axis=1)
    psi = np.linalg.solve(M, np.broadcast_to(src, (N, 4 * V, 4))).reshape(N, V, 4, 4)  # [n, x, spin, b]
    pp = np.einsum("st,nxtb->nxsb", P_PLUS, psi)
    pm = np.einsum("st,nxtb->nxsb", P_MINUS, psi)
    d1p = np.einsum("ij,njb->nib", D1f, pp.reshape(N, 4 * V, 4)).reshape(N, V, 4, 4)
    d1m = np.einsum("ij,njb->nib", D1f, pm.reshape(N, 4 * V, 4)).reshape(N, V, 4, 4)
    f, fs = phis @ Kt.T, np.conj(phis) @ Kt.T
    gp = f[:, :, None, None] * np.einsum("st,nxtb->nxsb", GAMMA[0], pp)
    gm = fs[:, :, None, None] * np.einsum("st,nxtb->nxsb", GAMMA[0], pm)
    ph = phis[:, :, None, None]
    kv = g * (2 * ph * gp + ph ** 2 * d1p) + np.conj(g) * (2 * np.conj(ph) * gm + np.conj(ph) ** 2 * d1m)
    WR = kv.sum(axis=1)
    F = -np.sum(np.conj(m) * np.conj(phis) + np.conj(g) * np.conj(phis) ** 2, axis=1)
    return pf, SB, WR, F


@pytest.mark.slow
def test_ward_identity_holds_over_the_exact_measure_periodic_T3():
    dims = (3, 1, 1, 1)
    P = oracle.Params(dims=dims, m=2.0 + 0.5j, g=1.0 - 0.4j)
    rng = np.random.default_rng(2)
    # the batched evaluation is the dense route
    phis = rng.normal(size=(2, 3)) + 1j * rng.normal(size=(2, 3))
    _, _, WR, _ = batched_ward(P, phis)
    for i in range(2):
        np.testing.assert_allclose(WR[i], dense_ward_right(P, phis[i].reshape(dims), antiperiodic=False),
                                   rtol=0, atol=1e-12)
    # importance sampling from Gaussians at the two classical vacua phi = 0, -m/g
    vac, sigma, chunk, nchunk = -P.m / P.g, 0.8, 100000, 10
    acc = np.zeros(4, complex)
    parts = []
    for _ in range(nchunk):
        c0 = np.where(rng.random(chunk) < 0.5, 0.0, vac)[:, None]
        phis = c0 + (rng.normal(size=(chunk, 3)) + 1j * rng.normal(size=(chunk, 3))) * sigma / np.sqrt(2)
        q = sum(0.5 * np.exp(-np.sum(np.abs(phis - c) ** 2, axis=1) / sigma ** 2) for c in (0.0, vac))
        pf, SB, WR, F = batched_ward(P, phis)
        w = pf * np.exp(-SB) / q
        part = np.array([w.sum(), (w * WR[:, 0, 1]).sum(), (w * WR[:, 2, 3]).sum(), (w * F).sum()])
        parts.append(part[1:] / part[0])
        acc += part
    R01, R23, Fm = acc[1:] / acc[0]
    err = np.std(np.array(parts), axis=0, ddof=1) / np.sqrt(nchunk)
    # W_L[0][1] = F^* C[0][1] = -F^*, W_L[2][3] = F C[2][3] = F
    L01, L23 = -np.conj(Fm), Fm
    e = abs(err[2]) + 1e-12
    assert abs(R01 - L01) < 4 * e and abs(R23 - L23) < 4 * e
    assert abs(R01 + L01) > 4 * e                # not the opposite sign
    assert abs(R01 - (-Fm)) > 4 * e              # not F~ in every column
