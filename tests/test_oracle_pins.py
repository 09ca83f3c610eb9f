"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it follows.  None of these tests compares the
oracle with itself: the references are printed values (tests/golden), closed
forms, algebraic identities, brute force on tiny lattices, dense position-space
constructions from the Sec. 2.2 definitions, dense LU, and finite differences.
"""

import itertools
import json
import os

import numpy as np
import pytest

from oracle import cg, dense, fftops, force, hmc, momentum, philox
from oracle.conventions import CCONJ, GAMMA, GAMMA5, P_MINUS, P_PLUS, Params

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def rnd_field(shape, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def dense44():
    dims = (4, 4, 4, 4)
    D1, D2, D = dense.build_overlap(dims)
    return dims, D1, D2, D


@pytest.fixture(scope="module")
def dense2():
    dims = (2, 2, 2, 2)
    D1, D2, D = dense.build_overlap(dims)
    return dims, D1, D2, D


# ------------------------------------------------------------------ conventions (Sec. 2.1)


def test_gamma_matrices_match_printed():
    gm = GOLDEN["gamma_matrices"]
    for mu in range(4):
        g = np.array(gm[f"gamma{mu}"], dtype=float)
        assert np.array_equal(g[..., 0] + 1j * g[..., 1], GAMMA[mu])
    assert np.array_equal(np.diag(GAMMA5).real, np.array(gm["gamma5_diag"], dtype=float))


def test_clifford_algebra_and_charge_conjugation():
    I4 = np.eye(4)
    for mu, nu in itertools.product(range(4), repeat=2):
        ac = GAMMA[mu] @ GAMMA[nu] + GAMMA[nu] @ GAMMA[mu]
        assert np.allclose(ac, 2.0 * (mu == nu) * I4, atol=0)
    for mu in range(4):
        assert np.allclose(GAMMA[mu], GAMMA[mu].conj().T)
        assert np.allclose(GAMMA5 @ GAMMA[mu] + GAMMA[mu] @ GAMMA5, 0)
        Cinv = np.linalg.inv(CCONJ)
        assert np.allclose(CCONJ @ GAMMA[mu] @ Cinv, -GAMMA[mu].T)
    assert np.allclose(CCONJ.T, -CCONJ)
    assert np.allclose(P_PLUS + P_MINUS, I4) and np.allclose(P_PLUS @ P_MINUS, 0)


# ------------------------------------------------------------------ momentum space (Secs. 2.2, 3.1)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 6, 4, 2), (16, 4, 8, 12)])
def test_ginsparg_wilson_and_gamma5_hermiticity_per_momentum(dims):
    D = momentum.overlap_D(dims)
    g5 = GAMMA5
    gw = g5 @ D + D @ g5 - D @ g5 @ D
    assert np.abs(gw).max() < 1e-13
    Ddag = np.conj(np.swapaxes(D, -1, -2))
    assert np.abs(g5 @ D @ g5 - Ddag).max() < 1e-13
    V = np.eye(4) - D
    assert np.abs(V @ np.conj(np.swapaxes(V, -1, -2)) - np.eye(4)).max() < 1e-13
    ev = np.linalg.eigvals(D.reshape(-1, 4, 4))
    assert np.abs(np.abs(ev - 1.0) - 1.0).max() < 1e-13  # spectrum on |z - 1| = 1


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 2, 4, 8)])
def test_paper_identities_per_momentum(dims):
    """Gamma5^2 = 1 - D2/2, D^dagger D = 2 D2 (Sec. 2.2); D1^2 - D2^2 = -2 D2
    (Sec. 3.1); (1 - D2/2)^-1 D1 = (1 - D/2)^-1 D (Sec. 2.2); {Dslash, g5} = 0."""
    D1, D2 = momentum.D1_D2(dims)
    D = momentum.overlap_D(dims)
    I4 = np.eye(4)
    D2m = D2[..., None, None] * I4
    assert np.abs(D - (D1 + D2m)).max() < 1e-13
    Ddag = np.conj(np.swapaxes(D, -1, -2))
    assert np.abs(Ddag @ D - 2.0 * D2m).max() < 1e-13
    assert np.abs(D1 @ D1 - D2m @ D2m + 2.0 * D2m).max() < 1e-13
    G5 = GAMMA5 @ (I4 - 0.5 * D)
    assert np.abs(G5 @ G5 - (I4 - 0.5 * D2m)).max() < 1e-13
    ds = momentum.dslash_symbol(dims)
    alt = np.linalg.solve(I4 - 0.5 * D, D)
    assert rel(ds, alt) < 1e-12
    assert np.abs(ds @ GAMMA5 + GAMMA5 @ ds).max() < 1e-12
    # anti-Hermitian
    assert np.abs(ds + np.conj(np.swapaxes(ds, -1, -2))).max() < 1e-12


@pytest.mark.parametrize("L", [2, 4, 6, 8])
def test_doubler_zeros_periodic(L):
    """Eq. woube: 1 - D2/2 vanishes exactly on the 15 doublers, 2 D2 = 4 there."""
    dims = (L, L, L, L)
    D2, K = momentum.scalar_D2_K(dims)
    gold = GOLDEN["doublers"]
    h = L // 2
    corners = [c for c in itertools.product((0, h), repeat=4) if any(c)]
    assert len(corners) == gold["count"]
    for c in corners:
        assert K[c] == gold["one_minus_half_D2_on_doublers"]
        assert 2.0 * D2[c] == gold["two_D2_on_doublers"]
    mask = np.ones(dims, bool)
    for c in corners:
        mask[c] = False
    assert K[mask].min() > 0.0
    assert D2[0, 0, 0, 0] == 0.0


@pytest.mark.parametrize("T", [2, 4, 8, 16, 32])
def test_no_zero_modes_antiperiodic_even_T(T):
    """Sec. 3.1: antiperiodic time with even T removes the zeros of 1 - D2/2."""
    dims = (T, 4, 4, 4)
    b, omega, s = momentum.symbol_parts(dims, fermion=True)
    assert ((omega + b) / (2 * omega)).min() > 0.0


def test_max_eigenvalue_grows_with_T():
    """Sec. 3.1: the largest eigenvalue of Dslash diverges as T grows."""
    vals = []
    for T in (8, 16, 32, 64):
        h = momentum.h_of_p((T, 4, 4, 4))
        _, _, s = momentum.symbol_parts((T, 4, 4, 4))
        vals.append((h * np.sqrt(sum(x * x for x in s))).max())
    assert all(b > 1.8 * a for a, b in zip(vals, vals[1:]))


# ------------------------------------------------------------------ FFT vs brute-force DFT


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 3, 2), (4, 4, 4, 4)])
def test_fft_matches_brute_force_dft(dims):
    psi = rnd_field(dims + (4,), 3)
    T, Z, Y, X = dims
    x = np.stack(np.meshgrid(*[np.arange(n) for n in dims], indexing="ij"), -1).reshape(-1, 4)
    pt = np.pi * (2 * np.arange(T) + 1) / T
    pz, py, px = (2 * np.pi * np.arange(n) / n for n in (Z, Y, X))
    p = np.stack(np.meshgrid(pt, pz, py, px, indexing="ij"), -1).reshape(-1, 4)
    E = np.exp(-1j * p @ x.T)
    ref = (E @ psi.reshape(-1, 4)).reshape(dims + (4,))
    assert rel(fftops.fft4_fermion(psi), ref) < 1e-13
    assert rel(fftops.ifft4_fermion(ref), psi) < 1e-13


# ------------------------------------------------------------------ dense position space (Sec. 2.2)


def test_dense_ginsparg_wilson(dense44):
    dims, D1, D2, D = dense44
    g5 = dense.gamma5_dense(256)
    assert np.abs(g5 @ D + D @ g5 - D @ g5 @ D).max() < 1e-13
    assert np.abs(g5 @ D @ g5 - D.conj().T).max() < 1e-13
    ev = np.linalg.eigvals(D)
    assert np.abs(np.abs(ev - 1.0) - 1.0).max() < 1e-12
    assert np.abs(D.conj().T @ D - 2.0 * D2).max() < 1e-12  # D^dag D = 2 D2


@pytest.mark.parametrize("which", ["2", "44"])
def test_dense_M_matches_fft_apply(which, dense2, dense44):
    dims, D1, D2, _ = dense2 if which == "2" else dense44
    P = Params(dims=dims, m=0.1 + 0.03j, g=0.3 - 0.1j)
    phi = rnd_field(dims, 5, 0.5)
    n = D1.shape[0]
    dsl = np.linalg.solve(np.eye(n) - 0.5 * D2, D1)
    M = dsl + dense.build_Y(P, phi)
    vecs = rnd_field((3, n), 6)
    for v in vecs:
        psi = v.reshape(dims + (4,))
        assert rel(fftops.apply_M(P, phi, psi).ravel(), M @ v) < 1e-12
        assert rel(fftops.apply_Mdag(P, phi, psi).ravel(), M.conj().T @ v) < 1e-12
    # {Dslash, gamma5} = 0 in position space (Sec. 3.1)
    g5 = dense.gamma5_dense(n // 4)
    assert np.abs(dsl @ g5 + g5 @ dsl).max() < 1e-11


@pytest.mark.parametrize("which", ["2", "44"])
def test_dense_overlap_matches_fft_apply(which, dense2, dense44):
    """The overlap operator applied through the FFT equals the dense
    position-space D = 1 - A (A^dag A)^-1/2 of Sec. 2.2 (eigendecomposition of
    the dense Wilson kernel with the antiperiodic time hop)."""
    dims, _, _, D = dense2 if which == "2" else dense44
    for v in rnd_field((3, D.shape[0]), 12):
        assert rel(fftops.apply_overlap(v.reshape(dims + (4,))).ravel(), D @ v) < 1e-12


def test_dense_scalar_D2_matches_fft(dense2):
    dims = (2, 4, 2, 2)
    D2blk = dense.build_scalar_D2(dims)
    assert np.abs(D2blk[:, 1, :, 1] - D2blk[:, 0, :, 0]).max() < 1e-13
    assert np.abs(D2blk[:, 0, :, 1]).max() < 1e-13
    P = Params(dims=dims)
    f = rnd_field(dims, 8)
    assert rel(fftops.apply_D2_scalar(P, f).ravel(), D2blk[:, 0, :, 0] @ f.ravel()) < 1e-12


def test_charge_conjugation_antisymmetry_and_real_pfaffian(dense2):
    """Sec. 7.1: C M is antisymmetric and Pf(CM) is real, so det M = Pf^2 / det C
    is real and non-negative."""
    dims, D1, D2, D = dense2
    P = Params(dims=dims, m=0.2 + 0.1j, g=0.4 + 0.2j)
    phi = rnd_field(dims, 9, 0.7)
    n = D1.shape[0]
    M = np.linalg.solve(np.eye(n) - 0.5 * D2, D1) + dense.build_Y(P, phi)
    CM = dense.cconj_dense(n // 4) @ M
    assert np.abs(CM + CM.T).max() < 1e-12 * np.abs(CM).max()
    sign, _ = np.linalg.slogdet(M)
    assert abs(sign - 1.0) < 1e-9  # real, positive


@pytest.mark.parametrize("which", ["2", "44"])
def test_auxiliary_block_schur_and_determinant(which, dense2, dense44):
    """Eqs. kisu, lata: integrating X out of the block operator leaves M, and
    det K = det(D - 2) det M.  At 4^4 the block operator is 2048 x 2048."""
    dims, D1, D2, D = dense2 if which == "2" else dense44
    P = Params(dims=dims, m=0.1, g=0.1)
    phi = rnd_field(dims, 10, 0.5)
    n = D.shape[0]
    K = dense.build_aux_block(P, phi, D)
    assert K.shape == (2 * n, 2 * n)
    # change of variables chi = chi~ - X
    Tm = np.block([[np.eye(n), -np.eye(n)], [np.zeros((n, n)), np.eye(n)]])
    Kp = Tm.T @ K @ Tm
    A, B, C_, E = Kp[:n, :n], Kp[:n, n:], Kp[n:, :n], Kp[n:, n:]
    schur = A - B @ np.linalg.solve(E, C_)
    M = np.linalg.solve(np.eye(n) - 0.5 * D2, D1) + dense.build_Y(P, phi)
    assert rel(schur, M) < 1e-11
    sK, lK = np.linalg.slogdet(K)
    sE, lE = np.linalg.slogdet(D - 2.0 * np.eye(n))
    sM, lM = np.linalg.slogdet(M)
    assert abs(lK - (lE + lM)) < 1e-9 * max(1.0, abs(lK))
    assert abs(sK - sE * sM) < 1e-8


# ------------------------------------------------------------------ free theory (Sec. 7.3)


def test_free_preconditioner_closed_form():
    dims = (8, 4, 4, 4)
    P = Params(dims=dims, m=0.3 - 0.2j)
    M0p = fftops.M0_symbol(P)
    M0dag = np.conj(np.swapaxes(M0p, -1, -2))
    den = momentum.free_norm(dims, P.m)
    assert rel(M0dag @ M0p, den[..., None, None] * np.eye(4)) < 1e-13
    assert rel(fftops.M0inv_symbol(P) @ M0p, np.broadcast_to(np.eye(4), M0p.shape)) < 1e-13


def test_free_solve_closed_form():
    dims = (4, 4, 4, 4)
    P = Params(dims=dims, m=0.2, g=0.0)
    phi = np.zeros(dims, complex)
    b = rnd_field(dims + (4,), 11)
    x, it, res = cg.solve_MdagM(P, phi, b, tol=1e-13)
    den = momentum.free_norm(dims, P.m)
    xref = fftops.ifft4_fermion(fftops.fft4_fermion(b) / den[..., None])
    assert rel(x, xref) < 1e-11 and res < 1e-12


# ------------------------------------------------------------------ CG vs dense LU


@pytest.mark.parametrize("which", ["2", "44"])
def test_cg_matches_dense_lu(which, dense2, dense44):
    dims, D1, D2, _ = dense2 if which == "2" else dense44
    P = Params(dims=dims, m=0.1, g=0.3)
    phi = rnd_field(dims, 12, 0.5)
    n = D1.shape[0]
    M = np.linalg.solve(np.eye(n) - 0.5 * D2, D1) + dense.build_Y(P, phi)
    b = rnd_field(dims + (4,), 13)
    xref = np.linalg.solve(M.conj().T @ M, b.ravel())
    x, _, res = cg.solve_MdagM(P, phi, b, tol=1e-13)
    assert res < 1e-12 and rel(x.ravel(), xref) < 1e-10
    xs, _, _ = cg.solve_MdagM(P, phi, b, shift=0.7, tol=1e-13)
    xsref = np.linalg.solve(M.conj().T @ M + 0.7 * np.eye(n), b.ravel())
    assert rel(xs.ravel(), xsref) < 1e-10
    xp, itp, resp = cg.solve_MdagM_pc(P, phi, b, tol=1e-13)
    assert resp < 1e-11 and rel(xp.ravel(), xref) < 1e-9


def test_yukawa_coefficient_reading():
    """Eq. fmat (2 g) versus Sec. 7.1 (g): coefficient 1 at g equals 2 at g/2."""
    dims = (4, 4, 4, 4)
    phi = rnd_field(dims, 14, 0.5)
    psi = rnd_field(dims + (4,), 15)
    a = fftops.apply_M(Params(dims=dims, m=0.1, g=0.4, yukawa=1.0), phi, psi)
    b = fftops.apply_M(Params(dims=dims, m=0.1, g=0.2, yukawa=2.0), phi, psi)
    assert rel(a, b) < 1e-15


# ------------------------------------------------------------------ forces vs finite differences


def _fd(fun, phi, site, comp, eps):
    e = np.zeros_like(phi)
    e[site] = eps if comp == 0 else 1j * eps
    return (fun(phi + e) - fun(phi - e)) / (2 * eps)


def test_bosonic_action_dense_and_force_fd():
    dims = (2, 4, 2, 2)
    P = Params(dims=dims, m=0.3 + 0.1j, g=0.5 - 0.2j)
    phi = rnd_field(dims, 16, 0.5)
    D2d = dense.build_scalar_D2(dims)[:, 0, :, 0]
    W = (P.m * phi + P.g * phi * phi).ravel()
    Kd = np.eye(D2d.shape[0]) - 0.5 * D2d
    Sref = (2 * np.vdot(phi.ravel(), D2d @ phi.ravel()) + np.vdot(W, Kd @ W)).real
    assert abs(force.bosonic_action(P, phi) - Sref) < 1e-12 * abs(Sref)
    G = force.bosonic_force(P, phi)
    for site in [(0, 0, 0, 0), (1, 3, 1, 0), (0, 2, 1, 1)]:
        for comp in (0, 1):
            fd = _fd(lambda f: force.bosonic_action(P, f), phi, site, comp, 1e-5)
            an = G[site].real if comp == 0 else G[site].imag
            assert abs(fd - an) < 1e-7 * max(1.0, abs(an))


def test_pseudofermion_force_fd():
    dims = (4, 2, 2, 2)
    P = Params(dims=dims, m=0.2 + 0.05j, g=0.4 + 0.1j)
    phi = rnd_field(dims, 17, 0.5)
    eta = rnd_field(dims + (4,), 18)
    G = force.pf_force(P, phi, eta, tol=1e-14)
    for site in [(0, 0, 0, 0), (3, 1, 0, 1), (2, 0, 1, 1)]:
        for comp in (0, 1):
            fd = _fd(lambda f: force.pf_action(P, f, eta, tol=1e-14), phi, site, comp, 1e-5)
            an = G[site].real if comp == 0 else G[site].imag
            assert abs(fd - an) < 1e-6 * max(1.0, abs(an))


# ------------------------------------------------------------------ HMC invariants


def test_hmc_reversibility_and_dt_scaling():
    dims = (4, 2, 2, 2)
    P = Params(dims=dims, m=0.3, g=0.3)
    phi0 = rnd_field(dims, 19, 0.5)
    pi0 = rnd_field(dims, 20, 1.0 / np.sqrt(2))
    R = rnd_field((1,) + dims + (4,), 21, 0.5)
    etas = [fftops.apply_Mdag(P, phi0, R[0])]
    phi1, pi1, _ = hmc.integrate(P, phi0, pi0, etas, 0.5, 10, "leapfrog", 1e-14)
    phi2, pi2, _ = hmc.integrate(P, phi1, -pi1, etas, 0.5, 10, "leapfrog", 1e-14)
    assert np.abs(phi2 - phi0).max() < 1e-10 and np.abs(pi2 + pi0).max() < 1e-10
    H0 = hmc.hamiltonian(P, phi0, pi0, etas, 1e-14)
    dH = []
    for n in (8, 16):
        f, p, _ = hmc.integrate(P, phi0, pi0, etas, 0.5, n, "leapfrog", 1e-14)
        dH.append(abs(hmc.hamiltonian(P, f, p, etas, 1e-14) - H0))
    assert 3.0 < dH[0] / dH[1] < 5.0  # second-order integrator: dH ~ dt^2
    for n in (4, 8):
        f, p, _ = hmc.integrate(P, phi0, pi0, etas, 0.5, n, "omelyan", 1e-14)
        dH.append(abs(hmc.hamiltonian(P, f, p, etas, 1e-14) - H0))
    assert 3.0 < dH[2] / dH[3] < 5.0
    # initial pseudofermion action equals |R|^2 (heatbath with eta = M^dag R)
    X, _, _ = cg.solve_MdagM(P, phi0, etas[0], tol=1e-14)
    assert abs(np.vdot(etas[0], X).real - np.vdot(R[0], R[0]).real) < 1e-10 * np.vdot(R[0], R[0]).real


def test_md_integrators_at_g0_are_the_exact_mode_maps():
    """At g = 0 without pseudofermions the molecular dynamics of Sec. 7.2
    decouples into one harmonic oscillator per periodic momentum p, with
    omega^2(p) = 4 D2(p) + 2 |m|^2 K(p): the bosonic action is
    2 phi^* D2 phi + |m|^2 phi^* K phi and its real gradient is twice that
    operator on phi.  Leapfrog and the second-order minimum-norm scheme of
    Omelyan, Mryglod and Folk (velocity form, published lambda =
    0.1931833275037836) are then products of 2 x 2 kick and drift maps per
    mode, applied here to the Fourier modes with D2 and K written from their
    closed forms; the oracle's position-space MD must agree, and a different
    lambda must not."""
    dims = (4, 4, 4, 4)
    m = 0.4 + 0.2j
    P = Params(dims=dims, m=m, g=0.0)
    phi0 = rnd_field(dims, 31, 0.5)
    pi0 = rnd_field(dims, 32, 0.7)
    p = np.meshgrid(*[2.0 * np.pi * np.arange(n) / n for n in dims], indexing="ij")
    b = 1.0 - sum(2.0 * np.sin(0.5 * x) ** 2 for x in p)
    s = np.sqrt(b * b + sum(np.sin(x) ** 2 for x in p))
    D2 = 1.0 - b / s
    K = 1.0 - 0.5 * D2
    w2 = 4.0 * D2 + 2.0 * abs(m) ** 2 * K

    def evolve(seq):
        f, q = np.fft.fftn(phi0), np.fft.fftn(pi0)
        for kind, c in seq:
            if kind == "kick":
                q = q - c * w2 * f
            else:
                f = f + c * q
        return np.fft.ifftn(f), np.fft.ifftn(q)

    tau, n = 0.6, 3
    eps = tau / n

    def omelyan(lam):
        return [("kick", lam * eps), ("drift", 0.5 * eps), ("kick", (1.0 - 2.0 * lam) * eps),
                ("drift", 0.5 * eps), ("kick", lam * eps)] * n

    leapfrog = [("kick", 0.5 * eps)] + [("drift", eps), ("kick", eps)] * (n - 1) + [("drift", eps), ("kick", 0.5 * eps)]
    for name, seq in (("omelyan", omelyan(0.1931833275037836)), ("leapfrog", leapfrog)):
        f_ref, q_ref = evolve(seq)
        f, q, _ = hmc.integrate(P, phi0, pi0, [], tau, n, name)
        assert np.abs(f - f_ref).max() < 1e-12 and np.abs(q - q_ref).max() < 1e-12, name
    f_other, _ = evolve(omelyan(0.25))
    f, _, _ = hmc.integrate(P, phi0, pi0, [], tau, n, "omelyan")
    assert np.abs(f - f_other).max() > 1e-6


# ------------------------------------------------------------------ locality (Sec. 3.2)


def test_locality_probe():
    """Eq. uir / Fig. rfig on the paper's 16^4 lattice: f(0) = 0 for Dslash and
    even r lie below odd r (checked from r = 4 on: at r = 2 the even value sits
    between f(1) and f(3); the figure itself is not in the source).  The
    overlap D decays exponentially with the taxi-driver distance, Dslash has a
    much longer tail."""
    L = 16
    dims = (L, L, L, L)
    eta = np.zeros(dims + (4,), complex)
    eta[0, 0, 0, 0, 0] = 1.0
    psi = fftops.apply_dslash(eta)
    d = [np.minimum(np.arange(n), n - np.arange(n)) for n in dims]
    r = sum(np.meshgrid(*d, indexing="ij"))
    nrm = np.sqrt((np.abs(psi) ** 2).sum(-1))
    f = np.array([nrm[r == k].max() for k in range(r.max() + 1)])
    assert f[0] <= GOLDEN["locality"]["f_at_0"] + 1e-15
    for k in range(4, r.max(), 2):
        assert f[k] < f[k - 1] and f[k] < f[k + 1]
    Dp = momentum.overlap_D(dims)
    psiD = fftops.ifft4_fermion(fftops.spin_mult(Dp, fftops.fft4_fermion(eta)))
    nD = np.sqrt((np.abs(psiD) ** 2).sum(-1))
    fD = np.array([nD[r == k].max() for k in range(r.max() + 1)])
    slope = np.polyfit(np.arange(1, 13), np.log(fD[1:13]), 1)[0]
    assert slope < -0.5
    slope_dslash = np.polyfit(np.arange(9, 25, 2), np.log(f[9:25:2]), 1)[0]
    assert slope_dslash > 0.5 * slope  # Dslash: no comparable exponential decay


# ------------------------------------------------------------------ Philox (Salmon et al.)


def test_philox_known_answers():
    for v in GOLDEN["philox4x32_10_kat"]["vectors"]:
        ctr = np.array([int(c, 16) for c in v["ctr"]], dtype=np.uint64)
        key = np.array([int(k, 16) for k in v["key"]], dtype=np.uint64)
        out = philox.philox4x32_10(ctr, key)
        assert [int(w) for w in out] == [int(o, 16) for o in v["out"]]


def test_gaussian_draw_moments():
    z = philox.momentum_field(1234, 0, (16, 16, 16, 16))
    assert abs(z.real.mean()) < 0.01 and abs(z.imag.mean()) < 0.01
    assert abs(z.real.var() - 1.0) < 0.02 and abs(z.imag.var() - 1.0) < 0.02
    R = philox.pseudofermion_source(1234, 0, (8, 8, 8, 8), 2)
    assert abs((np.abs(R) ** 2).mean() - 1.0) < 0.02
