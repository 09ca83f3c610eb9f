"""Shifted solves, rational applies and RHMC on the GPU against the oracle
(Eqs. jkjk, hbeq, yuier; Secs. 7.2, 7.4).

Coefficients come from tests/golden/rational_coeffs.json (oracle Remez, written
by tests/golden/make_rational.py), so both sides evaluate the same rational
function.  Tolerances: every solve runs to FP64 true residual 1e-12, so a
solution differs from the oracle's by about cond * 1e-12; compared at 1e-8.
"""

import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import cg as ocg, force as oforce, hmc as ohmc, momentum, philox, rational  # noqa: E402
from paper_1005_3276_gb300 import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def wz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1005_3276_gb300 import binding
    return binding


def coeffs(name, kind):
    with open(os.path.join(HERE, "golden", "rational_coeffs.json")) as f:
        c = dict(json.load(f)[name][kind])
    c["alpha"], c["beta"] = np.array(c["alpha"]), np.array(c["beta"])
    return c


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("mixed", [True, False])
@pytest.mark.parametrize("pc", [False, True])
def test_multishift_matches_oracle(wz, mixed, pc):
    dims = (8, 8, 8, 8)
    P = oracle.Params(dims=dims, m=0.3 + 0.1j, g=0.4)
    phi = synth.scalar_field(dims, 0.5, 1)
    b = synth.spinor_rhs(2, dims, 2)
    shifts = [0.0, 0.5, 3.0, 40.0, 700.0]
    lat = wz.Lattice(dims, m=P.m, g=P.g)
    lat.set_phi(phi)
    x = np.zeros((len(shifts) * 2,) + b.shape[1:], np.complex128)
    rc, st, res = lat.solve_multishift(b, x, shifts, tol=1e-12, mixed=mixed, pc=pc, resid=True)
    assert rc == wz.WZ_OK and st["converged"] == len(shifts) * 2
    assert max(res) <= 1e-12 * 1.01
    for i, sh in enumerate(shifts):
        for j in range(2):
            ref, _, _ = ocg.solve_MdagM(P, phi, b[j], sh, 1e-13)
            assert rel(x[i * 2 + j], ref) <= 1e-8, (i, j)


@pytest.mark.parametrize("kind", ["action", "heatbath"])
def test_rational_apply_matches_oracle(wz, kind):
    dims = (4, 4, 4, 4)
    P = oracle.Params(dims=dims, m=0.5, g=0.3)
    phi = synth.scalar_field(dims, 0.4, 3)
    eta = synth.spinor_rhs(2, dims, 4)
    c = coeffs("L4_m0.5_d8", kind)
    lat = wz.Lattice(dims, m=P.m, g=P.g)
    lat.set_phi(phi)
    out = np.zeros_like(eta)
    st = lat.rational_apply(c, eta, out, tol=1e-12)
    assert st["converged"] == c["d"] * 2
    for j in range(2):
        ref = rational.rational_apply(P, phi, eta[j], c, tol=1e-13)
        assert rel(out[j], ref) <= 1e-9


def test_rational_apply_preconditioned_poles(wz):
    """Poles beta <= 100 solved in the preconditioned form, the rest without
    (Sec. 7.4): the same r(M^dag M) eta as the unpreconditioned apply."""
    dims = (8, 8, 8, 8)
    P = oracle.Params(dims=dims, m=0.5, g=0.2)
    phi = synth.scalar_field(dims, 0.3, 5)
    eta = synth.spinor_rhs(1, dims, 6)
    c = coeffs("L8_m0.5_d10", "action")
    assert (c["beta"] <= 100).any() and (c["beta"] > 100).any()
    lat = wz.Lattice(dims, m=P.m, g=P.g)
    lat.set_phi(phi)
    a = np.zeros_like(eta)
    b = np.zeros_like(eta)
    s_plain = lat.rational_apply(c, eta, a, tol=1e-12)
    s_pc = lat.rational_apply(c, eta, b, tol=1e-12, pc=True, pc_cutoff=100.0)
    ref = rational.rational_apply(P, phi, eta[0], c, tol=1e-13)
    assert rel(a[0], ref) <= 1e-9
    assert rel(b[0], ref) <= 1e-9
    print("rational apply iterations: plain", s_plain["total_iterations"], "pc", s_pc["total_iterations"])


def test_heatbath_action_identity(wz):
    """eta = r_h(M^dag M) R with r_h ~ x^1/8 and r_a ~ x^-1/4: eta^dag r_a eta = |R|^2
    up to the approximation errors (the RHMC heatbath property)."""
    dims = (8, 8, 8, 8)
    phi = synth.scalar_field(dims, 0.3, 7)
    R = philox.pseudofermion_source(3, 0, dims, 1)
    ca, ch = coeffs("L8_m0.5_d10", "action"), coeffs("L8_m0.5_d10", "heatbath")
    lat = wz.Lattice(dims, m=0.5, g=0.2)
    lat.set_phi(phi)
    eta = np.zeros_like(R)
    lat.rational_apply(ch, R, eta, tol=1e-12)
    y = np.zeros_like(R)
    lat.rational_apply(ca, eta, y, tol=1e-12)
    S = float(np.vdot(eta, y).real)
    RR = float(np.vdot(R, R).real)
    bound = (1 + ch["err"]) ** 2 * (1 + ca["err"]) - 1
    assert abs(S / RR - 1) <= bound + 1e-10


@pytest.mark.parametrize("dims,m", [((4, 4, 4, 4), 0.5), ((16, 16, 16, 16), 0.1), ((16, 8, 8, 8), 0.3 + 0.2j)])
def test_spectral_bounds(wz, dims, m):
    lat = wz.Lattice(dims, m=m, g=0.1)
    lo, hi = lat.spectral_bounds()
    den = momentum.free_norm(dims, m)
    assert lo == pytest.approx(den.min(), rel=1e-13)
    assert hi == pytest.approx(den.max(), rel=1e-13)


def test_rhmc_force_matches_oracle(wz):
    dims = (4, 4, 4, 4)
    P = oracle.Params(dims=dims, m=0.5, g=0.3 + 0.1j)
    phi = synth.scalar_field(dims, 0.4, 8)
    eta = synth.spinor_rhs(2, dims, 9)
    c = coeffs("L4_m0.5_d8", "action")
    lat = wz.Lattice(dims, m=P.m, g=P.g)
    lat.set_phi(phi)
    G = np.zeros(dims, np.complex128)
    sb, spf, st = lat.rhmc_force(eta, 2, c, G, tol=1e-12)
    refG = oforce.bosonic_force(P, phi) + sum(oforce.rational_pf_force(P, phi, e, c, tol=1e-13) for e in eta)
    refS = sum(oforce.rational_pf_action(P, phi, e, c, tol=1e-13) for e in eta)
    assert rel(G, refG) <= 1e-8
    assert abs(spf - refS) <= 1e-10 * abs(refS)
    assert abs(sb - oforce.bosonic_action(P, phi)) <= 1e-12 * abs(sb)
    assert st["converged"] == 2 * c["d"]


def test_rhmc_trajectory_matches_oracle_4(wz):
    dims = (4, 4, 4, 4)
    P = oracle.Params(dims=dims, m=0.5, g=0.3)
    phi0 = synth.scalar_field(dims, 0.4, 0)
    ca, ch = coeffs("L4_m0.5_d8", "action"), coeffs("L4_m0.5_d8", "heatbath")
    seed, traj = 77, 3
    lat = wz.Lattice(dims, m=P.m, g=P.g)
    lat.set_phi(phi0)
    st = lat.rhmc_trajectory(ca, ch, tau=0.5, nsteps=6, npf=1, tol=1e-12, seed=seed, traj_index=traj,
                             flags=wz.WZ_HMC_FP64_SOLVES)
    phi_gpu = np.zeros_like(phi0)
    lat.get_phi(phi_gpu)
    pi0 = philox.momentum_field(seed, traj, dims)
    R = philox.pseudofermion_source(seed, traj, dims, 1)
    u = philox.accept_uniform(seed, traj)
    ref = ohmc.rhmc_trajectory(P, phi0, pi0, R, u, ca, ch, tau=0.5, nsteps=6, tol=1e-13)
    assert abs(st["H0"] - ref["H0"]) <= 1e-10 * abs(ref["H0"])
    assert abs(st["dH"] - ref["dH"]) <= 1e-8 * max(1.0, abs(ref["dH"]))
    assert bool(st["accept"]) == ref["accept"]
    assert rel(phi_gpu, ref["phi"]) <= 1e-9
    assert st["force_evals"] == 7


def test_rhmc_trajectory_graph_equals_eager(wz, monkeypatch):
    dims = (8, 8, 8, 8)
    phi0 = synth.scalar_field(dims, 0.3, 4)
    ca, ch = coeffs("L8_m0.5_d10", "action"), coeffs("L8_m0.5_d10", "heatbath")
    runs = {}
    for flag in ("0", "1"):
        monkeypatch.setenv("WZ_NO_GRAPHS", flag)
        lat = wz.Lattice(dims, m=0.5, g=0.3)
        lat.set_phi(phi0)
        out = []
        for t in range(3):
            st = lat.rhmc_trajectory(ca, ch, tau=0.5, nsteps=4, npf=2, tol=1e-10, seed=5, traj_index=t)
            out.append((st["dH"], st["accept"], st["cg_iterations"], st["force_evals"]))
        phi = np.zeros(dims, np.complex128)
        lat.get_phi(phi)
        runs[flag] = (out, phi)
        lat.close()
    assert runs["0"][0] == runs["1"][0]
    assert np.array_equal(runs["0"][1], runs["1"][1])


def test_rhmc_dH_scales_as_dt2(wz):
    dims = (8, 8, 8, 8)
    phi0 = synth.scalar_field(dims, 0.3, 6)
    ca, ch = coeffs("L8_m0.5_d10", "action"), coeffs("L8_m0.5_d10", "heatbath")
    dH = []
    for n in (6, 12):
        lat = wz.Lattice(dims, m=0.5, g=0.3)
        lat.set_phi(phi0)
        st = lat.rhmc_trajectory(ca, ch, tau=0.5, nsteps=n, npf=1, tol=1e-12, seed=8, traj_index=0,
                                 flags=wz.WZ_HMC_NO_METROPOLIS)
        dH.append(abs(st["dH"]))
        lat.close()
    assert 3.0 < dH[0] / dH[1] < 5.0, dH


def test_heatbath_table_lattice_quick_convergence(wz):
    """The rational heatbath of the paper's heatbath table on 8^3 x 32 (m = 1,
    g = 0.1, degree 20, poles up to beta = 100 preconditioned, Sec. 7.4): the
    preconditioned systems converge within the solver's first chunk of
    iterations, so the solver's tuner times chunks in which every system has
    already finished.  Two mixed applies at 1e-6 in a row must agree with the
    FP64 apply at 1e-12 to the order of that tolerance."""
    dims = (32, 8, 8, 8)
    lat = wz.Lattice(dims, m=1.0, g=0.1)
    lat.set_phi(torch.from_numpy(synth.scalar_field(dims, 0.5, 0)).cuda())
    lo, hi = lat.spectral_bounds()
    rh = wz.wz_rational_minimax(0.125, 0.5 * lo, 2.0 * hi, 20)
    R = torch.from_numpy(synth.spinor_rhs(1, dims, 1)).cuda()
    ref = torch.empty_like(R)
    lat.rational_apply(rh, R, ref, tol=1e-12, mixed=False, pc=True)
    for _ in range(2):
        eta = torch.full_like(R, float("nan"))
        lat.rational_apply(rh, R, eta, tol=1e-6, mixed=True, pc=True)
        torch.cuda.synchronize()
        assert float((eta - ref).abs().max() / ref.abs().max()) <= 1e-4
    lat.close()
