"""GPU forces, actions, molecular dynamics and HMC checked against the oracle,
against exact central differences, and against the HMC invariants.

Tolerances: actions and the bosonic force are FP64 kernels compared at 1e-12
relative; the pseudofermion force depends on solves to a true residual tol, so
its error is about cond(M^dag M) * tol -- with tol = 1e-12 it is compared at
1e-8.  The finite-difference check follows the differentiation workload
(16^4, m = 0.1, g = 0.5, eps = 1e-6, 64 random sites, relative 1e-6).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import fftops, force as oforce, hmc as ohmc, philox  # noqa: E402
from paper_1005_3276_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def wz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1005_3276_gb300 import binding
    return binding


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 8, 8, 8), (16, 8, 8, 8)])
def test_actions_and_forces_match_oracle(wz, dims):
    P = oracle.Params(dims=dims, m=0.2 + 0.05j, g=0.4 - 0.1j)
    phi = synth.scalar_field(dims, 0.5, 3)
    eta = synth.spinor_rhs(2, dims, 4)
    lat = wz.Lattice(dims, m=P.m, g=P.g)
    lat.set_phi(phi)
    G = np.zeros(dims, dtype=np.complex128)
    sb, spf, _ = lat.force(eta, G, tol=1e-12, parts=wz.WZ_FORCE_BOSON)
    assert abs(sb - oforce.bosonic_action(P, phi)) <= 1e-12 * abs(sb)
    assert rel(G, oforce.bosonic_force(P, phi)) <= 1e-12
    sb2, spf, st = lat.force(eta, G, tol=1e-12, parts=wz.WZ_FORCE_FERMION)
    ref = sum(oforce.pf_force(P, phi, e, tol=1e-13) for e in eta)
    assert rel(G, ref) <= 1e-8
    spf_ref = sum(oforce.pf_action(P, phi, e, tol=1e-13) for e in eta)
    assert abs(spf - spf_ref) <= 1e-9 * abs(spf_ref)
    Gt = np.zeros_like(G)
    lat.force(eta, Gt, tol=1e-12)
    assert rel(Gt, ref + oforce.bosonic_force(P, phi)) <= 1e-8


def test_force_exact_central_difference_16(wz):
    """dS_pf/dphi at 64 random sites against (S(phi + eps e) - S(phi - eps e)) / 2 eps.

    At 16^4 S_pf ~ 1e5, so the difference is evaluated with the exact identity
    S+ - S- = (M_- X_+)^dag dY X_- + (dY X_+)^dag (M_+ X_-),  dY = Y(phi_-) - Y(phi_+),
    X_pm = (M_pm^dag M_pm)^-1 eta, which involves no cancellation."""
    w = synth.FORCE_16
    dims = w.dims
    phi = synth.scalar_field(dims, w.sigma, 0)
    R = philox.pseudofermion_source(7, 0, dims, 1)
    P = oracle.Params(dims=dims, m=w.m, g=w.g)
    eta = fftops.apply_Mdag(P, phi, R[0])[None]
    lat = wz.Lattice(dims, m=w.m, g=w.g)
    lat.set_phi(torch.from_numpy(phi).cuda())
    etad = torch.from_numpy(eta).cuda()
    G = torch.zeros(dims, dtype=torch.complex128, device="cuda")
    lat.force(etad, G, tol=1e-12, parts=wz.WZ_FORCE_FERMION)
    G = G.cpu().numpy()
    rng = np.random.default_rng(5)
    flat = rng.choice(int(np.prod(dims)), size=64, replace=False)
    eps = 1e-6
    c, g, m = 2.0, w.g, w.m
    worst = 0.0
    for fi in flat:
        site = np.unravel_index(fi, dims)
        for comp, e in ((0, 1.0), (1, 1j)):
            php, phm = phi.copy(), phi.copy()
            php[site] += eps * e
            phm[site] -= eps * e
            Xp = torch.zeros_like(etad)
            Xm = torch.zeros_like(etad)
            lat.set_phi(torch.from_numpy(php).cuda())
            lat.solve(etad, Xp, tol=1e-12)
            lat.set_phi(torch.from_numpy(phm).cuda())
            lat.solve(etad, Xm, tol=1e-12)
            MmXp = torch.empty_like(etad)
            lat.apply("M", Xp, MmXp)          # M_- X_+
            lat.set_phi(torch.from_numpy(php).cuda())
            MpXm = torch.empty_like(etad)
            lat.apply("M", Xm, MpXm)          # M_+ X_-
            torch.cuda.synchronize()
            d = phm[site] - php[site]         # -2 eps e
            dY = np.array([c * np.conj(g) * np.conj(d)] * 2 + [c * g * d] * 2)
            xp, xm = Xp[0][site].cpu().numpy(), Xm[0][site].cpu().numpy()
            zm, zp = MmXp[0][site].cpu().numpy(), MpXm[0][site].cpu().numpy()
            dS = np.sum(np.conj(zm) * dY * xm + np.conj(dY * xp) * zp)
            fd = dS.real / (2 * eps)
            an = G[site].real if comp == 0 else G[site].imag
            err = abs(fd - an) / max(abs(G[site]), 1e-12)
            worst = max(worst, err)
    assert worst <= 1e-6, worst


def test_trajectory_matches_oracle_4(wz):
    """One 4^4 trajectory (tau = 1, 10 leapfrog steps, one pseudofermion) with the
    device Philox draws reproduced by the oracle's Philox: same dH, decision, phi."""
    w = synth.SMALL_4
    dims = w.dims
    P = oracle.Params(dims=dims, m=w.m, g=w.g)
    phi0 = synth.scalar_field(dims, w.sigma, 0)
    seed, traj = 1234, 0
    lat = wz.Lattice(dims, m=w.m, g=w.g)
    lat.set_phi(phi0)
    st = lat.trajectory(tau=1.0, nsteps=10, npf=1, tol=1e-12, seed=seed, traj_index=traj,
                        flags=wz.WZ_HMC_FP64_SOLVES)
    phi_gpu = np.zeros_like(phi0)
    lat.get_phi(phi_gpu)
    pi0 = philox.momentum_field(seed, traj, dims)
    R = philox.pseudofermion_source(seed, traj, dims, 1)
    u = philox.accept_uniform(seed, traj)
    ref = ohmc.trajectory(P, phi0, pi0, R, u, tau=1.0, nsteps=10, tol=1e-13)
    assert abs(st["dH"] - ref["dH"]) <= 1e-8 * max(1.0, abs(ref["dH"]))
    assert abs(st["H0"] - ref["H0"]) <= 1e-10 * abs(ref["H0"])
    assert abs(st["u"] - u) == 0.0
    assert bool(st["accept"]) == ref["accept"]
    assert rel(phi_gpu, ref["phi"]) <= 1e-9
    assert st["force_evals"] == 11


def test_omelyan_trajectory_matches_oracle_4(wz):
    """One 4^4 Omelyan 2MN trajectory (lambda = 0.1931833275037836, tau = 1, 4
    steps) with two pseudofermions and complex couplings, from the device
    Philox draws reproduced by the oracle's Philox: same dH, decision and phi.
    The device merges the closing lambda-kick of a step with the opening one of
    the next (same phi, so the same force): 1 + 2 n force evaluations against
    the oracle's 3 n, with the same trajectory."""
    dims = (4, 4, 4, 4)
    P = oracle.Params(dims=dims, m=0.3 + 0.1j, g=0.6 - 0.2j)
    phi0 = synth.scalar_field(dims, 0.5, 5)
    seed, traj, nsteps = 4321, 2, 4
    lat = wz.Lattice(dims, m=P.m, g=P.g)
    lat.set_phi(phi0)
    st = lat.trajectory(tau=1.0, nsteps=nsteps, npf=2, integrator="omelyan", tol=1e-12, seed=seed,
                        traj_index=traj, flags=wz.WZ_HMC_FP64_SOLVES)
    phi_gpu = np.zeros_like(phi0)
    lat.get_phi(phi_gpu)
    pi0 = philox.momentum_field(seed, traj, dims)
    R = philox.pseudofermion_source(seed, traj, dims, 2)
    u = philox.accept_uniform(seed, traj)
    ref = ohmc.trajectory(P, phi0, pi0, R, u, tau=1.0, nsteps=nsteps, integrator="omelyan", tol=1e-13)
    print("omelyan 4^4 dH device", st["dH"], "oracle", ref["dH"])
    assert abs(st["dH"] - ref["dH"]) <= 1e-8 * max(1.0, abs(ref["dH"]))
    assert abs(st["H0"] - ref["H0"]) <= 1e-10 * abs(ref["H0"])
    assert bool(st["accept"]) == ref["accept"]
    assert rel(phi_gpu, ref["phi"]) <= 1e-9
    # the end of the molecular dynamics as well, whatever the decision
    lat.set_phi(phi0)
    pi = torch.from_numpy(pi0.copy()).cuda()
    etas = torch.from_numpy(np.stack(ref["etas"])).cuda()
    lat.md_integrate(pi, etas, tau=1.0, nsteps=nsteps, integrator="omelyan", tol=1e-12,
                      flags=wz.WZ_HMC_FP64_SOLVES)
    phi_md = torch.zeros_like(pi)
    lat.get_phi(phi_md)
    assert rel(phi_md.cpu().numpy(), ref["phi_md"]) <= 1e-9
    assert rel(pi.cpu().numpy(), ref["pi_md"]) <= 1e-9
    assert st["force_evals"] == 1 + 2 * nsteps


def test_ten_trajectories_4(wz):
    w = synth.SMALL_4
    lat = wz.Lattice(w.dims, m=w.m, g=w.g)
    lat.set_phi(synth.scalar_field(w.dims, w.sigma, 0))
    dh, acc = [], 0
    for t in range(w.extra["ntraj"]):
        st = lat.trajectory(tau=w.extra["tau"], nsteps=w.extra["nsteps"], npf=1, tol=1e-10, seed=99,
                            traj_index=t)
        dh.append(st["dH"])
        acc += st["accept"]
    assert np.all(np.isfinite(dh)) and acc >= 1
    print("4^4 dH:", np.round(dh, 4), "accepted", acc)


def test_reversibility_16(wz):
    """Differentiation workload: tau = 1, 20 leapfrog steps forward, momenta
    negated, 20 steps back: |delta phi| < 1e-10 (FP64 state)."""
    w = synth.FORCE_16
    dims = w.dims
    P = oracle.Params(dims=dims, m=w.m, g=w.g)
    phi0 = synth.scalar_field(dims, w.sigma, 0)
    R = philox.pseudofermion_source(11, 0, dims, 1)
    eta = torch.from_numpy(fftops.apply_Mdag(P, phi0, R[0])[None]).cuda()
    pi = torch.from_numpy(philox.momentum_field(11, 0, dims)).cuda()
    lat = wz.Lattice(dims, m=w.m, g=w.g)
    lat.set_phi(torch.from_numpy(phi0).cuda())
    kw = dict(tau=1.0, nsteps=w.extra["nsteps"], tol=1e-12)
    lat.md_integrate(pi, eta, **kw)
    pi.neg_()
    lat.md_integrate(pi, eta, **kw)
    phi = torch.zeros_like(pi)
    lat.get_phi(phi)
    dphi = float((phi - torch.from_numpy(phi0).cuda()).abs().max())
    print("16^4 reversibility |dphi| =", dphi)
    assert dphi < 1e-10


def test_dH_scales_as_dt2(wz):
    dims = (8, 8, 8, 8)
    P = oracle.Params(dims=dims, m=0.3, g=0.3)
    phi0 = synth.scalar_field(dims, 0.5, 2)
    R = philox.pseudofermion_source(3, 0, dims, 1)
    eta = torch.from_numpy(fftops.apply_Mdag(P, phi0, R[0])[None]).cuda()
    pi0 = torch.from_numpy(philox.momentum_field(3, 0, dims)).cuda()
    lat = wz.Lattice(dims, m=P.m, g=P.g)
    G = torch.zeros(dims, dtype=torch.complex128, device="cuda")

    def H(pi):
        sb, spf, _ = lat.force(eta, G, tol=1e-13)
        return 0.5 * float((pi.abs() ** 2).sum()) + sb + spf

    dH = []
    for n in (8, 16):
        lat.set_phi(torch.from_numpy(phi0).cuda())
        h0 = H(pi0)
        pi = pi0.clone()
        lat.md_integrate(pi, eta, tau=0.5, nsteps=n, tol=1e-13)
        dH.append(abs(H(pi) - h0))
    assert 3.0 < dH[0] / dH[1] < 5.0, dH


def test_autograd_function(wz):
    from paper_1005_3276_gb300.autograd import PseudofermionAction
    dims = (4, 4, 4, 4)
    P = oracle.Params(dims=dims, m=0.1, g=0.5)
    phi_np = synth.scalar_field(dims, 0.5, 8)
    eta_np = synth.spinor_rhs(1, dims, 9)
    lat = wz.Lattice(dims, m=P.m, g=P.g)
    phi = torch.from_numpy(phi_np).cuda().requires_grad_(True)
    eta = torch.from_numpy(eta_np).cuda()
    S = PseudofermionAction.apply(lat, phi, eta, 1e-12)
    S.backward()
    ref = oforce.pf_force(P, phi_np, eta_np[0], tol=1e-13)
    assert abs(float(S) - oforce.pf_action(P, phi_np, eta_np[0], tol=1e-13)) <= 1e-9 * abs(float(S))
    assert rel(phi.grad.cpu().numpy(), ref) <= 1e-8


def test_trajectory_graph_equals_eager(wz, monkeypatch):
    """Whole-trajectory CUDA graph (solver loops as conditional nodes) replayed
    for three consecutive trajectories equals the eagerly launched sequence."""
    dims = (8, 8, 8, 8)
    phi0 = synth.scalar_field(dims, 0.5, 4)
    runs = {}
    for flag in ("0", "1"):
        monkeypatch.setenv("WZ_NO_GRAPHS", flag)
        lat = wz.Lattice(dims, m=0.2, g=0.4)
        lat.set_phi(phi0)
        out = []
        for t in range(3):
            st = lat.trajectory(tau=0.5, nsteps=5, npf=2, tol=1e-10, seed=5, traj_index=t)
            out.append((st["dH"], st["accept"], st["cg_iterations"], st["force_evals"]))
        phi = np.zeros(dims, np.complex128)
        lat.get_phi(phi)
        runs[flag] = (out, phi)
        lat.close()
    assert runs["0"][0] == runs["1"][0]
    assert np.array_equal(runs["0"][1], runs["1"][1])


def test_action_matches_force_actions(wz):
    dims = (8, 8, 8, 8)
    P = oracle.Params(dims=dims, m=0.3, g=0.4)
    phi = synth.scalar_field(dims, 0.5, 12)
    eta = synth.spinor_rhs(2, dims, 13)
    lat = wz.Lattice(dims, m=P.m, g=P.g)
    lat.set_phi(phi)
    sb, spf, _ = lat.action(eta, 2, tol=1e-12)
    assert abs(sb - oforce.bosonic_action(P, phi)) <= 1e-12 * abs(sb)
    ref = sum(oforce.pf_action(P, phi, e, tol=1e-13) for e in eta)
    assert abs(spf - ref) <= 1e-9 * abs(ref)
