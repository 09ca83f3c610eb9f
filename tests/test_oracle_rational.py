"""Pins of the oracle's rational approximation and RHMC pieces (Eqs. jkjk, hbeq,
yuier; Secs. 7.2, 7.4) against closed forms and theorems, not against itself:

* degree 0: the best constant relative approximation of x^gamma in closed form;
* gamma = -1/2: Zolotarev's closed-form optimum (elliptic functions);
* Chebyshev's alternation theorem: 2d+2 alternating extrema of equal size and no
  larger error anywhere (de la Vallee Poussin bounds the optimum from both sides);
* Stieltjes structure: x^-gamma (0 < gamma < 1) has positive residues and poles
  on the negative axis, x^+gamma negative residues;
* free field: M0^dagger M0 is diagonal in momentum space, so r(M0^dagger M0) eta
  via shifted CG equals r(den(p)) in momentum space, and lies within the
  approximation error of den(p)^gamma;
* the rational pseudofermion force is the gradient of the rational action
  (central differences).
"""

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

import oracle
from oracle import fftops, force, momentum, rational
from paper_1005_3276_gb300 import synth


def dense_logx(lo, hi, n=200001):
    return np.exp(np.linspace(np.log(lo), np.log(hi), n))


@pytest.mark.parametrize("gamma", [-0.25, 0.125])
def test_degree_zero_closed_form(gamma):
    lo, hi = 1.0, 100.0
    c = rational.minimax(gamma, lo, hi, 0)
    u, v = lo ** -gamma, hi ** -gamma
    assert c["a0"] == pytest.approx(2.0 / (u + v), rel=1e-14)
    assert c["err"] == pytest.approx(abs(v - u) / (u + v), rel=1e-14)


def test_inverse_sqrt_is_zolotarev():
    lo, hi, d = 0.01, 100.0, 6
    c = rational.minimax(-0.5, lo, hi, d)
    poles, zeros, C, err = rational.zolotarev_inverse_sqrt(lo, hi, d)
    assert c["err"] == pytest.approx(err, rel=1e-6)
    np.testing.assert_allclose(c["beta"], np.sort(poles), rtol=1e-8)


@pytest.mark.parametrize("gamma,lo,hi,d", [(-0.25, 0.5, 3000.0, 6), (0.125, 0.5, 3000.0, 6), (-0.25, 0.01, 100.0, 3)])
def test_alternation_theorem(gamma, lo, hi, d):
    c = rational.minimax(gamma, lo, hi, d)
    x = dense_logx(lo, hi)
    e = rational.relative_error(c, gamma, x)
    E = c["err"]
    assert np.abs(e).max() <= E * (1 + 1e-6)
    # count alternating extrema reaching the level
    s, last, count = 0, 0, 0
    for v in e:
        if abs(v) >= E * (1 - 1e-3):
            sg = 1 if v > 0 else -1
            if sg != last:
                count += 1
                last = sg
    assert count >= 2 * d + 2


def test_stieltjes_signs_and_degree_monotone():
    lo, hi = 0.5, 3000.0
    prev = {}
    for gamma in (-0.25, 0.125):
        errs = []
        for d in (2, 4, 6):
            c = rational.minimax(gamma, lo, hi, d)
            assert np.all(c["beta"] > 0)
            if gamma < 0:
                assert np.all(c["alpha"] > 0) and c["a0"] > 0
            else:
                assert np.all(c["alpha"] < 0) and c["a0"] > 0
            errs.append(c["err"])
        assert errs[0] > errs[1] > errs[2]
        prev[gamma] = c
    # heatbath squared times action ~ 1 (x^(1/8))^2 x^(-1/4) = 1
    x = dense_logx(lo, hi, 20001)
    comp = rational.evaluate(prev[0.125], x) ** 2 * rational.evaluate(prev[-0.25], x)
    bound = (1 + prev[0.125]["err"]) ** 2 * (1 + prev[-0.25]["err"]) - 1
    assert np.abs(comp - 1).max() <= bound * (1 + 1e-9)


def test_rational_apply_free_field_momentum_space():
    dims = (4, 4, 4, 4)
    P = oracle.Params(dims=dims, m=0.5, g=0.0)
    den = momentum.free_norm(dims, P.m)
    lo, hi = den.min() * 0.9, den.max() * 1.1
    coef = rational.minimax(-0.25, lo, hi, 5)
    eta = synth.spinor_rhs(1, dims, 3)[0]
    phi = np.zeros(dims, complex)
    out = rational.rational_apply(P, phi, eta, coef, tol=1e-14)
    exact_r = fftops.ifft4_fermion(rational.evaluate(coef, den)[..., None] * fftops.fft4_fermion(eta))
    np.testing.assert_allclose(out, exact_r, rtol=0, atol=1e-11 * np.abs(exact_r).max())
    power = fftops.ifft4_fermion(den[..., None] ** -0.25 * fftops.fft4_fermion(eta))
    assert np.linalg.norm(out - power) <= coef["err"] * np.linalg.norm(power) * (1 + 1e-6) + 1e-12


def test_rational_force_is_gradient():
    dims = (4, 4, 4, 4)
    P = oracle.Params(dims=dims, m=0.5, g=0.3)
    phi = synth.scalar_field(dims, 0.3, 5)
    eta = synth.spinor_rhs(1, dims, 6)[0]
    coef = rational.minimax(-0.25, 0.5, 1600.0, 3)
    G = force.rational_pf_force(P, phi, eta, coef, tol=1e-14)
    rng = np.random.default_rng(0)
    h = 1e-5
    for _ in range(4):
        site = tuple(int(rng.integers(0, n)) for n in dims)
        for comp, unit in ((0, 1.0), (1, 1j)):
            dp = np.zeros(dims, complex)
            dp[site] = unit * h
            sp = force.rational_pf_action(P, phi + dp, eta, coef, tol=1e-14)
            sm = force.rational_pf_action(P, phi - dp, eta, coef, tol=1e-14)
            fd = (sp - sm) / (2 * h)
            an = G[site].real if comp == 0 else G[site].imag
            assert fd == pytest.approx(an, rel=1e-6, abs=1e-8)
