"""Ward-identity observables (Eq. exid) and the D1 apply on the GPU against the oracle."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import ward  # noqa: E402
from paper_1005_3276_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def wz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1005_3276_gb300 import binding
    return binding


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 8, 8, 8), (16, 8, 8, 8)])
def test_d1_apply_matches_oracle(wz, dims):
    P = oracle.Params(dims=dims, m=0.3, g=0.2)
    psi = synth.spinor_rhs(2, dims, 7)
    lat = wz.Lattice(dims, m=P.m, g=P.g)
    lat.set_phi(synth.scalar_field(dims, 0.5, 1))
    out = np.zeros_like(psi)
    lat.apply("D1", psi, out, 2)
    for k in range(2):
        ref = ward.spinor_d1(P, psi[k])
        assert np.abs(out[k] - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("dims,mixed", [((4, 4, 4, 4), False), ((8, 8, 8, 8), False), ((8, 8, 8, 8), True)])
def test_ward_identity_matches_oracle(wz, dims, mixed):
    P = oracle.Params(dims=dims, m=0.4 + 0.1j, g=0.3 - 0.2j)
    phi = synth.scalar_field(dims, 0.5, 3)
    lat = wz.Lattice(dims, m=P.m, g=P.g)
    lat.set_phi(phi)
    WR, WL, st = lat.ward_identity(tol=1e-12, mixed=mixed)
    assert st["converged"] == 4
    refR = ward.ward_right(P, phi, tol=1e-14)
    refL = ward.ward_left(P, phi)
    assert np.abs(WR - refR).max() <= 1e-8 * np.abs(refR).max()
    assert np.abs(WL - refL).max() <= 1e-12 * np.abs(refL).max()
