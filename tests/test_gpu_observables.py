"""Observables on the GPU against the oracle: the auxiliary-field VEV (Sec. 7.5)
and the locality probes f(r) of Dslash and of the overlap operator D (Sec. 3.2,
Eq. uir; the oracle pins f(0) = 0 and even r below odd r for Dslash, and the
exponential decay of |D(x, 0)|, on the paper's 16^4 lattice)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import fftops, force as oforce  # noqa: E402
from paper_1005_3276_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def wz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1005_3276_gb300 import binding
    return binding


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (16, 16, 16, 16)])
def test_aux_vev_matches_oracle(wz, dims):
    P = oracle.Params(dims=dims, m=0.5 + 0.1j, g=0.1 - 0.05j)
    phi = synth.scalar_field(dims, 0.5, 9)
    lat = wz.Lattice(dims, m=P.m, g=P.g)
    lat.set_phi(phi)
    F = lat.aux_vev()
    ref = oforce.auxiliary_vev(P, phi)
    assert abs(F - ref) <= 1e-13 * max(1.0, abs(ref))


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (16, 16, 16, 16)])
def test_locality_probe_matches_oracle(wz, dims):
    lat = wz.Lattice(dims)
    f = lat.locality()
    eta = np.zeros(dims + (4,), complex)
    eta[0, 0, 0, 0, 0] = 1.0
    psi = fftops.apply_dslash(eta)
    d = [np.minimum(np.arange(n), n - np.arange(n)) for n in dims]
    r = sum(np.meshgrid(*d, indexing="ij"))
    nrm = np.sqrt((np.abs(psi) ** 2).sum(-1))
    ref = np.array([nrm[r == k].max() for k in range(r.max() + 1)])
    assert f[0] <= 1e-14
    assert np.abs(f - ref).max() <= 1e-13 * ref.max()


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (16, 16, 16, 16), (32, 16, 16, 16)])
def test_overlap_locality_matches_oracle(wz, dims):
    lat = wz.Lattice(dims)
    f = lat.locality("D")
    eta = np.zeros(dims + (4,), complex)
    eta[0, 0, 0, 0, 0] = 1.0
    psi = fftops.apply_overlap(eta)
    d = [np.minimum(np.arange(n), n - np.arange(n)) for n in dims]
    r = sum(np.meshgrid(*d, indexing="ij"))
    nrm = np.sqrt((np.abs(psi) ** 2).sum(-1))
    ref = np.array([nrm[r == k].max() for k in range(r.max() + 1)])
    assert np.abs(f - ref).max() <= 1e-13 * ref.max()
    if dims == (16, 16, 16, 16):
        # exponential decay in the taxi-driver distance (the oracle's pin)
        slope = np.polyfit(np.arange(1, 13), np.log(f[1:13]), 1)[0]
        print("16^4 overlap |D(x,0)| log-slope per unit distance", slope)
        assert slope < -0.5


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_overlap_apply_matches_oracle(wz, dtype):
    """WZ_OP_D on random fields (several right-hand sides, both precisions)."""
    dims = (16, 8, 8, 8)
    lat = wz.Lattice(dims)
    x = synth.spinor_rhs(3, dims, 21)
    y = torch.empty((3,) + dims + (4,), dtype=dtype, device="cuda")
    lat.apply("D", torch.from_numpy(x).to(dtype).cuda(), y, 3)
    ref = np.stack([fftops.apply_overlap(xk) for xk in x])
    err = np.abs(y.cpu().numpy().astype(np.complex128) - ref).max() / np.abs(ref).max()
    assert err <= (1e-12 if dtype == torch.complex128 else 2e-6), err
