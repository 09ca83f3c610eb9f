"""GPU parity of the FFT-based operator applies against the FP64 oracle.

FP64 fields must match to 1e-12 relative (max-norm over the whole output);
FP32 fields to 2e-6, the rounding of a few FFT stages of length <= 32 in
single precision (unit roundoff 6e-8 times ~log2 V stages, with margin).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import fftops  # noqa: E402
from paper_1005_3276_gb300 import synth  # noqa: E402

TOL64 = 1e-12
TOL32 = 2e-6


@pytest.fixture(scope="module")
def wz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1005_3276_gb300 import binding
    return binding


def oracle_apply(op, P, phi, psi, shift=0.0):
    f = {
        "M": lambda v: fftops.apply_M(P, phi, v),
        "Mdag": lambda v: fftops.apply_Mdag(P, phi, v),
        "MdagM": lambda v: fftops.apply_MdagM(P, phi, v, shift),
        "Dslash": lambda v: fftops.apply_dslash(v, P.r, P.M0),
        "M0inv": lambda v: fftops.apply_M0inv(P, v),
        "M0inv_dag": lambda v: fftops.apply_M0inv(P, v, dagger=True),
        "Mtilde": lambda v: fftops.apply_Mtilde(P, phi, v),
        "Mtilde_dag": lambda v: fftops.apply_Mtilde_dag(P, phi, v),
        "Mtilde_dagM": lambda v: fftops.apply_Mtilde_dag(P, phi, fftops.apply_Mtilde(P, phi, v)) + shift * v,
    }[op]
    return np.stack([f(v) for v in psi])


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


ALL_OPS = ["M", "Mdag", "MdagM", "Dslash", "M0inv", "M0inv_dag", "Mtilde", "Mtilde_dag", "Mtilde_dagM"]
# (T, Z, Y, X): L^4 sizes, a ragged plane count (L = 6, 12), paper-shaped L^3 x T
DIMS = [(4, 4, 4, 4), (6, 6, 6, 6), (8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 16),
        (16, 8, 8, 8), (32, 8, 8, 8)]


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("op", ALL_OPS)
def test_apply_fp64_matches_oracle(wz, dims, op):
    nrhs = 2 if np.prod(dims) >= 65536 else 3
    P = oracle.Params(dims=dims, m=0.1 + 0.02j, g=0.3 - 0.05j)
    phi = synth.scalar_field(dims, 0.5, 0)
    psi = synth.spinor_rhs(nrhs, dims, 1)
    lat = wz.Lattice(dims, m=P.m, g=P.g)
    lat.set_phi(torch.from_numpy(phi).cuda())
    x = torch.from_numpy(psi).cuda()
    y = torch.empty_like(x)
    shift = 0.37 if op.endswith("M") else 0.0
    lat.apply(op, x, y, nrhs, shift)
    torch.cuda.synchronize()
    ref = oracle_apply(op, P, phi, psi, shift)
    assert rel(y.cpu().numpy(), ref) < TOL64


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (12, 12, 12, 12), (16, 16, 16, 16), (32, 8, 8, 8)])
@pytest.mark.parametrize("op", ["M", "Mdag", "MdagM", "Mtilde_dagM"])
def test_apply_fp32_matches_oracle(wz, dims, op):
    nrhs = 2
    P = oracle.Params(dims=dims, m=0.05, g=0.3)
    phi = synth.scalar_field(dims, 0.5, 2)
    psi = synth.spinor_rhs(nrhs, dims, 3)
    lat = wz.Lattice(dims, m=P.m, g=P.g)
    lat.set_phi(torch.from_numpy(phi).cuda())
    x = torch.from_numpy(psi.astype(np.complex64)).cuda()
    y = torch.empty_like(x)
    lat.apply(op, x, y, nrhs, 0.0)
    torch.cuda.synchronize()
    ref = oracle_apply(op, P, phi, psi.astype(np.complex64).astype(np.complex128))
    assert rel(y.cpu().numpy().astype(np.complex128), ref) < TOL32


def test_apply_host_buffers_and_aliasing(wz):
    dims = (8, 8, 8, 8)
    P = oracle.Params(dims=dims, m=0.2, g=0.4)
    phi = synth.scalar_field(dims, 0.5, 4)
    psi = synth.spinor_rhs(2, dims, 5)
    lat = wz.Lattice(dims, m=P.m, g=P.g)
    lat.set_phi(phi)  # host pointer
    out = np.empty_like(psi)
    lat.apply("MdagM", psi, out)  # host in, host out
    assert rel(out, oracle_apply("MdagM", P, phi, psi)) < TOL64
    x = torch.from_numpy(psi).cuda()
    lat.apply("M", x, x)  # in place
    torch.cuda.synchronize()
    assert rel(x.cpu().numpy(), oracle_apply("M", P, phi, psi)) < TOL64


def test_empty_batch_is_noop(wz):
    lat = wz.Lattice((4, 4, 4, 4))
    x = torch.zeros(1, dtype=torch.complex128, device="cuda")
    lat.apply("M", x, x, 0)


@pytest.mark.parametrize("dims", [(32, 32, 32, 32), (32, 16, 16, 16), (64, 32, 32, 32)])
@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_apply_L32(wz, dims, dt):
    """32-point lines (the 32^4 workload and the L = 32 apply sweep) and the
    paper's largest lattice 32^3 x 64 (64-point time lines)."""
    P = oracle.Params(dims=dims, m=0.02, g=1.0)
    phi = synth.scalar_field(dims, 1.0, 0)
    psi = synth.spinor_rhs(1, dims, 1)
    lat = wz.Lattice(dims, m=P.m, g=P.g)
    lat.set_phi(torch.from_numpy(phi).cuda())
    tdt = torch.complex128 if dt == "c128" else torch.complex64
    x = torch.from_numpy(psi).to(tdt).cuda()
    y = torch.empty_like(x)
    lat.apply("MdagM", x, y, 1)
    torch.cuda.synchronize()
    ref = oracle_apply("MdagM", P, phi, x.cpu().numpy().astype(np.complex128))
    assert rel(y.cpu().numpy().astype(np.complex128), ref) < (TOL64 if dt == "c128" else TOL32)


def test_full_size_sampled(wz):
    """16^4 with 12 right-hand sides (the precision workload), FP32 and FP64:
    two sampled right-hand sides checked in full against the oracle."""
    w = synth.PRECISION_16
    P = oracle.Params(dims=w.dims, m=w.m, g=w.g)
    phi = synth.scalar_field(w.dims, w.sigma, 0)
    psi = synth.spinor_rhs(w.nrhs, w.dims, 1)
    lat = wz.Lattice(w.dims, m=w.m, g=w.g)
    lat.set_phi(torch.from_numpy(phi).cuda())
    for dt, tol in ((torch.complex128, TOL64), (torch.complex64, TOL32)):
        x = torch.from_numpy(psi).to(dt).cuda()
        y = torch.empty_like(x)
        lat.apply("MdagM", x, y, w.nrhs)
        torch.cuda.synchronize()
        for k in (0, w.nrhs - 1):
            src = x[k].cpu().numpy().astype(np.complex128)
            ref = fftops.apply_MdagM(P, phi, src)
            assert rel(y[k].cpu().numpy().astype(np.complex128), ref) < tol
