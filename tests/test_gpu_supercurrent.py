"""Supercurrent correlators of Eq. sitre on the GPU against the oracle.

Every solve runs to FP64 true residual 1e-12 (the correlators are linear in the
solutions), so the device and oracle values agree to about cond * 1e-12;
compared at 1e-9 of the largest entry.  The 32^4 case (the large-lattice size,
16 chunks per time slice) uses a constant scalar, for which the
correlator has a closed form through the zero-momentum free propagator.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import supercurrent  # noqa: E402
from oracle.conventions import GAMMA, P_MINUS, P_PLUS  # noqa: E402
from paper_1005_3276_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def wz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1005_3276_gb300 import binding
    return binding


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def point(dims, z0):
    w = np.zeros(dims, np.complex128)
    w[z0] = 1.0
    return w


@pytest.mark.parametrize("dims,src", [((4, 4, 4, 4), "point"), ((16, 8, 4, 4), "noise"), ((12, 12, 4, 4), "point"),
                                      ((8, 8, 8, 8), "wall")])
def test_supercurrent_matches_oracle(wz, dims, src):
    P = oracle.Params(dims=dims, m=1.0 + 0.1j, g=0.3 - 0.2j)
    phi = synth.scalar_field(dims, 0.4, 11)
    if src == "point":
        w = point(dims, (dims[0] - 1, 1, 2, 3))
    elif src == "noise":
        w = synth.scalar_field(dims, 1.0, 12)
    else:
        w = np.zeros(dims, np.complex128)
        w[1] = 1.0
    lat = wz.Lattice(dims, m=P.m, g=P.g)
    lat.set_phi(phi)
    wd = torch.from_numpy(w).cuda() if src != "point" else w  # device and host source paths
    R, st = lat.supercurrent(wd, tol=1e-12)
    assert st["converged"] == 4 and st["max_true_residual"] <= 1e-12 * 1.01
    ref = supercurrent.correlators(P, phi, w, tol=1e-13)
    assert rel(R, ref) <= 1e-9
    lat.close()


def test_supercurrent_mixed_precision(wz):
    dims = (8, 8, 8, 8)
    phi = synth.scalar_field(dims, 0.5, 13)
    w = synth.scalar_field(dims, 1.0, 14)
    lat = wz.Lattice(dims, m=0.3, g=0.5)
    lat.set_phi(phi)
    R64, _ = lat.supercurrent(w, tol=1e-11)
    R32, st = lat.supercurrent(w, tol=1e-11, mixed=True)
    assert st["converged"] == 4 and st["reliable_updates"] > 0
    assert rel(R32, R64) <= 1e-8
    lat.close()


def test_supercurrent_constant_scalar_32(wz):
    dims = (32, 32, 32, 32)
    T, V3 = dims[0], 32 ** 3
    m, g, c = 0.02, 1.0, 0.2 + 0.05j
    z0 = (30, 5, 17, 9)
    lat = wz.Lattice(dims, m=m, g=g)
    lat.set_phi(np.full(dims, c, np.complex128))
    R, st = lat.supercurrent(torch.from_numpy(point(dims, z0)).cuda(), tol=1e-11, mixed=True)
    assert st["converged"] == 4
    # sum_xvec S(t, xvec) = -(1/T) sum_pt e^{i pt (t - t0)} M^-1(pvec = 0, pt), antiperiodic pt
    meff = m + 2.0 * g * c
    pt = (2 * np.arange(T) + 1) * np.pi / T
    b = 1.0 - 2.0 * np.sin(0.5 * pt) ** 2
    om = np.sqrt(b * b + np.sin(pt) ** 2)
    Mp = (1j * 2.0 / (om + b) * np.sin(pt))[:, None, None] * GAMMA[0] + meff * P_PLUS + np.conj(meff) * P_MINUS
    Minv = np.linalg.inv(Mp)
    Wp = m * c + g * c * c
    ref = np.zeros_like(R)
    for dx in range(T):
        sgn = -1.0 if z0[0] + dx >= T else 1.0
        tx = (z0[0] + dx) % T
        # the propagator at the lattice time tx of the sink; sgn undoes the antiperiodic wrap
        Ssum = -np.einsum("p,pab->ab", np.exp(1j * pt * (tx - z0[0])), Minv) / T
        for mu in range(4):
            Gam = np.sqrt(2.0) * (Wp * GAMMA[mu] @ P_MINUS + np.conj(Wp) * GAMMA[mu] @ P_PLUS)
            for s, Phi in enumerate((V3 * c, V3 * np.conj(c))):
                ref[s, mu, dx, :] = sgn * Phi * (Gam @ Ssum)
    assert rel(R, ref) <= 1e-8
    lat.close()


def test_supercurrent_rejects_bad_arguments(wz):
    dims = (4, 4, 4, 4)
    lat = wz.Lattice(dims, m=0.5, g=0.3)
    lat.set_phi(synth.scalar_field(dims, 0.5, 1))
    with pytest.raises(wz.WzError):
        lat.supercurrent(point(dims, (0, 0, 0, 0)), tol=0.0)
    lat.close()
