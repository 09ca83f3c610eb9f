"""HMC on the device against exact results of the free theory (Sec. 7.2).

At g = 0 the fermion matrix does not depend on phi, so the pseudofermion force
vanishes and the chain samples the Gaussian bosonic action of Eq. lata,
2 phi^* D2 phi + |m|^2 phi^* K phi: <|phi(x)|^2> = (1/V) sum_p 1 / (2 D2(p) +
|m|^2 K(p)) on the periodic momenta, and <exp(-dH)> = 1 for any step size
(the area-preservation identity of the leapfrog).  Statistical checks with a
fixed seed, errors from 20 bins, 4 sigma.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1005_3276_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def wz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1005_3276_gb300 import binding
    return binding


def exact_phi2(dims, m):
    k = [2 * np.pi * np.arange(n) / n for n in dims]
    p = np.meshgrid(*k, indexing="ij")
    b = 1.0 - 2.0 * sum(np.sin(0.5 * q) ** 2 for q in p)
    om = np.sqrt(b * b + sum(np.sin(q) ** 2 for q in p))
    D2, K = 1.0 - b / om, 0.5 * (1.0 + b / om)
    return float(np.mean(1.0 / (2.0 * D2 + abs(m) ** 2 * K)))


def binned(x, nb=20):
    x = np.asarray(x)
    b = x[: len(x) // nb * nb].reshape(nb, -1).mean(axis=1)
    return float(x.mean()), float(b.std(ddof=1) / np.sqrt(nb))


@pytest.mark.parametrize("integrator,nsteps", [("leapfrog", 10), ("omelyan", 5)])
def test_free_scalar_two_point_and_exp_dH(wz, integrator, nsteps):
    dims = (4, 4, 4, 4)
    m = 0.6 + 0.2j
    lat = wz.Lattice(dims, m=m, g=0.0)
    lat.set_phi(synth.scalar_field(dims, 0.5, 0))
    phi = np.zeros(dims, np.complex128)
    q, edh, acc = [], [], 0
    ntherm, nmeas = 50, 600
    for t in range(ntherm + nmeas):
        st = lat.trajectory(tau=1.0, nsteps=nsteps, integrator=integrator, npf=1, tol=1e-10, seed=2024,
                            traj_index=t)
        if t >= ntherm:
            lat.get_phi(phi)
            q.append(float(np.mean(np.abs(phi) ** 2)))
            edh.append(float(np.exp(-st["dH"])))
            acc += st["accept"]
    lat.close()
    exact = exact_phi2(dims, m)
    mq, eq = binned(q)
    me, ee = binned(edh)
    print(f"{integrator}: <|phi|^2> = {mq:.4f} +- {eq:.4f} (exact {exact:.4f}), "
          f"<exp(-dH)> = {me:.4f} +- {ee:.4f}, acceptance {acc / nmeas:.2f}")
    assert acc / nmeas > 0.5
    assert abs(mq - exact) < 4.0 * eq + 1e-3 * exact
    assert abs(me - 1.0) < 4.0 * ee + 1e-3
