"""Batches of lattices of uneven extent and coupling against single-lattice runs.

A lattice in a batch runs the same per-right-hand-side recursion and the same
Philox draws (key seed + lattice index) as the same lattice alone, so the
batched solutions and trajectories must equal the single-lattice ones; the
oracle recomputes the true residuals.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import cg as ocg  # noqa: E402
from paper_1005_3276_gb300 import synth  # noqa: E402

TOL = 1e-10


@pytest.fixture(scope="module")
def wz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1005_3276_gb300 import binding
    return binding


LATS = [dict(dims=(4, 4, 4, 4), m=0.1, g=0.3), dict(dims=(8, 8, 8, 8), m=0.2, g=0.5),
        dict(dims=(4, 4, 4, 4), m=0.05, g=0.8), dict(dims=(12, 12, 12, 12), m=0.15, g=0.2),
        dict(dims=(8, 8, 8, 8), m=0.08, g=1.0), dict(dims=(16, 16, 16, 16), m=0.1, g=0.6)]


def test_batch_solve_matches_single(wz):
    bt = wz.Batch(LATS)
    assert bt.groups == 4
    nrhs = 2
    phis = [synth.scalar_field(l["dims"], 0.5, 10 + i) for i, l in enumerate(LATS)]
    bs = [torch.from_numpy(synth.spinor_rhs(nrhs, l["dims"], 20 + i)).cuda() for i, l in enumerate(LATS)]
    xs = [torch.zeros_like(b) for b in bs]
    for i, p in enumerate(phis):
        bt.set_phi(i, p)
    st = bt.solve(bs, xs, nrhs, tol=TOL)
    assert st["converged"] == nrhs * len(LATS)
    for i, l in enumerate(LATS):
        P = oracle.Params(dims=l["dims"], m=l["m"], g=l["g"])
        xi = xs[i].cpu().numpy()
        bi = bs[i].cpu().numpy()
        assert max(ocg.true_residual(P, phis[i], bi[k], xi[k]) for k in range(nrhs)) <= TOL
        lat = wz.Lattice(l["dims"], m=l["m"], g=l["g"])
        lat.set_phi(phis[i])
        xr = torch.zeros_like(bs[i])
        lat.solve(bs[i], xr, tol=TOL)
        assert float((xr - xs[i]).abs().max() / xr.abs().max()) <= 1e-14


def test_batch_trajectory_matches_single(wz):
    bt = wz.Batch(LATS)
    phis = [synth.scalar_field(l["dims"], 0.5, 30 + i) for i, l in enumerate(LATS)]
    for i, p in enumerate(phis):
        bt.set_phi(i, p)
    kw = dict(tau=0.5, nsteps=4, npf=2, tol=1e-10, seed=77, traj_index=3)
    sts = bt.trajectory(**kw)
    for i, l in enumerate(LATS):
        lat = wz.Lattice(l["dims"], m=l["m"], g=l["g"])
        lat.set_phi(phis[i])
        ref = lat.trajectory(**dict(kw, seed=77 + i))
        assert abs(sts[i]["dH"] - ref["dH"]) <= 1e-9 * max(1.0, abs(ref["dH"]))
        assert sts[i]["accept"] == ref["accept"]
        a = np.zeros(l["dims"], np.complex128)
        b = np.zeros(l["dims"], np.complex128)
        bt.get_phi(i, a)
        lat.get_phi(b)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_batch_64_lattice_workload(wz):
    """The 64-lattice batching workload as the benchmark runs it: 16 each of
    4^4, 8^4, 12^4 and 16^4, (m, g) on the 8 x 8 grid, 8 right-hand sides each,
    one mixed solve to 1e-10.  The oracle recomputes the true residual of every
    one of the 512 returned solutions."""
    ws = synth.batch_workloads()
    bt = wz.Batch([dict(dims=x.dims, m=x.m, g=x.g) for x in ws])
    assert bt.groups == 4
    phis, bs, xs = [], [], []
    for i, x in enumerate(ws):
        phis.append(synth.scalar_field(x.dims, x.sigma, 100 + i))
        bt.set_phi(i, phis[-1])
        bs.append(torch.from_numpy(synth.spinor_rhs(x.nrhs, x.dims, 200 + i)).cuda())
        xs.append(torch.zeros_like(bs[-1]))
    st = bt.solve(bs, xs, ws[0].nrhs, tol=TOL)
    assert st["converged"] == 512 and st["max_true_residual"] <= TOL
    # site-weighted work: between the smallest and the largest lattice's share
    n = st["total_iterations"] + st["reliable_updates"]
    assert 4 ** 4 * n < st["site_applies"] < 16 ** 4 * n
    worst = 0.0
    for i, x in enumerate(ws):
        P = oracle.Params(dims=x.dims, m=x.m, g=x.g)
        xi, bi = xs[i].cpu().numpy(), bs[i].cpu().numpy()
        worst = max(worst, max(ocg.true_residual(P, phis[i], bi[k], xi[k]) for k in range(x.nrhs)))
    print("64-lattice batch: worst oracle true residual", worst)
    assert worst <= TOL
