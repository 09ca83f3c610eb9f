"""GPU conjugate-gradient solves of (M^dagger M + shift) x = b checked by the oracle.

The pass criterion is the one of the precision workload: the FP64 true
relative residual ||b - A x|| / ||b||, recomputed here by the oracle from the
returned x, is at most tol = 1e-10.  On 4^4 the solution is also compared with
a dense LU solve; the allowed error is cond(A) * 1e-10 (the forward error of a
solution whose backward error is 1e-10), with cond(A) from the dense matrix.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import cg as ocg, dense, fftops  # noqa: E402
from paper_1005_3276_gb300 import synth  # noqa: E402

TOL = 1e-10


@pytest.fixture(scope="module")
def wz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1005_3276_gb300 import binding
    return binding


def oracle_residual(P, phi, b, x, shift=0.0):
    return max(ocg.true_residual(P, phi, b[k], x[k], shift) for k in range(len(b)))


@pytest.fixture(scope="module")
def small():
    w = synth.SMALL_4
    P = oracle.Params(dims=w.dims, m=w.m, g=w.g)
    phi = synth.scalar_field(w.dims, w.sigma, 0)
    b = synth.spinor_rhs(w.nrhs, w.dims, 1)
    M = dense.build_M(P, phi)
    A = M.conj().T @ M
    ev = np.linalg.eigvalsh(A)
    xref = np.linalg.solve(A, b.reshape(w.nrhs, -1).T).T.reshape(b.shape)
    return w, P, phi, b, xref, ev.max() / ev.min()


@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("pc", [False, True])
def test_solve_4x4_matches_dense_lu(wz, small, mixed, pc):
    w, P, phi, b, xref, cond = small
    lat = wz.Lattice(w.dims, m=w.m, g=w.g)
    lat.set_phi(torch.from_numpy(phi).cuda())
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    rc, st, res = lat.solve(bd, x, tol=TOL, mixed=mixed, pc=pc, resid=True)
    xs = x.cpu().numpy()
    assert st["converged"] == w.nrhs
    assert oracle_residual(P, phi, b, xs) <= TOL
    assert st["max_true_residual"] <= TOL
    assert max(res) <= TOL
    err = np.abs(xs - xref).max() / np.abs(xref).max()
    assert err <= cond * TOL
    if mixed:
        assert st["reliable_updates"] >= w.nrhs


def test_solve_with_shift(wz, small):
    w, P, phi, b, _, _ = small
    lat = wz.Lattice(w.dims, m=w.m, g=w.g)
    lat.set_phi(phi)
    x = np.zeros_like(b)
    rc, st, _ = lat.solve(b, x, shift=0.5, tol=TOL)  # host buffers
    assert oracle_residual(P, phi, b, x, 0.5) <= TOL


def test_solve_is_deterministic(wz, small):
    w, P, phi, b, _, _ = small
    lat = wz.Lattice(w.dims, m=w.m, g=w.g)
    lat.set_phi(phi)
    bd = torch.from_numpy(b).cuda()
    x1, x2 = torch.zeros_like(bd), torch.zeros_like(bd)
    lat.solve(bd, x1, tol=TOL)
    lat.solve(bd, x2, tol=TOL)
    assert torch.equal(x1, x2)


def test_not_converged_and_zero_rhs(wz, small):
    w, P, phi, b, _, _ = small
    lat = wz.Lattice(w.dims, m=w.m, g=w.g)
    lat.set_phi(phi)
    x = np.zeros_like(b)
    rc, st, _ = lat.solve(b, x, tol=TOL, maxiter=2, raise_on_nonconvergence=False)
    assert rc == wz.WZ_NOT_CONVERGED and st["converged"] == 0
    with pytest.raises(wz.WzError):
        lat.solve(b, x, tol=TOL, maxiter=2)
    z = np.zeros_like(b)
    rc, st, _ = lat.solve(z, x, tol=TOL)
    assert rc == wz.WZ_OK and np.all(x == 0) and st["converged"] == w.nrhs


@pytest.mark.parametrize("dims", [(12, 12, 12, 12), (32, 8, 8, 8), (32, 32, 32, 32)])
def test_solve_other_shapes(wz, dims):
    P = oracle.Params(dims=dims, m=0.1, g=0.3)
    phi = synth.scalar_field(dims, 0.5, 7)
    b = synth.spinor_rhs(2, dims, 8)
    lat = wz.Lattice(dims, m=P.m, g=P.g)
    lat.set_phi(phi)
    x = np.zeros_like(b)
    lat.solve(b, x, tol=TOL, mixed=True, pc=True)
    assert oracle_residual(P, phi, b, x) <= TOL


@pytest.mark.parametrize("pc", [False, True])
def test_solve_paper_lattice_32x64(wz, pc):
    """The paper's largest lattice, 32^3 x 64, at its solver-table couplings
    (m = 1, g = 0.2): mixed solve to 1e-10, residual recomputed by the oracle."""
    dims = (64, 32, 32, 32)
    P = oracle.Params(dims=dims, m=1.0, g=0.2)
    phi = synth.scalar_field(dims, 0.5, 0)
    b = synth.spinor_rhs(1, dims, 1)
    lat = wz.Lattice(dims, m=P.m, g=P.g)
    lat.set_phi(phi)
    x = np.zeros_like(b)
    rc, st, _ = lat.solve(b, x, tol=TOL, mixed=True, pc=pc)
    print("32^3 x 64", "PC" if pc else "no PC", st["iterations"], "iterations")
    assert oracle_residual(P, phi, b, x) <= TOL


@pytest.mark.parametrize("mixed", [True, False])
def test_precision_workload_16(wz, mixed):
    """16^4, m = 0.05, g = 0.3, 12 RHS to 1e-10 true residual (FP64 and mixed);
    the oracle recomputes the residual of two sampled right-hand sides."""
    w = synth.PRECISION_16
    P = oracle.Params(dims=w.dims, m=w.m, g=w.g)
    phi = synth.scalar_field(w.dims, w.sigma, 0)
    b = synth.spinor_rhs(w.nrhs, w.dims, 1)
    lat = wz.Lattice(w.dims, m=w.m, g=w.g)
    lat.set_phi(torch.from_numpy(phi).cuda())
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    rc, st, res = lat.solve(bd, x, tol=TOL, mixed=mixed, resid=True)
    assert st["converged"] == w.nrhs and max(res) <= TOL
    xs = x.cpu().numpy()
    for k in (0, w.nrhs - 1):
        assert ocg.true_residual(P, phi, b[k], xs[k]) <= TOL
    print(f"16^4 mixed={mixed}: {st}")


def test_workspace_reuse_across_precisions(wz, small):
    """A mixed solve after an FP64 solve on the same context reuses the
    workspace with another layout; nothing of the old contents may leak in."""
    w, P, phi, b, _, _ = small
    lat = wz.Lattice(w.dims, m=w.m, g=w.g)
    lat.set_phi(phi)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    for mixed in (False, True, False, True):
        lat.solve(bd, x, tol=TOL, mixed=mixed)
        assert oracle_residual(P, phi, b, x.cpu().numpy()) <= TOL


def test_graph_and_eager_launches_agree(wz, small, monkeypatch):
    """The cached CUDA-graph solve and the eagerly launched solve run the same
    kernels in the same order: the solutions are bitwise equal."""
    w, P, phi, b, _, _ = small
    bd = torch.from_numpy(b).cuda()
    xs = []
    for flag in ("0", "1"):
        monkeypatch.setenv("WZ_NO_GRAPHS", flag)
        lat = wz.Lattice(w.dims, m=w.m, g=w.g)
        lat.set_phi(phi)
        x = torch.zeros_like(bd)
        rc, st, _ = lat.solve(bd, x, tol=TOL)
        rc, st2, _ = lat.solve(bd, x, tol=TOL)  # second solve replays the cached graph
        assert st2["total_iterations"] == st["total_iterations"]
        xs.append(x)
        lat.close()
    assert torch.equal(xs[0], xs[1])


@pytest.mark.parametrize("where", ["phi", "b"])
@pytest.mark.parametrize("mixed", [True, False])
def test_nonfinite_input_stops_with_status(wz, where, mixed):
    """Host-side fault injection: a NaN in phi or an Inf in b ends the solve at
    once with WZ_ENONFINITE (not after maxiter iterations, not as converged),
    and the context keeps working."""
    dims = (4, 4, 4, 4)
    lat = wz.Lattice(dims, m=0.3, g=0.4)
    phi = synth.scalar_field(dims, 0.5, 1)
    b = synth.spinor_rhs(2, dims, 2)
    if where == "phi":
        phi[1, 2, 3, 0] = np.nan
    else:
        b[1, 0, 1, 2, 3, 1] = np.inf
    lat.set_phi(phi)
    x = np.zeros_like(b)
    with pytest.raises(wz.WzError) as e:
        lat.solve(b, x, tol=1e-10, maxiter=100000, mixed=mixed)
    assert e.value.code == wz.WZ_ENONFINITE
    lat.set_phi(synth.scalar_field(dims, 0.5, 1))
    rc, st, _ = lat.solve(synth.spinor_rhs(2, dims, 2), x, tol=1e-10, mixed=mixed)
    assert rc == wz.WZ_OK and st["converged"] == 2
    lat.close()
