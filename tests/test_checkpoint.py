"""Checkpoint / resume of an HMC chain.

CPU: the file round trip (phi bit for bit, parameters, seed, next trajectory,
settings) and rejection of foreign files.  GPU: a chain resumed from a
checkpoint repeats the uninterrupted chain's trajectories bit for bit.
"""

import numpy as np
import pytest

from paper_1005_3276_gb300 import binding, checkpoint, synth


class FakeLattice:
    def __init__(self, dims, phi):
        self.dims = dims
        self.params = binding.make_params(dims, 0.3 - 0.1j, 0.5 + 0.2j, 1.0, 1.0, 2.0)
        self._phi = phi

    def get_phi(self, out):
        out[...] = self._phi


def test_round_trip(tmp_path):
    dims = (4, 4, 4, 4)
    phi = synth.scalar_field(dims, 0.7, 3)
    path = tmp_path / "chain.npz"
    settings = {"tau": 1.0, "nsteps": 10, "integrator": "omelyan", "npf": 2, "tol": 1e-10}
    checkpoint.save(path, FakeLattice(dims, phi), seed=41, next_traj=17, settings=settings)
    meta, phi2 = checkpoint.load(path)
    assert np.array_equal(phi2.view(np.uint64), phi.view(np.uint64))
    assert meta["dims"] == list(dims) and complex(*meta["m"]) == 0.3 - 0.1j and complex(*meta["g"]) == 0.5 + 0.2j
    assert (meta["seed"], meta["next_traj"], meta["settings"]) == (41, 17, settings)


def test_rejects_foreign_file(tmp_path):
    path = tmp_path / "other.npz"
    np.savez(path, phi=np.zeros((4, 4, 4, 4), np.complex128), meta=np.array('{"format": "something else"}'))
    with pytest.raises(ValueError):
        checkpoint.load(path)


@pytest.mark.gpu
def test_resumed_chain_repeats_the_uninterrupted_chain(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dims = (8, 8, 8, 8)
    kw = dict(tau=0.5, nsteps=6, npf=1, tol=1e-10)
    seed = 5
    ref = binding.Lattice(dims, m=0.4, g=0.5)
    ref.set_phi(synth.scalar_field(dims, 0.5, 0))
    ref_stats = [ref.trajectory(seed=seed, traj_index=t, **kw) for t in range(4)]
    ref_phi = np.zeros(dims, np.complex128)
    ref.get_phi(ref_phi)
    ref.close()

    a = binding.Lattice(dims, m=0.4, g=0.5)
    a.set_phi(synth.scalar_field(dims, 0.5, 0))
    stats = [a.trajectory(seed=seed, traj_index=t, **kw) for t in range(2)]
    path = tmp_path / "chain.npz"
    checkpoint.save(path, a, seed, 2, kw)
    a.close()
    b, seed2, t0, kw2 = checkpoint.resume(path)
    stats += [b.trajectory(seed=seed2, traj_index=t, **kw2) for t in range(t0, t0 + 2)]
    phi = np.zeros(dims, np.complex128)
    b.get_phi(phi)
    b.close()
    assert [(s["dH"], s["accept"], s["cg_iterations"]) for s in stats] == \
        [(s["dH"], s["accept"], s["cg_iterations"]) for s in ref_stats]
    assert np.array_equal(phi.view(np.uint64), ref_phi.view(np.uint64))
