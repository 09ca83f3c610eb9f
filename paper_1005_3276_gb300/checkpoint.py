"""Checkpoint and resume of an HMC chain.

The state of a chain between trajectories is the scalar field (FP64), the
lattice and action parameters, the Philox seed and the index of the next
trajectory: every random number of trajectory t (momenta, pseudofermion
sources, the accept uniform) is a counter-based draw keyed by (seed, t), so a
chain resumed from a checkpoint repeats the trajectories of the uninterrupted
chain bit for bit.  Optional trajectory settings (tau, nsteps, integrator, npf,
tol, ...) travel with it as JSON.  The file is a plain .npz (no pickles).
"""

import json

import numpy as np

from . import binding

FORMAT = "wz-hmc-checkpoint-1"


def save(path, lattice, seed, next_traj, settings=None):
    """Write the chain state of ``lattice`` (its current phi) to ``path`` (.npz)."""
    phi = np.zeros(lattice.dims, np.complex128)
    lattice.get_phi(phi)
    p = lattice.params
    meta = {
        "format": FORMAT,
        "dims": list(lattice.dims),
        "m": [p.m_re, p.m_im],
        "g": [p.g_re, p.g_im],
        "r": p.r,
        "M0": p.M0,
        "yukawa": p.yukawa,
        "seed": int(seed),
        "next_traj": int(next_traj),
        "settings": dict(settings or {}),
    }
    np.savez(path, phi=phi, meta=np.array(json.dumps(meta)))


def load(path):
    """(meta dict, phi) of a checkpoint written by ``save``."""
    with np.load(path, allow_pickle=False) as z:
        meta = json.loads(str(z["meta"]))
        phi = np.array(z["phi"])
    if meta.get("format") != FORMAT:
        raise ValueError(f"{path}: not a {FORMAT} file")
    if tuple(phi.shape) != tuple(meta["dims"]) or phi.dtype != np.complex128:
        raise ValueError(f"{path}: phi does not match the stored lattice")
    return meta, phi


def resume(path, stream=None):
    """A new Lattice holding the checkpoint's phi, with (seed, next_traj, settings)."""
    meta, phi = load(path)
    lat = binding.Lattice(meta["dims"], m=complex(*meta["m"]), g=complex(*meta["g"]), r=meta["r"], M0=meta["M0"],
                          yukawa=meta["yukawa"], stream=stream)
    lat.set_phi(phi)
    return lat, meta["seed"], meta["next_traj"], meta["settings"]
