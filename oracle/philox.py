"""Philox4x32-10 counter-based generator and Box-Muller Gaussians.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Philox4x32-10 as published by Salmon, Moraes, Dror and Shaw, "Parallel random
numbers: as easy as 1, 2, 3" (SC'11): a 128-bit counter (c0, c1, c2, c3) and a
64-bit key (k0, k1); each of 10 rounds forms the two 32x32->64 bit products
M0*c0 and M1*c2 and outputs (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key
is bumped by the Weyl constants (W0, W1) between rounds.  Written here with
numpy uint64 arithmetic, vectorised over counters.

Mapping used by the HMC (the same rule is written independently on the device):

* key   = (seed mod 2^32, seed >> 32)
* counter = (site, draw, stream, trajectory)
* one call yields four words (w0, w1, w2, w3); the 53-bit integers
  n1 = (w0 << 21) | (w1 >> 11) and n2 = (w2 << 21) | (w3 >> 11) give the
  uniforms u = (n + 1) * 2^-53 in (0, 1], and Box-Muller gives
  z0 = sqrt(-2 ln u1) cos(2 pi u2), z1 = sqrt(-2 ln u1) sin(2 pi u2).
"""

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)

STREAM_MOMENTUM = 1
STREAM_PSEUDOFERMION = 2
STREAM_ACCEPT = 3


def philox4x32_10(ctr, key):
    """ctr: uint array (..., 4); key: uint array (..., 2). Returns uint32 (..., 4)."""
    c = [np.asarray(ctr[..., i], dtype=np.uint64) & MASK for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint64) & MASK
    k1 = np.asarray(key[..., 1], dtype=np.uint64) & MASK
    for rnd in range(10):
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c = [(hi1 ^ c[1] ^ k0) & MASK, lo1, (hi0 ^ c[3] ^ k1) & MASK, lo0]
        if rnd < 9:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
    return np.stack(c, axis=-1).astype(np.uint32)


def _key(seed, shape):
    seed = int(seed)
    key = np.empty(shape + (2,), dtype=np.uint64)
    key[..., 0] = seed & 0xFFFFFFFF
    key[..., 1] = (seed >> 32) & 0xFFFFFFFF
    return key


def _unit53(a, b):
    n = (a.astype(np.uint64) << np.uint64(21)) | (b.astype(np.uint64) >> np.uint64(11))
    return (n.astype(np.float64) + 1.0) * (2.0 ** -53)


def words(seed, site, draw, stream, traj):
    """Philox words for counters (site, draw, stream, traj) (broadcast)."""
    site, draw = np.broadcast_arrays(np.asarray(site), np.asarray(draw))
    ctr = np.empty(site.shape + (4,), dtype=np.uint64)
    ctr[..., 0] = site
    ctr[..., 1] = draw
    ctr[..., 2] = stream
    ctr[..., 3] = traj
    return philox4x32_10(ctr, _key(seed, site.shape))


def gaussian_pair(w):
    u1 = _unit53(w[..., 0], w[..., 1])
    u2 = _unit53(w[..., 2], w[..., 3])
    rho = np.sqrt(-2.0 * np.log(u1))
    return rho * np.cos(2.0 * np.pi * u2), rho * np.sin(2.0 * np.pi * u2)


def uniform(w):
    return _unit53(w[..., 0], w[..., 1])


def momentum_field(seed, traj, dims):
    """pi(x) with Re, Im each N(0, 1): one call per site, draw 0."""
    V = int(np.prod(dims))
    z0, z1 = gaussian_pair(words(seed, np.arange(V), 0, STREAM_MOMENTUM, traj))
    return (z0 + 1j * z1).reshape(dims)


def pseudofermion_source(seed, traj, dims, npf):
    """R_k(x) with density exp(-|R|^2): Re, Im each N(0, 1/2).

    Spinor component (k, x, s) uses draw = 4 k + s at counter site x.
    Returns shape (npf,) + dims + (4,).
    """
    V = int(np.prod(dims))
    site = np.arange(V)[None, :, None]
    draw = (4 * np.arange(npf)[:, None, None] + np.arange(4)[None, None, :])
    z0, z1 = gaussian_pair(words(seed, site, draw, STREAM_PSEUDOFERMION, traj))
    R = (z0 + 1j * z1) * np.sqrt(0.5)
    return R.reshape((npf,) + tuple(dims) + (4,))


def accept_uniform(seed, traj):
    return float(uniform(words(seed, np.array(0), 0, STREAM_ACCEPT, traj)))
