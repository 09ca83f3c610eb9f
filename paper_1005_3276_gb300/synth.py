"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke run.

This module holds random-number generation and workload descriptions only; it
contains none of the method's arithmetic.  The paper's simulations use random
Gaussian scalar fields and Gaussian right-hand sides (Secs. 7.3, 7.4); the
workloads below reproduce those shapes on L^4 lattices.

Conventions: a "sigma" Gaussian complex field has Re and Im each N(0, sigma^2);
right-hand sides have Re and Im each N(0, 1).  Draws use
``numpy.random.default_rng(seed)`` in C order with (re, im) interleaved.
"""

from dataclasses import dataclass, field

import numpy as np


def complex_gaussian(shape, sigma, seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(size=tuple(shape) + (2,)) * sigma
    return np.ascontiguousarray(v[..., 0] + 1j * v[..., 1])


def scalar_field(dims, sigma=0.5, seed=0):
    """Complex scalar phi of shape (T, Z, Y, X)."""
    return complex_gaussian(dims, sigma, seed)


def spinor_rhs(nrhs, dims, seed=1):
    """nrhs spinor fields of shape (nrhs, T, Z, Y, X, 4)."""
    return complex_gaussian((nrhs,) + tuple(dims) + (4,), 1.0, seed)


@dataclass
class Workload:
    name: str
    dims: tuple
    m: float
    g: float
    sigma: float
    nrhs: int
    tol: float = 1e-10
    r: float = 1.0
    M0: float = 1.0
    extra: dict = field(default_factory=dict)


# Plain method: 4^4, m = 0.1, g = 0.1, sigma 0.5, 4 RHS, 10 trajectories.
SMALL_4 = Workload("wz-4^4-m0.1-g0.1", (4, 4, 4, 4), 0.1, 0.1, 0.5, 4,
                   extra={"tau": 1.0, "nsteps": 10, "ntraj": 10})
# Precision: 16^4, m = 0.05, g = 0.3, sigma 0.5, 12 RHS to 1e-10 true residual.
PRECISION_16 = Workload("wz-16^4-m0.05-g0.3-12rhs", (16, 16, 16, 16), 0.05, 0.3, 0.5, 12)
# Differentiation: 16^4, m = 0.1, g = 0.5, one pseudofermion, 20 leapfrog steps.
FORCE_16 = Workload("wz-16^4-m0.1-g0.5-hmc", (16, 16, 16, 16), 0.1, 0.5, 0.5, 1,
                    extra={"tau": 1.0, "nsteps": 20, "ntraj": 50})
# Large single lattice: 32^4, m = 0.02, g = 1.0, hot start sigma 1.0.
LARGE_32 = Workload("wz-32^4-m0.02-g1.0", (32, 32, 32, 32), 0.02, 1.0, 1.0, 4,
                    extra={"tau": 1.0, "nsteps": 40, "integrator": "omelyan"})


def batch_workloads(sizes=(4, 8, 12, 16), per_size=16, nrhs=8):
    """64 independent lattices (16 of each size), (m, g) on an 8 x 8 grid.

    m in linspace(0.02, 0.2, 8), g in linspace(0.1, 1.0, 8); lattice j takes
    grid point j and size sizes[j % len(sizes)] (round-robin).
    """
    ms = np.linspace(0.02, 0.2, 8)
    gs = np.linspace(0.1, 1.0, 8)
    out = []
    n = per_size * len(sizes)
    for j in range(n):
        L = sizes[j % len(sizes)]
        out.append(Workload(f"batch-{j}-{L}^4", (L, L, L, L), float(ms[j // 8 % 8]),
                            float(gs[j % 8]), 0.5, nrhs))
    return out
