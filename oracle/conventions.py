"""Spinor conventions of Sec. 2.1 and the lattice parameter set.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Chiral basis of Sec. 2.1, with i = 1, 2, 3:

    gamma_0 = [[0, 1], [1, 0]],  gamma_i = [[0, i sigma_i], [-i sigma_i, 0]],
    gamma_5 = diag(-1, -1, 1, 1),  P_pm = (1 pm gamma_5) / 2,  C = gamma_0 gamma_2.

So P_- projects on spin components 0, 1 and P_+ on 2, 3.

Field layout used everywhere in the oracle (and by the tests that compare with
the device): a spinor field is a complex128 array of shape (T, Z, Y, X, 4), a
scalar field has shape (T, Z, Y, X).  Axis 0 is time, the direction with
antiperiodic fermion boundary conditions (Sec. 3.1, T even).  Direction index
mu = 0 is time and pairs with gamma_0; mu = 1, 2, 3 are x, y, z and pair with
gamma_1, gamma_2, gamma_3 (a fixed reading: the paper does not assign axes).
"""

from dataclasses import dataclass, field

import numpy as np

SIGMA = (
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
)

_Z2 = np.zeros((2, 2), dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)


def _block(a, b, c, d):
    return np.block([[a, b], [c, d]])


GAMMA = np.stack(
    [_block(_Z2, _I2, _I2, _Z2)]
    + [_block(_Z2, 1j * s, -1j * s, _Z2) for s in SIGMA]
)  # shape (4, 4, 4): GAMMA[mu] for mu = 0..3
GAMMA5 = np.diag([-1, -1, 1, 1]).astype(np.complex128)
P_PLUS = 0.5 * (np.eye(4) + GAMMA5)
P_MINUS = 0.5 * (np.eye(4) - GAMMA5)
CCONJ = GAMMA[0] @ GAMMA[2]

# array axis (in a (T, Z, Y, X) field) that direction mu runs along
MU_AXIS = (0, 3, 2, 1)


@dataclass
class Params:
    """Lattice and action parameters.

    dims    (T, Z, Y, X); T must be even (Sec. 3.1).
    m, g    bare mass and Yukawa coupling (complex allowed, Eq. fmat).
    r, M0   Wilson parameter and the constant in A = M0 - a D_W (Sec. 2.2 has
            r = M0 = 1; both are kept as parameters, defaults as in the paper).
    yukawa  coefficient c in the site term c g phi P_+ + c g^* phi^* P_-.
            Eq. fmat has c = 2; the simulation section (Sec. 7.1) writes g phi,
            i.e. c = 1.  Default 2.
    """

    dims: tuple
    m: complex = 0.1
    g: complex = 0.1
    r: float = 1.0
    M0: float = 1.0
    yukawa: float = 2.0
    extra: dict = field(default_factory=dict)

    @property
    def volume(self):
        T, Z, Y, X = self.dims
        return T * Z * Y * X

    def check(self):
        T = self.dims[0]
        if T % 2:
            raise ValueError("T must be even for antiperiodic fermions (Sec. 3.1)")
