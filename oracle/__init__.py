"""Plain FP64 CPU oracle for the lattice Wess-Zumino fermion-matrix hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its Python binding) never
imports, calls or links anything here, and nothing here imports the product.

What is computed (Chen, Dzienkowski, Giedt, "Lattice Wess-Zumino model with
Ginsparg-Wilson fermions"):

* ``conventions``  gamma matrices, chiral projectors, charge conjugation (Sec. 2.1).
* ``momentum``     closed-form overlap operator in momentum space: D1(p), D2(p),
                   Dslash(p) = (1 - D2/2)^-1 D1, the free preconditioner M0^-1
                   (Sec. 2.2, Eq. fmat, Eq. d1mom, Sec. 7.3).
* ``fftops``       M, M^dagger, M^dagger M applied through a 4D FFT with the
                   antiperiodic-time twist (Sec. 7.2, "FFT trick"); the scalar
                   operators D2 and K = 1 - D2/2 with periodic BC (Eq. acws).
* ``dense``        dense position-space builders of A, D1, D2, D, Dslash, M and
                   of the auxiliary-fermion block operator (Eqs. kisu, lata),
                   with (A^dagger A)^-1/2 by Hermitian eigendecomposition.
* ``cg``           plain conjugate gradient on M^dagger M + beta (Eq. yuier),
                   with and without the M0^-1 preconditioning (Eq. theprob).
* ``force``        bosonic action of Eq. acws and its gradient; pseudofermion
                   action eta^dagger (M^dagger M)^-1 eta and its gradient.
* ``rational``     minimax relative rational approximations of x^gamma (Remez
                   exchange in mpmath) and r(M^dagger M) eta by shifted solves
                   (Eqs. jkjk, hbeq, yuier); Zolotarev's x^-1/2 as a pin.
* ``hmc``          leapfrog / Omelyan molecular dynamics and the Metropolis step;
                   RHMC with rational action and heatbath.
* ``philox``       Philox4x32-10 counter-based generator (Salmon et al., SC'11)
                   and Box-Muller Gaussians, so that random draws made on the
                   device can be reproduced here bit for bit.

Every function is written from the paper's definitions; no blocking, fusion or
reordering beyond what the definition states.  Floating point is FP64
(complex128) throughout.
"""

from . import conventions, momentum, fftops, dense, cg, force, hmc, philox  # noqa: F401
from .conventions import Params  # noqa: F401
