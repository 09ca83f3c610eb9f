"""The seeded synthetic workloads (CPU): shapes, seeds and the batching recipe.

The batching workload is 64 independent lattices, 16 each of 4^4, 8^4, 12^4
and 16^4 assigned round robin, with (m, g) on the 8 x 8 grid m in
linspace(0.02, 0.2, 8), g in linspace(0.1, 1.0, 8) and 8 right-hand sides each;
the generators are seeded, so the same call gives the same fields.
"""

import numpy as np

from paper_1005_3276_gb300 import synth


def test_batch_recipe():
    ws = synth.batch_workloads()
    assert len(ws) == 64
    sizes = [w.dims[0] for w in ws]
    assert all(w.dims == (w.dims[0],) * 4 for w in ws)
    assert sizes[:4] == [4, 8, 12, 16] and all(sizes.count(L) == 16 for L in (4, 8, 12, 16))
    grid = {(round(w.m, 12), round(w.g, 12)) for w in ws}
    want = {(round(m, 12), round(g, 12)) for m in np.linspace(0.02, 0.2, 8) for g in np.linspace(0.1, 1.0, 8)}
    assert grid == want
    assert all(w.nrhs == 8 and w.tol == 1e-10 for w in ws)


def test_fields_are_seeded_and_shaped():
    dims = (4, 4, 4, 6)
    a = synth.scalar_field(dims, 0.5, 7)
    assert a.shape == dims and a.dtype == np.complex128
    assert np.array_equal(a, synth.scalar_field(dims, 0.5, 7))
    assert not np.array_equal(a, synth.scalar_field(dims, 0.5, 8))
    b = synth.spinor_rhs(3, dims, 1)
    assert b.shape == (3,) + dims + (4,)
    # Re and Im each N(0, sigma^2): the sample variance of a large draw
    z = synth.scalar_field((32, 32, 32, 32), 0.5, 0)
    assert abs(z.real.var() - 0.25) < 0.01 and abs(z.imag.var() - 0.25) < 0.01
