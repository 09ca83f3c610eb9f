"""Failure paths on the GPU that neither fault nor hang it.

A bounded device wait is made to run out on a barrier that nothing completes
(no copy is issued), and the status comes back as WZ_ETIMEOUT; the device keeps
working afterwards.
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


def test_bounded_wait_runs_out_with_status(wz):
    polls = 1024
    status, cycles = wz.wz_selftest_wait_timeout(polls)
    assert status == wz.WZ_ETIMEOUT
    assert cycles > 0
    per_poll = cycles / polls
    # the staged passes give up after 2^20 polls
    print(f"mbarrier.try_wait: {per_poll:.0f} cycles per failed poll; 2^20 polls = "
          f"{per_poll * (1 << 20) / 2.07e9:.3f} s at 2.07 GHz")
    with pytest.raises(wz.WzError):
        wz.wz_selftest_wait_timeout(0)
    dims = (4, 4, 4, 4)
    lat = wz.Lattice(dims, m=0.3, g=0.4)
    lat.set_phi(synth.scalar_field(dims, 0.5, 1))
    x = np.zeros((2,) + dims + (4,), np.complex128)
    rc, st, _ = lat.solve(synth.spinor_rhs(2, dims, 2), x, tol=1e-10)
    assert rc == wz.WZ_OK and st["converged"] == 2
    lat.close()
