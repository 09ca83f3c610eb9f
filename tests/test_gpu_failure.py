"""Failure paths on the GPU that neither fault nor hang it.

A bounded device wait is made to run out on a barrier that nothing completes
(no copy is issued), and the status comes back as WZ_ETIMEOUT; the device keeps
working afterwards.  An out-of-memory workspace growth is made on the host: a
workspace cap below what a solve needs refuses the growth the way cudaMalloc
refuses one beyond free memory, the call returns WZ_ENOMEM, and the same
context then solves once the cap is lifted.
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


def test_workspace_growth_refused_with_enomem(wz):
    from oracle import cg as ocg
    import oracle
    dims = (8, 8, 8, 8)
    P = oracle.Params(dims=dims, m=0.2, g=0.5)
    phi = synth.scalar_field(dims, 0.5, 3)
    b = torch.from_numpy(synth.spinor_rhs(4, dims, 4)).cuda()
    x = torch.zeros_like(b)
    lat = wz.Lattice(dims, m=P.m, g=P.g)
    lat.set_phi(phi)
    # one right-hand side fits and leaves workspace behind
    lat.solve(b[:1].contiguous(), x[:1].contiguous(), tol=1e-10)
    held = lat.workspace_bytes()
    assert held > 0
    lat.set_workspace_limit(held)  # exactly what it holds: no room to grow
    with pytest.raises(wz.WzError) as e:
        lat.solve(b, x, tol=1e-10)
    assert e.value.code == wz.WZ_ENOMEM
    assert lat.workspace_bytes() == held  # the refused growth released nothing
    # a call that fits the existing workspace still runs under the cap
    x1 = torch.zeros_like(b[:1])
    rc, st, _ = lat.solve(b[:1].contiguous(), x1, tol=1e-10)
    assert rc == wz.WZ_OK
    lat.set_workspace_limit(0)
    rc, st, _ = lat.solve(b, x, tol=1e-10)
    assert rc == wz.WZ_OK and st["converged"] == 4
    xb, bb = x.cpu().numpy(), b.cpu().numpy()
    assert max(ocg.true_residual(P, phi, bb[k], xb[k]) for k in range(4)) <= 1e-10
    lat.close()


def test_fma_peak_microkernel(wz):
    """The FMA throughput microkernel that the FP64 roofline is reported
    against: finite, positive, and FP32 well above FP64 on this part."""
    f64, ms64 = wz.wz_fma_peak(8, 2000)
    f32, ms32 = wz.wz_fma_peak(4, 20000)
    print(f"FMA throughput: FP64 {f64:.2f} TFLOP/s, FP32 {f32:.1f} TFLOP/s")
    assert f64 > 0 and f32 > 0 and ms64 > 0 and ms32 > 0
    assert f32 > 4 * f64
    with pytest.raises(wz.WzError):
        wz.wz_fma_peak(2, 10)
