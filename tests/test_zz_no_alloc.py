"""The allocation-free M^dagger M apply against the regular one.

wz_apply_mdagm_noalloc is for callers that cannot allocate device memory when
they apply the operator; it keeps the pass intermediates in a fixed device
array instead of the context workspace.  Two calls in a row (different
inputs, both precisions) and one in place must give what wz_apply gives,
within the apply tolerances used everywhere else (1e-12 FP64, 2e-6 FP32
relative); requests larger than the array must be refused with a message.
This file is collected last so that a stop-at-first-failure run has run every
other test first.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1005_3276_gb300 import synth  # noqa: E402

TOL = {torch.complex128: 1e-12, torch.complex64: 2e-6}


@pytest.fixture(scope="module")
def wz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1005_3276_gb300 import binding
    return binding


def rel(a, b):
    a = a.to(torch.complex128)
    b = b.to(torch.complex128)
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_noalloc_matches_apply_two_calls(wz, dtype):
    dims = (16, 16, 16, 16)
    lat = wz.Lattice(dims, m=0.05, g=0.3)
    lat.set_phi(torch.from_numpy(synth.scalar_field(dims, 0.5, 0)).cuda())
    for call, seed in enumerate((11, 12)):
        x = torch.from_numpy(synth.spinor_rhs(2, dims, seed)).to(dtype).cuda()
        y_ref = torch.empty_like(x)
        y = torch.full_like(x, float("nan"))
        shift = 0.25 * call
        lat.apply("MdagM", x, y_ref, 2, shift)
        wz.wz_apply_mdagm_noalloc(lat.ctx, x, y, 2, shift)
        torch.cuda.synchronize()
        assert rel(y, y_ref) <= TOL[dtype], f"call {call}"
    # in place (input and output the same field), with a shift: the shift term
    # reads the input last, after the passes have written the output elsewhere
    y_ref = torch.empty_like(x)
    lat.apply("MdagM", x, y_ref, 2, 0.25)
    y = x.clone()
    wz.wz_apply_mdagm_noalloc(lat.ctx, y, y, 2, 0.25)
    torch.cuda.synchronize()
    assert rel(y, y_ref) <= TOL[dtype], "in place"


def test_noalloc_rejects_oversize(wz):
    dims = (16, 16, 16, 16)
    lat = wz.Lattice(dims, m=0.05, g=0.3)
    x = torch.zeros((8,) + dims + (4,), dtype=torch.complex128, device="cuda")
    with pytest.raises(wz.WzError) as e:
        wz.wz_apply_mdagm_noalloc(lat.ctx, x, x, 8, 0.0)
    assert e.value.code == wz.WZ_EINVAL and "scratch" in str(e.value)
    h = np.zeros((1,) + dims + (4,), dtype=np.complex128)
    with pytest.raises(wz.WzError):
        wz.wz_apply_mdagm_noalloc(lat.ctx, h, h, 1, 0.0)  # host pointers are refused
