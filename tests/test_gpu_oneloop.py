"""One-loop lattice sums on the GPU against the oracle (Sec. 5)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oneloop  # noqa: E402


@pytest.fixture(scope="module")
def wz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1005_3276_gb300 import binding
    return binding


@pytest.mark.parametrize("N,ma", [(4, 2.0), (8, 0.5), (16, 0.5), (12, 1.0 / 3.0), (32, 0.25), (64, 0.125)])
def test_one_loop_matches_oracle(wz, N, ma):
    z = wz.wz_one_loop(N, ma)
    ref = oneloop.sums(N, ma)
    np.testing.assert_allclose(z, ref, rtol=1e-11, atol=1e-14)


def test_one_loop_rejects_bad_sizes(wz):
    for N, ma in ((7, 0.5), (2, 0.5), (8, 0.0), (8192, 0.5)):
        with pytest.raises(wz.WzError):
            wz.wz_one_loop(N, ma)
