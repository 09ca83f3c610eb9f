"""The library's host-side minimax (wz_rational_minimax, product-form Remez in
double precision) against the oracle's coefficient-form Remez in mpmath: the
stored cases of tests/golden/rational_coeffs.json (written by
tests/golden/make_rational.py from the oracle only) and live small cases.

The optimum is unique, so both must give the same function: their ratio is 1
within the sum of the two errors on the interval, the shifts agree where the
optimum is well determined, and the library's reported error is its measured
maximum.  No GPU is involved (the computation is host code of libwz.so).
"""

import json
import os

import numpy as np
import pytest

from oracle import rational

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def wz():
    from paper_1005_3276_gb300 import binding
    return binding


def golden():
    with open(os.path.join(HERE, "golden", "rational_coeffs.json")) as f:
        return json.load(f)


def compare(lib, orc, gamma, lo, hi, beta_rtol):
    x = np.exp(np.linspace(np.log(lo), np.log(hi), 50001))
    rl = rational.evaluate(lib, x)
    ro = rational.evaluate(orc, x)
    bound = lib["err"] + orc["err"]
    assert np.abs(rl / ro - 1).max() <= bound * 1.01 + 1e-14
    el = np.abs(rational.relative_error(lib, gamma, x)).max()
    assert el <= lib["err"] * (1 + 1e-4) + 1e-15
    # the optimum: no worse than the oracle's by more than a hair
    assert lib["err"] <= orc["err"] * 1.001 + 2e-14
    if beta_rtol is not None:
        np.testing.assert_allclose(lib["beta"], orc["beta"], rtol=beta_rtol)
        np.testing.assert_allclose(lib["alpha"], orc["alpha"], rtol=beta_rtol * 10)
        assert lib["a0"] == pytest.approx(orc["a0"], rel=beta_rtol * 10)


@pytest.mark.parametrize("name", ["L4_m0.5_d8", "L8_m0.5_d10", "L16_m0.1_d20"])
@pytest.mark.parametrize("kind", ["action", "heatbath"])
def test_library_minimax_matches_stored_oracle(wz, name, kind):
    case = golden()[name]
    orc = dict(case[kind])
    orc["alpha"], orc["beta"] = np.array(orc["alpha"]), np.array(orc["beta"])
    lib = wz.wz_rational_minimax(orc["gamma"], case["lo"], case["hi"], orc["d"]).as_dict()
    assert lib["d"] == orc["d"]
    compare(lib, orc, orc["gamma"], case["lo"], case["hi"], 1e-5 if orc["err"] > 1e-9 else None)


@pytest.mark.parametrize("gamma,lo,hi,d", [(-0.25, 1.0, 100.0, 0), (-0.5, 0.01, 100.0, 6), (0.125, 0.5, 3000.0, 5),
                                           (-0.25, 0.01, 100.0, 4)])
def test_library_minimax_matches_live_oracle(wz, gamma, lo, hi, d):
    pytest.importorskip("mpmath")
    orc = rational.minimax(gamma, lo, hi, d)
    lib = wz.wz_rational_minimax(gamma, lo, hi, d).as_dict()
    compare(lib, orc, gamma, lo, hi, 1e-6)


def test_minimax_rejects_bad_arguments(wz):
    for args in [(0.0, 1.0, 2.0, 4), (-0.25, 0.0, 2.0, 4), (-0.25, 2.0, 1.0, 4), (-0.25, 1.0, 2.0, 65),
                 (1.5, 1.0, 2.0, 4)]:
        with pytest.raises(wz.WzError):
            wz.wz_rational_minimax(*args)


def test_minimax_below_double_precision_widens_the_interval(wz):
    # the optimum of degree 20 on [1, 100] is far below 1e-15: the library
    # widens the interval until the exchange resolves and stays below 1e-13
    r = wz.wz_rational_minimax(-0.25, 1.0, 100.0, 20).as_dict()
    assert r["err"] < 1e-13
    assert r["build_lo"] <= 1.0 and r["build_hi"] >= 100.0
    x = np.exp(np.linspace(0, np.log(100.0), 20001))
    assert np.abs(rational.relative_error(r, -0.25, x)).max() < 1e-13
