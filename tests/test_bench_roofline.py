"""Roofline arithmetic of bench.py on made-up probe results (CPU only).

The probe times only the launches it has event pairs for and counts the bytes
of exactly those launches, so the achieved rate must equal the bytes of one
timed launch over its average time, and the dominant class must be the one
with the most time per solve once every launch is counted.
"""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_achieved_is_bytes_per_launch_over_avg_time():
    probes = {
        # 11808 launches, 8192 of them timed at 12.344 us each, 36.49 MB each
        "cg_p1_fp32": {"launches": 11808, "timed_launches": 8192, "total_ms": 8192 * 12.344e-3,
                       "bytes": 8192 * 36.49e6},
        # more launches, shorter each: more time per solve in total
        "zt_fp32": {"launches": 23616, "timed_launches": 23616, "total_ms": 23616 * 10.36e-3,
                    "bytes": 23616 * 12.9e6},
    }
    k = bench.kernel_table(probes)
    p1 = k["cg_p1_fp32"]
    assert p1["avg_launch_us"] == pytest.approx(12.344)
    assert p1["algorithmic_bytes_per_launch"] == pytest.approx(36.49e6)
    assert p1["achieved_GB_s"] == pytest.approx(36.49e6 / 12.344e-6 / 1e9)
    assert p1["ms_per_solve"] == pytest.approx(11808 * 12.344e-3)
    assert bench.dominant_class(k) == "zt_fp32"
    assert k["zt_fp32"]["achieved_GB_s"] / 6773.0 == pytest.approx(12.9e6 / 10.36e-6 / 1e9 / 6773.0)
    assert sum(x["share_of_probed_time"] for x in k.values()) == pytest.approx(1.0)


def test_class_without_timed_launches():
    k = bench.kernel_table({"ru_p1_fp64": {"launches": 5, "timed_launches": 0, "total_ms": 0.0, "bytes": 0.0},
                            "zt_fp32": {"launches": 2, "timed_launches": 2, "total_ms": 0.02, "bytes": 2e6}})
    assert k["ru_p1_fp64"]["achieved_GB_s"] is None
    assert bench.dominant_class(k) == "zt_fp32"


def test_solve_gflops_matches_the_paper_counting():
    """The paper's solver table: 8^3 x 32, single precision, 830 iterations in
    1.3 s at 14 Gflop/s, i.e. about 1340 flops per site and iteration; the
    bench's count (two M applies of two 4D FFTs of 4 spin components at
    5 N log2 N, plus the site terms) gives 1312 at V = 16384."""
    V = 8 ** 3 * 32
    assert bench.mdagm_flops_per_site(V) == pytest.approx(1312.0)
    assert bench.solve_gflops(830, V, 1.3) == pytest.approx(14.0, rel=0.03)
