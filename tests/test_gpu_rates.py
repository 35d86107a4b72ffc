"""The FP64 issue-rate probe (hprqp_fp64_rate) gives a consistent roof on the GPU.

The FP64 peak that bench.py divides by is the probe's full-warp FP64 FMA rate; these checks
hold for any consistent measurement: the three FP64 operations issue at the same rate, a
half-active warp costs the same issue slot (so half the lane rate), FP32 runs far faster, and
the SM clock derived from clock64 lies within the device's range.
"""
import pytest

pytestmark = pytest.mark.gpu


def test_fp64_rate_is_consistent():
    import paper_2507_02470_gb300 as pkg

    pkg.build()
    fma = pkg.fp64_rate(0, 32)
    add = pkg.fp64_rate(1, 32)
    mul = pkg.fp64_rate(2, 32)
    half = pkg.fp64_rate(0, 16)
    f32 = pkg.fp64_rate(3, 32)
    r = fma["lanes_per_clk"]
    assert 0.25 <= r <= 64.0, fma
    for o in (add, mul):
        assert abs(o["lanes_per_clk"] - r) <= 0.25 * r, (fma, o)
    # issue-bound: a warp with half its lanes active takes the same slot
    assert half["lanes_per_clk"] <= 0.75 * r, (fma, half)
    assert f32["lanes_per_clk"] >= 4.0 * r, (fma, f32)
    assert 300.0 <= fma["sm_mhz"] <= 2500.0, fma


def test_fp64_rate_rejects_bad_arguments():
    import ctypes as C

    import paper_2507_02470_gb300 as pkg

    pkg.build()
    v = C.c_double()
    assert pkg.lib().hprqp_fp64_rate(7, 32, C.byref(v), None, None) == 4
    assert pkg.lib().hprqp_fp64_rate(0, 0, C.byref(v), None, None) == 4
    assert pkg.lib().hprqp_fp64_rate(0, 33, C.byref(v), None, None) == 4
