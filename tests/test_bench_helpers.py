"""Host-side arithmetic of bench.py (no GPU): the nominal flop count and the
bulge chase's two rooflines."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_nominal_flops():
    n, m = 10000, 10000
    assert bench.nominal_flops(n, m) == pytest.approx(32.0 / 3.0 * n ** 3 + 12.0 * n * n * m)
    assert bench.nominal_flops(10000, 10000) == pytest.approx(2.267e13, rel=1e-3)


def test_chase_roofline():
    r = bench.chase_roofline({"ms": 500.0, "bytes": 1e9, "flops": 2e11}, 8000.0, 1.0)
    assert r["hbm_gbs"] == pytest.approx(2.0) and r["hbm_frac"] == pytest.approx(2.0 / 8000.0)
    assert r["fp64_tflops"] == pytest.approx(0.4) and r["dfma_frac"] == pytest.approx(0.4)
    assert bench.chase_roofline(None, 8000.0, 1.0) is None
    assert bench.chase_roofline({"ms": 0.0, "bytes": 1.0, "flops": 1.0}, 8000.0, 1.0) is None
    r = bench.chase_roofline({"ms": 1.0, "bytes": 1e6, "flops": 0.0}, None, None)
    assert r["hbm_frac"] is None and r["dfma_frac"] is None
