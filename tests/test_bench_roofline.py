"""The roofline arithmetic of bench.py, recomputed by hand (no GPU).

The scope table's algorithmic counts for the cached sweep: per element-direction the inflow and
outflow traces, 2 d (p+1)^(d-1) float64 values (96 B for 2D Q2, 192 B for 3D Q1), per element the
scalar flux read and written plus three material values (168 B for Q2), and the reuse floor of
2 n^2 flops per element-direction (162 for Q2).  The line's frac is achieved / peak."""
import os
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
bench = pytest.importorskip("bench")


def test_algorithmic_counts():
    assert bench.trace_bytes_per_item(9, 2, 2) == 96
    assert bench.trace_bytes_per_item(8, 3, 1) == 192
    assert bench.element_bytes(9) == 168
    assert bench.element_bytes(8) == 152
    assert bench.reuse_floor_flops(9) == 162
    assert bench.flops_per_item(9) == pytest.approx((2 / 3) * 729 + 6 * 81)
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(152 * 2 * 2 * 2.07e9 / 1e12)


def test_sweep_roofline_config2_by_hand():
    mesh = SimpleNamespace(n_nodes=9, n_elem=256 * 256, n_dirs=40, n_levels=679)
    prob = SimpleNamespace(dim=2, p=2)
    sweep_ms = 2.2
    r = bench.sweep_roofline(mesh, prob, sweep_ms, ("static", 128, 4), 1, "c2")
    items = 256 * 256 * 40
    achieved = 162 * items / (sweep_ms / 1e3) / 1e12
    assert r["achieved"] == pytest.approx(achieved)
    assert r["frac"] == pytest.approx(achieved / bench.FP64_PEAK_TFLOPS)
    alg = 96 * items + 168 * 256 * 256
    assert r["hbm"]["algorithmic_bytes_per_sweep"] == alg
    assert r["hbm"]["achieved_gbs"] == pytest.approx(alg / (sweep_ms / 1e3) / 1e9)
    # the measured DRAM traffic of one launch: 878 B per element-direction
    assert r["traffic"] == pytest.approx(bench.SWEEP_DRAM_BYTES_PER_ITEM[("static", "c2")] * items)
    assert 860 < r["traffic"] / items < 880
    # a schedule without a capture reports no traffic
    assert bench.sweep_roofline(mesh, prob, sweep_ms, ("levels", 64, 2), 1358, "c2")["traffic"] is None
