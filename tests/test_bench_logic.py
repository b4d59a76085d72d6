"""Host logic of bench.py that needs no GPU: the roofline of the dominant kernel, the
measured-traffic lookup and the reference arm's line shape."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

PEAKS = {"sm_max_mhz": 2000.0, "bf16_tflops_sustained": 1600.0}


def _level(m, tiles_ms, t3_ms, nodes):
    return {"m": m, "grng": {"kernel_ms": {"tiles": tiles_ms, "tier3": t3_ms}, "tier3_nodes_tested": nodes}}


def _stats(rng_tiles, rng_t3, layers):
    return {"rng": {"kernel_ms": {"tiles": rng_tiles, "tier3": rng_t3}, "tier3_nodes_tested": 10}, "layers": layers}


def test_dominant_kernel_and_fractions():
    st = _stats(1000.0, 5.0, [_level(100, 1.0, 4000.0, 2_000_000_000)])
    r = bench.kernel_rooflines(st, n=10_000, D=96, precision="bf16", peaks=PEAKS, sms=100)
    assert r["kernel"] == "tier3_kernel (pivot layer m=100)" and r["bound"] == "alu"
    alu = 100 * 128 * 2000.0 / 1000.0  # Gop/s
    want = 2_000_000_000 * 2 * 2 * 96 / 4.0 / 1e9
    assert r["peak"] == pytest.approx(alu) and r["achieved"] == pytest.approx(want)
    assert r["frac"] == pytest.approx(want / alu)
    others = {o["kernel"]: o for o in r["others"]}
    tc = others["tc_sweep_kernel (exemplar Gram tiles, tcgen05 split-BF16)"]
    assert tc["unit"] == "TFLOP/s" and tc["frac"] == pytest.approx((10_000 * 9_999 / 2 * 2 * 96 / 1.0 / 1e12) / 1600.0)


def test_fp32_sweep_reports_lane_peak():
    st = _stats(1000.0, 1.0, [])
    r = bench.kernel_rooflines(st, n=1000, D=16, precision="fp32", peaks={}, sms=10)
    assert r["kernel"].startswith("tile_pass_kernel (exemplar") and r["unit"] == "Gop/s"
    assert r["peak"] == pytest.approx(10 * 128 * 2070.0 / 1000.0)  # default clock when the file has none


def test_measured_traffic_lookup():
    """roofline.traffic comes from the committed capture only for the same kernel, size and revision."""
    k = "tc_sweep_kernel (exemplar Gram tiles, tcgen05 split-BF16)"
    assert bench.measured_traffic(k, 1_000_000) == 3_119_250_631_168 + 12_933_911_040
    assert bench.measured_traffic(k, 999_999) is None                      # another size
    assert bench.measured_traffic("tier3_kernel (pivot layer m=131072)", 1_000_000) is None  # never captured
    saved = dict(bench.KERNEL_REVS)
    try:
        bench.KERNEL_REVS["tc_sweep_kernel"] = "changed"                  # the kernel changed since the capture
        assert bench.measured_traffic(k, 1_000_000) is None
    finally:
        bench.KERNEL_REVS.clear()
        bench.KERNEL_REVS.update(saved)
