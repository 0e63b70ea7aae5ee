"""Host-side arithmetic of bench.py (no GPU): the clip roofline from the
step counters."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _stage(fast, fp64, exact, nv, ms):
    return {"pred_fast": fast, "pred_fp64": fp64, "pred_exact": exact, "clip_vertices": nv, "ms_clip_kernels": ms}


def test_clip_roofline_counts_algorithmic_flop():
    # 1000 sign tests of which 60 are vertex orientations (10 + 20 + 30
    # constructed vertices), timed at 0.5 and 1.5 ms
    st = [_stage(990, 9, 1, [10, 20, 30], 0.5), _stage(990, 9, 1, [10, 20, 30], 1.5)]
    r = bench.clip_roofline(st, 152, "block_c2", "fp32")
    flop = 7 * (1000 - 60) + 17 * 10 + 26 * 20 + 73 * 30
    assert r["flop_per_launch"] == flop
    assert abs(r["ms_per_launch"] - 1.0) < 1e-12
    assert abs(r["achieved"] - flop / 1e-3 / 1e12) < 1e-15
    mhz = float(bench.measured_peaks().get("sm_max_mhz", 2070.0))
    assert abs(r["peak"] - 152 * 128 * 2 * mhz * 1e6 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-18
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["traffic"] == bench.CLIP_TRAFFIC_BYTES[("block_c2", "fp32")]
    assert bench.clip_roofline(st, 152, "torus_c1", "fp32")["traffic"] is None
