"""Host-side arithmetic of bench.py (no GPU): the clip roofline from the
step counters and the measured peaks."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _stage(fast, fp64, exact, nv, ms, pieces):
    return {"pred_fast": fast, "pred_fp64": fp64, "pred_exact": exact, "clip_vertices": nv, "ms_clip_kernels": ms,
            "n_pieces": pieces}


PEAKS = {"fp32": {"tflops": 80.0}, "fp64": {"tflops": 1.25}}


def test_clip_roofline_uses_the_planned_work_per_piece():
    # 1000 sign tests of which 60 are vertex orientations (10 + 20 + 30
    # constructed vertices), 400 pieces, timed at 0.5 and 1.5 ms
    st = [_stage(990, 9, 1, [10, 20, 30], 0.5, 400), _stage(990, 9, 1, [10, 20, 30], 1.5, 400)]
    r = bench.clip_roofline(st, 32, "block_c2", "fp32", PEAKS, 6700.0)
    assert r["flop_per_piece"] == 4500.0
    assert r["flop_per_launch"] == 4500.0 * 400
    assert abs(r["ms_per_launch"] - 1.0) < 1e-12
    assert abs(r["achieved"] - 4500.0 * 400 / 1e-3 / 1e12) < 1e-15
    assert r["peak"] == 80.0 and abs(r["frac"] - r["achieved"] / 80.0) < 1e-18
    executed = 7 * (1000 - 60) + 17 * 10 + 26 * 20 + 73 * 30
    assert r["flop_executed_per_launch"] == executed
    assert abs(r["fractions"]["fp32_executed"] - executed / 1e-3 / 1e12 / 80.0) < 1e-15
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["traffic"] == bench.CLIP_TRAFFIC_BYTES.get(("block_c2", "fp32"))
    # k = 16 takes the 2.5 kFLOP figure; an unmeasured workload has no traffic and no HBM fraction
    r16 = bench.clip_roofline(st, 16, "no_such_workload", "fp32", PEAKS, 6700.0)
    assert r16["flop_per_piece"] == 2500.0 and r16["traffic"] is None and "hbm" not in r16["fractions"]


def test_clip_roofline_fp64_mode_and_binding():
    st = [_stage(990, 9, 1, [10, 20, 30], 1.0, 400)]
    st64 = [_stage(990, 9, 1, [10, 20, 30], 2.0, 400)]
    r = bench.clip_roofline(st, 32, "block_c2", "fp32", PEAKS, 6700.0, stage64=st64)
    want64 = 4500.0 * 400 / 2e-3 / 1e12 / 1.25
    assert abs(r["fractions"]["fp64_mode_fp64"] - want64) < 1e-15
    # binding is judged on executed work (the planned count overstates FP64 mode)
    named = ("fp32_executed", "fp64_mode_fp64_executed")
    assert r["binding"] == max(named, key=lambda k: r["fractions"][k])
    assert r["binding"] == "fp64_mode_fp64_executed"   # 1 TF-class FP64 vs 80 TF FP32 at half the speed
    assert "hbm" in r["fractions"] or bench.CLIP_TRAFFIC_BYTES.get(("block_c2", "fp32")) is None
    r64 = bench.clip_roofline(st64, 32, "block_c2", "fp64", PEAKS, 6700.0)
    assert r64["peak"] == 1.25 and "fp64" in r64["fractions"]


def test_cpu_samples_cover_every_workload():
    for name in bench.WORKLOADS:
        c = bench.CPU_SAMPLES[name]
        assert c["oracle"] >= 1 and c["oracle_1t"] >= 1 and 0 < c["fair"] <= 1 and c["ref"] >= 1


def _row(genus, plain, learned):
    def arm(ms, rounds, inserted, failing, iters, rej):
        return {"ms": ms, "rounds": rounds, "inserted": inserted, "failing": failing, "shrink_pins": inserted,
                "shrink_iters": iters, "rejected": rej}
    return {"genus": genus, "tets": 1000, "plain": arm(*plain), "learned": arm(*learned)}


def test_repair_summary_splits_repaired_and_stalled_shapes():
    rows = [_row(0, (1.0, 0, 0, 0, 0, 0), (0.5, 0, 0, 0, 0, 0)),
            _row(1, (4.0, 2, 3, 0, 30, 0), (3.0, 2, 3, 0, 20, 1)),
            _row(1, (9.0, 5, 7, 4, 70, 0), (8.0, 5, 7, 4, 50, 2)),
            _row(0, (2.0, 1, 1, 0, 10, 0), (2.5, 1, 1, 0, 6, 0))]
    s = bench.repair_summary(rows)
    assert s["shapes"] == 4 and s["repaired"] == 3 and s["same_result"]
    assert [r["index"] for r in s["stalled"]] == [2]
    assert s["total_repaired"]["plain"]["ms"] == 7.0 and s["total_repaired"]["learned"]["shrink_iters"] == 26
    assert s["total"]["plain"]["failing"] == 4 and s["total"]["learned"]["rejected"] == 3
    g0, g1 = s["by_genus"]["0"], s["by_genus"]["1"]
    assert (g0["shapes"], g0["repaired"], g0["needed_repair"]) == (2, 2, 1)
    assert (g1["shapes"], g1["repaired"], g1["needed_repair"]) == (2, 1, 2)
    assert g1["plain"]["inserted"] == 10
    # arms that end differently on some shape are flagged
    rows[1]["learned"]["inserted"] = 4
    assert not bench.repair_summary(rows)["same_result"]
