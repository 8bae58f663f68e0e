"""The bench's roofline arithmetic (host logic, no GPU): achieved bandwidth
from the algorithmic bytes per cell update times the cells of an average
recorded launch over its average duration, the wet-cell share of it, the
operation rate from the counted operations per wet cell update, the peak
taken from the measured file and labelled (or the 6.8 TB/s fallback,
labelled as such), the binding side chosen as the larger fraction, and the
traffic figure carried along."""
import bench


def _launches(ms_total=3.0, n=100, cells_per_launch=1024 * 1024, wet=10, updates=100):
    return {"k_ms": ms_total, "k_n": n, "cells": cells_per_launch * n, "wet": wet,
            "updates": updates}


def test_algorithmic_bytes_per_cell_follow_the_cost_model():
    # read h, hu, hv, b and write h, hu, hv: 7 values; FP32 adds the three
    # compensation terms once
    assert bench.BYTES_PER_CELL_FP64 == 7 * 8
    assert bench.BYTES_PER_CELL_FP32 == 7 * 4 + 3 * 4


def test_hbm_side_from_algorithmic_bytes_and_measured_peak():
    r = _launches()
    out = bench.roofline(r, 1, {"hbm_gbs": 6000.0, "sm_max_mhz": 2000.0}, traffic=12345)
    avg_s = 3.0 / 1e3 / 100
    gbs = bench.BYTES_PER_CELL_FP32 * 1024 * 1024 / avg_s / 1e9
    assert abs(out["hbm"]["achieved"] - gbs) <= 1e-9 * gbs
    assert out["hbm"]["peak"] == 6000.0 and out["hbm"]["peak_source"] == "measured"
    assert abs(out["hbm"]["frac"] - gbs / 6000.0) <= 1e-12
    assert abs(out["hbm"]["frac_of_nominal_7900"] - gbs / 7900.0) <= 1e-12
    assert abs(out["hbm"]["frac_wet"] - 0.1 * gbs / 6000.0) <= 1e-12
    assert out["traffic"] == 12345
    assert abs(out["avg_launch_ms"] - 0.03) <= 1e-12
    assert out["cells_per_launch"] == 1024 * 1024


def test_cells_are_averaged_over_the_recorded_launches():
    # two launches of different sizes: the average launch carries the mean
    r = {"k_ms": 2.0, "k_n": 2, "cells": 1000 + 3000, "wet": 1, "updates": 1}
    out = bench.roofline(r, 0, {"hbm_gbs": 5000.0})
    assert out["cells_per_launch"] == 2000
    assert abs(out["hbm"]["achieved"] - 56 * 2000 / 1e-3 / 1e9) <= 1e-9


def test_fallback_peak_is_labelled():
    out = bench.roofline(_launches(), 1, {})
    assert out["hbm"]["peak"] == 6800.0
    assert out["hbm"]["peak_source"].startswith("fallback")
    assert out["traffic"] is None


def test_alu_side_counts_wet_cell_updates_and_binding_side_is_the_larger():
    # FP64: 2 lanes per SM make the ALU side the larger fraction
    r = _launches(wet=50, updates=100)
    out = bench.roofline(r, 0, {"hbm_gbs": 6000.0, "sm_max_mhz": 2000.0})
    avg_s = 3.0 / 1e3 / 100
    ops = bench.OPS_PER_WET_CELL_FP64 * 0.5 * 1024 * 1024
    peak = bench.N_SM * bench.FP64_LANES_PER_SM * 2000.0 / 1e3
    assert abs(out["alu"]["achieved"] - ops / avg_s / 1e9) <= 1e-9 * ops / avg_s / 1e9
    assert abs(out["alu"]["peak"] - peak) <= 1e-12 * peak
    assert out["bound"] == ("alu" if out["alu"]["frac"] >= out["hbm"]["frac"] else "hbm")
    assert out["frac"] == max(out["alu"]["frac"], out["hbm"]["frac"])


def test_uniform_cpu_sample_is_a_bounded_oracle_run():
    """The uniform workload's CPU sample: the oracle on one core over the
    first steps of the 1024 x 1024 radial dam break, every cell counted."""
    out = bench.cpu_baseline_uniform(steps=1)
    assert out["kind"] == "oracle" and out["cores"] == 1
    assert out["unit"] == "cell-updates/s" and out["value"] > 0
    assert "1024 x 1024 radial dam break" in out["sample"] and "first 1 steps" in out["sample"]
