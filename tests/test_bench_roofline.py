"""The bench's roofline arithmetic (host logic, no GPU): achieved bandwidth
and operation rate from the algorithmic bytes and counted operations of an
average launch, the peak taken from the measured file and labelled (or the
6.8 TB/s fallback, labelled as such), the binding side chosen as the larger
fraction, and the traffic figure of the committed capture carried along."""
import bench


def _launches(ms_total=3.0, n=100, wet=10, updates=100):
    return {"k_ms": ms_total, "k_n": n, "cells": 1024 * 1024, "wet": wet, "updates": updates,
            "g_ms": 0.0, "g_n": 0}


def test_hbm_side_from_algorithmic_bytes_and_measured_peak():
    r = _launches()
    out = bench.roofline(r, 1, {"hbm_gbs": 6000.0, "sm_max_mhz": 2000.0})
    avg_s = 3.0 / 1e3 / 100
    gbs = bench.BYTES_PER_CELL_FP32 * 1024 * 1024 / avg_s / 1e9
    assert abs(out["hbm"]["achieved"] - gbs) <= 1e-9 * gbs
    assert out["hbm"]["peak"] == 6000.0 and out["hbm"]["peak_source"] == "measured"
    assert abs(out["hbm"]["frac"] - gbs / 6000.0) <= 1e-12
    assert abs(out["hbm"]["frac_of_nominal_7900"] - gbs / 7900.0) <= 1e-12
    assert out["traffic"] == bench.TRAFFIC_PER_LAUNCH_FP32
    assert abs(out["avg_launch_ms"] - 0.03) <= 1e-12


def test_fallback_peak_is_labelled():
    out = bench.roofline(_launches(), 1, {})
    assert out["hbm"]["peak"] == 6800.0
    assert out["hbm"]["peak_source"].startswith("fallback")


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
    assert out["traffic"] == bench.TRAFFIC_PER_LAUNCH_FP64
