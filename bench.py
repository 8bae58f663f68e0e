"""Benchmark: cell-updates/s of the GeoFlood wave-propagation hot path.

Headline workload (one bench "step" = one run of it): the 4 km x 2 km
synthetic V-valley dam break on a quadtree of 32 x 32 patches, 16 x 8 blocks
on levels 2-4 (finest cells 0.49 m), side slope 0.05, down-valley slope
0.005, 0.5 m of seeded fractal noise, a 20 m reservoir behind a full breach
at x = 500 m, dry downstream, Manning n = 0.033, CFL 0.9, from t = 0 over
the first VALLEY_T seconds of the flood.  Every accepted step does the ghost
exchange, the augmented Riemann solves, limited corrections, transverse
terms, update, Manning friction and the CFL control on every patch; the
plain refinement criterion is checked every 4 steps and the forest is
regridded (tags, 2:1 balance, refine and coarsen, new tables, fills).

The metric is a pair of runs on that workload:
  value      FP32 surface-deviation form with the learned refinement
             predictor, regrid every 64 steps (the plain criterion still
             judges every 4 steps and forces a regrid on a miss);
  fp64_plain the paper's method: plain FP64, plain tags, regrid every 4;
  fp32_plain the control: FP32 with plain tags, regrid every 4 (the
             network's own gain is fp32_plain's wall time over value's);
with the gauge-depth and arrival-time differences against plain FP64.
cell-updates/s = sum over accepted steps of (patches x 32^2) / time, timed
with CUDA events on the library's stream around each whole run (steps,
checks, regrids, host quadtree), inputs resident on the device (each run
restarts from a checkpoint of the initial state), the L2 flushed (a 256 MB
write) before every run.  e2e: the same run through the C ABI from pinned
host buffers (upload of the initial state, the run, read-back of the final
state and gauges).

Secondary workloads (single GPU only) follow in their own keys.
``--impl reference`` times the FP64 CPU oracle on a bounded sample of the
same workload (the paper has no other implementation to run).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PATCH = 32
VALLEY_T = 60.0
VALLEY_CAP = 16 * 8 * 4 ** 4  # every patch on the finest level
VALLEY_WORKLOAD = ("V-valley 4 km x 2 km, 16x8 blocks of 32x32 patches, levels 2-4 (finest dx "
                   "0.49 m), 20 m reservoir, full breach at x = 500 m, n = 0.033, t 0->%g s")
CNN_SCALE = (4.0, 8.0, 8.0, 4.0)
TRAIN_T = 30.0
# regrid interval of the learned arm (the network is trained on labels over
# the same interval; the plain criterion still checks every 4 steps and
# forces a regrid on a miss): measured on this workload, 16 / 32 / 64 steps
# take 1.33 / 1.20 / 1.05 s per run against 1.38 s for plain tags every 4,
# at the same gauge depths within 1.4e-5 m
LEARNED_REGRID = 64

N_CELLS = 1024
T_UNIFORM = 60.0
UNIFORM_WORKLOAD = "radial dam break 1024x1024, 32x32 patches, dx 2 m, t 0->60 s"

# Algorithmic HBM bytes per cell update of the patch step: read h, hu, hv, b
# and write h, hu, hv -- 7 values: 56 B in FP64, 28 B in FP32, plus 12 B for
# the three FP32 compensation terms of the deviation form (counted once, as
# the cost model of the hot-path scope does; the kernel reads the old terms
# and writes the new ones, 24 B, so the true traffic is 52 B per cell).
BYTES_PER_CELL_FP32 = 40
BYTES_PER_CELL_FP64 = 56
# Operations per wet cell update, counted from the scheme: two edge solves
# (74 each), two limited edge fluxes (81), two increments (9), two
# transverse splits (38), two transverse fluxes (9), the update (30) and
# Manning friction (16) = 468; the deviation form adds the compensated
# update (24) and the exact wet tests (8).
OPS_PER_WET_CELL_FP64 = 468
OPS_PER_WET_CELL_FP32 = 500
FP32_LANES_PER_SM = 128
FP64_LANES_PER_SM = 2  # measured: DFMA throughput 1.20 TFLOP/s on 152 SMs
N_SM = 152
# DRAM bytes (read + write) of one patch-step launch, from the ncu captures
# summarised in profiles/ (cold caches); None when the kernel has changed
# since.  Valley: the launch at t = 30 s (6827 patches) of the 608-thread
# variant that the autotuner picks there, 341 667 840 B over 6 990 848
# cells, scaled to the cells of an average timed launch.  Uniform workload:
# launch 151 (t = 29.5 s), 4 629 504 B.
TRAFFIC_PER_LAUNCH_FP32 = 4629504
TRAFFIC_PER_LAUNCH_FP64 = None
TRAFFIC_PER_CELL_VALLEY_FP32 = 341667840 / 6990848


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--t-end", type=float, default=VALLEY_T,
                    help="end of the headline window in simulated seconds")
    ap.add_argument("--headline-only", action="store_true",
                    help="skip the secondary workloads and CPU baselines")
    ap.add_argument("--pair-only", action="store_true",
                    help="only the valley pair and its control over --t-end, one run each "
                         "after a short warm-up (no profiled or e2e runs); prints its own "
                         "JSON line, not the benchmark line")
    ap.add_argument("--profile-case", type=int, default=0,
                    help="run N x N cells of the uniform workload for --profile-steps "
                         "steps and exit (for ncu captures; prints no JSON)")
    ap.add_argument("--profile-valley", type=float, default=0.0,
                    help="run the valley (FP32, plain tags, regrid every 4) to this time "
                         "and then --profile-steps more steps, and exit (for ncu captures)")
    ap.add_argument("--profile-steps", type=int, default=20)
    ap.add_argument("--profile-precision", type=int, default=1, choices=[0, 1],
                    help="0 = FP64, 1 = FP32 deviation form")
    ap.add_argument("--profile-variant", type=int, default=0,
                    help="patch-step kernel variant (see geoflood_autotune)")
    return ap.parse_args()


def run_profile_case(args):
    """Fixed-length run of the uniform workload at another size (no timing)."""
    from paper_2403_15435_gb300 import geoflood, inputs
    n = args.profile_case
    prob = inputs.radial_dambreak(n, PATCH, dx=2.0, radius=200.0 * n / N_CELLS)
    prob.cfg.precision = args.profile_precision
    f = geoflood.Forest(prob.cfg, prob.dem, max_patches=(n // PATCH) ** 2)
    f.set_state(prob.ic)
    f.set_variant(args.profile_variant)
    _, steps = f.step(1e9, args.profile_steps)
    print("profile case %d x %d: %d steps, t = %.3f s" % (n, n, steps, f.time()["t"]))


def run_profile_valley(args):
    """The valley to a time, then a fixed number of steps (no timing)."""
    from paper_2403_15435_gb300 import geoflood, inputs
    prob = inputs.v_valley()
    prob.cfg.precision = args.profile_precision
    f = geoflood.Forest(prob.cfg, prob.dem, max_patches=VALLEY_CAP)
    f.set_state(prob.ic)
    f.set_variant(args.profile_variant)
    f.advance(args.profile_valley, regrid_interval=4, check_interval=4)
    _, steps = f.step(1e9, args.profile_steps)
    print("profile valley: %d patches, %d steps, t = %.3f s" % (f.npatch, steps, f.time()["t"]))


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(
                    ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                     "--format=csv,noheader,nounits"], capture_output=True, text=True,
                    timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        import statistics
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4)
                          if len(s) > 4 + k and s[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def replica_throughput(units, seconds, world, device=None):
    """Whole-job rate of `world` independent replicas, each having processed
    `units` in its own `seconds`: all ranks' units over the slowest rank's
    time (the maximum over the process group), and that time."""
    import torch
    import torch.distributed as dist
    if world > 1 and dist.is_available() and dist.is_initialized():
        t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        seconds = float(t.item())
    return units * world / seconds, seconds


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def roofline(r, prec, peaks, traffic=None):
    """Roofline of the patch-step kernel from live per-launch events.

    r: k_ms (summed duration of the recorded launches), k_n (their number),
    cells (interior cells of the recorded launches, summed), wet and updates
    (wet and all cell updates over the same runs, for the wet fraction).
    HBM side: algorithmic bytes per cell update x cells per launch / the
    average launch time; frac_wet counts the wet cell updates only.  ALU
    side: counted operations per wet cell update.  The binding side is the
    larger fraction."""
    n = max(1, r["k_n"])
    avg = r["k_ms"] / 1e3 / n
    cells = r["cells"] / n
    wet_frac = r["wet"] / max(1, r["updates"])
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    if "hbm_gbs" in peaks:
        hbm, hbm_src = float(peaks["hbm_gbs"]), "measured"
    else:
        # no measurement on this machine: one earlier GB300 copy measurement
        hbm, hbm_src = 6800.0, "fallback: 6.8 TB/s"
    if prec == 0:
        bytes_cell, ops_wet = BYTES_PER_CELL_FP64, OPS_PER_WET_CELL_FP64
        alu_peak = N_SM * FP64_LANES_PER_SM * mhz / 1e3            # GOP/s
        alu_src = "152 SMs x 2 FP64 lanes x %.0f MHz" % mhz
    else:
        bytes_cell, ops_wet = BYTES_PER_CELL_FP32, OPS_PER_WET_CELL_FP32
        alu_peak = N_SM * FP32_LANES_PER_SM * mhz / 1e3            # GOP/s
        alu_src = "152 SMs x 128 FP32 lanes x %.0f MHz" % mhz
    ops = ops_wet * wet_frac * cells
    alu = ops / avg / 1e9
    gbs = bytes_cell * cells / avg / 1e9
    out = {"kernel": "patch_step (%s)" % ("FP64" if prec == 0 else "FP32 deviation form"),
           "avg_launch_ms": avg * 1e3, "cells_per_launch": cells, "wet_fraction": wet_frac,
           "timed_launches": r["k_n"],
           "timing": "CUDA events around every 4th patch-step launch of a separate "
                     "profiled run of the same workload",
           "bytes_per_cell": bytes_cell,
           "alu": {"achieved": alu, "peak": alu_peak, "unit": "GOP/s", "frac": alu / alu_peak,
                   "ops_per_launch": ops, "peak_source": "derived: " + alu_src},
           "hbm": {"achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                   "frac_of_nominal_7900": gbs / 7900.0,
                   "frac_wet": gbs * wet_frac / hbm,
                   "bytes_per_launch": bytes_cell * cells, "peak_source": hbm_src}}
    side = "alu" if out["alu"]["frac"] >= out["hbm"]["frac"] else "hbm"
    out.update({"bound": side, "achieved": out[side]["achieved"], "peak": out[side]["peak"],
                "unit": out[side]["unit"], "frac": out[side]["frac"],
                "frac_wet": out["hbm"]["frac_wet"], "traffic": traffic})
    return out


# ----------------------------------------------------------------------------
# headline: the valley, three arms
# ----------------------------------------------------------------------------

def train_network(stream, t_end=TRAIN_T, epochs=10, capacity=200000):
    """Network trained on the plain criterion's flags from another seed of the
    valley (FP32, regrid every LEARNED_REGRID steps, the criterion OR'ed over
    the checks up to the next regrid)."""
    import numpy as np
    from paper_2403_15435_gb300 import geoflood, inputs
    t0 = time.perf_counter()
    tr = inputs.v_valley(seed=inputs.SEED_BASE + 50)
    tr.cfg.precision = 1
    f = geoflood.Forest(tr.cfg, tr.dem, max_patches=VALLEY_CAP, stream=stream.cuda_stream)
    f.set_state(tr.ic)
    f.cnn_set_scale(CNN_SCALE)
    f.cnn_dataset(capacity)
    st = f.advance(t_end, regrid_interval=LEARNED_REGRID, check_interval=4, collect=True)
    _, y = f.cnn_dataset_read(0, st["samples"])
    npos = int(y.sum())
    pw = float(np.clip((len(y) - npos) / max(npos, 1), 1.0, 20.0))
    f.cnn_set_params(inputs.cnn_init(3))
    loss = f.cnn_train(epochs, 64, lr=2e-3, pos_weight=pw, seed=7)
    prm = f.cnn_get_params()
    f.close()
    # the positives' weight pw shifts the trained logit by log(pw): the
    # decision threshold pw / (1 + pw) undoes it
    thr = pw / (1.0 + pw)
    return prm, thr, {"workload": "V-valley 4 km x 2 km, seed + 50 (not the benchmarked "
                                  "terrain), FP32, t 0->%g s, labels over %d steps"
                                  % (t_end, LEARNED_REGRID),
                      "samples": int(len(y)), "positives": npos, "epochs": epochs,
                      "pos_weight": pw, "threshold": thr, "loss_first": float(loss[0]),
                      "loss_last": float(loss[-1]), "seconds": time.perf_counter() - t0}


def valley_gauges(prob):
    """The valley's own 16 seeded gauges, then 16 on the thalweg at x = 520,
    545, ..., 895 m, inside the reach of the flood's first minute."""
    import numpy as np
    thalweg = np.stack([520.0 + 25.0 * np.arange(16), np.full(16, 1000.0)], axis=1)
    return np.concatenate([prob.gauges, thalweg], axis=0)


class ValleyArm:
    """One arm of the pair: a context holding the valley at t = 0 and a
    checkpoint of it, from which every run restarts."""

    def __init__(self, stream, prec, learned, regrid, net=None, t_end=VALLEY_T):
        from paper_2403_15435_gb300 import geoflood, inputs
        self.stream = stream
        self.learned, self.regrid, self.t_end = learned, regrid, t_end
        self.prob = inputs.v_valley()
        self.prob.cfg.precision = prec
        f = geoflood.Forest(self.prob.cfg, self.prob.dem, max_patches=VALLEY_CAP,
                            max_gauges=32, stream=stream.cuda_stream)
        f.set_state(self.prob.ic)
        f.cnn_set_scale(CNN_SCALE)
        if learned:
            f.cnn_set_params(net[0])
            f.set_tagger(geoflood.TAGGER_LEARNED, net[1])
        f.set_gauges(valley_gauges(self.prob))
        self.f = f
        self.ckpt = f.save()
        self.cells0 = f.npatch * PATCH * PATCH

    def run(self, flush=None, t_end=None):
        """One whole run from the checkpoint; CUDA events on the library's
        stream around it.  Returns the advance statistics and the seconds."""
        import torch
        f = self.f
        f.load(self.ckpt)
        if flush is not None:
            with torch.cuda.stream(self.stream):
                flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        c0 = f.counters()
        torch.cuda.synchronize()
        a.record(self.stream)
        st = f.advance(self.t_end if t_end is None else t_end, regrid_interval=self.regrid,
                       check_interval=4, regrid_on_miss=self.learned)
        b.record(self.stream)
        torch.cuda.synchronize()
        c1 = f.counters()
        st["cell_updates_counted"] = c1[0] - c0[0]
        st["wet_updates_counted"] = c1[1] - c0[1]
        return st, a.elapsed_time(b) / 1e3

    def autotune(self, t_mid):
        """The patch-step kernel shape for this arm: every variant timed on
        the state at t_mid (the middle of the window), the fastest kept for
        the runs that follow (a checkpoint load keeps it)."""
        self.f.load(self.ckpt)
        self.f.advance(t_mid, regrid_interval=self.regrid, check_interval=4,
                       regrid_on_miss=self.learned)
        variant, ms = self.f.autotune(5)
        self.variant = {"chosen": int(variant), "ms_per_launch": [float(x) for x in ms if x == x],
                        "at_t_s": t_mid, "patches": self.f.npatch}
        return self.variant

    def summary(self, runs):
        """Rates of a list of (stats, seconds) runs and the last run's state."""
        cells = sum(st["patch_steps"] for st, _ in runs) * PATCH * PATCH
        sec = sum(s for _, s in runs)
        st = runs[-1][0]
        out, arr = self.f.gauges()
        return {"value": cells / sec, "unit": "cell-updates/s",
                "wall_s": sec / len(runs), "runs": len(runs),
                "kernel_variant": getattr(self, "variant", None),
                "steps": st["steps"], "regrids": st["regrids"],
                "regrids_on_miss": st["miss_regrids"], "checks": st["checks"],
                "criterion_misses": st["misses"],
                "cell_updates": st["patch_steps"] * PATCH * PATCH,
                "patches_at_end": self.f.npatch,
                "time_split_s": {"steps_and_checks": st["step_s"], "separate_checks": st["check_s"],
                                 "regrids": st["regrid_s"],
                                 "of_which_host_quadtree": st["regrid_host_s"]},
                "_gauge_h": out[:, 1].copy(), "_arrival": arr.copy()}

    def close(self):
        self.f.close()


def compare_gauges(ref, other):
    """Gauge depths and arrival times of `other` against `ref` (plain FP64)."""
    import numpy as np
    both = (ref["_arrival"] >= 0) & (other["_arrival"] >= 0)
    own = slice(0, 16)
    thal = slice(16, 32)

    def part(sl):
        b = both[sl]
        return {"depth_max_abs_m": float(np.abs(other["_gauge_h"][sl] - ref["_gauge_h"][sl]).max()),
                "arrival_max_abs_s": float(np.abs(other["_arrival"][sl] - ref["_arrival"][sl])[b].max())
                if b.any() else None,
                "reached": [int((ref["_arrival"][sl] >= 0).sum()),
                            int((other["_arrival"][sl] >= 0).sum())]}
    return {"valley_16_seeded_gauges": part(own), "thalweg_16_gauges": part(thal)}


def measure_valley(args, dev, stream, world, local, peaks):
    """The headline pair (and its control) on the valley: warm-up runs, then
    args.steps timed runs of FP32 + learned tags; plain FP64 and FP32 with
    plain tags timed once each after a warm-up; a separate profiled run of
    the headline arm for the patch step's per-launch time; the end-to-end
    runs through the C ABI from host buffers."""
    import numpy as np
    import torch

    net_prm, net_thr, train = train_network(stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    head = ValleyArm(stream, 1, True, LEARNED_REGRID, net=(net_prm, net_thr), t_end=args.t_end)
    head.run(flush)
    head.autotune(0.5 * args.t_end)
    for _ in range(args.warmup):
        head.run(flush)
    launches0 = head.f.launch_count()
    runs = []
    with ClockSampler(local) as clk:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        # an NVTX range around the timed runs, so that a profiler can be
        # told to record this region only
        torch.cuda.nvtx.range_push("timed")
        for _ in range(args.steps):
            runs.append(head.run(flush))
        torch.cuda.synchronize(dev)
        torch.cuda.nvtx.range_pop()
    launches = head.f.launch_count() - launches0
    sec = sum(s for _, s in runs)
    cells = sum(st["patch_steps"] for st, _ in runs) * PATCH * PATCH
    value, sec_max = replica_throughput(cells, sec, world, dev)
    learned = head.summary(runs)

    # the patch step's per-launch time: a separate run with every 4th launch
    # of each captured chunk bracketed by events
    head.f.profile(True, every=4)
    pst, _ = head.run(flush)
    k_ms, k_n = head.f.profile_read("patch_step")
    k_cells = head.f.profile_cells("patch_step")
    g_ms, g_n = head.f.profile_read("ghost_fill")
    head.f.profile(False)
    learned["level_change_ghost_fill_ms_per_launch"] = g_ms / g_n if g_n else None
    prof = {"k_ms": k_ms, "k_n": k_n, "cells": k_cells, "wet": pst["wet_updates_counted"],
            "updates": pst["cell_updates_counted"]}
    traffic = None
    if TRAFFIC_PER_CELL_VALLEY_FP32 is not None and k_n:
        traffic = TRAFFIC_PER_CELL_VALLEY_FP32 * k_cells / k_n
    roof = roofline(prof, 1, peaks, traffic)

    # end to end through the C ABI: the initial state uploaded from pinned
    # host arrays, the run, the final state and the gauges read back
    f = head.f
    f.load(head.ckpt)
    h0, hu0, hv0, _ = f.read()
    pin = lambda n: torch.empty((n, PATCH, PATCH), dtype=torch.float64, pin_memory=True).numpy()
    H, HU, HV = pin(len(h0)), pin(len(h0)), pin(len(h0))
    H[:], HU[:], HV[:] = h0, hu0, hv0
    n_end = learned["patches_at_end"]
    OH, OHU, OHV = pin(n_end), pin(n_end), pin(n_end)
    e2e_t, e2e_cells, d2h = [], [], 0
    for _ in range(max(1, min(args.steps, 3))):
        f.load(head.ckpt)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        f.write(H, HU, HV)
        f.set_time(0.0, head.prob.cfg.dt_initial)
        st = f.advance(args.t_end, regrid_interval=LEARNED_REGRID, check_interval=4,
                       regrid_on_miss=True)
        if f.npatch != n_end:
            OH, OHU, OHV = pin(f.npatch), pin(f.npatch), pin(f.npatch)
            n_end = f.npatch
        f.read_into(OH, OHU, OHV)
        gout, garr = f.gauges()
        e2e_t.append(time.perf_counter() - t0)
        e2e_cells.append(st["patch_steps"] * PATCH * PATCH)
        d2h = 3 * OH.nbytes + gout.nbytes + garr.nbytes
    e2e = {"value": sum(e2e_cells) * world / sum(e2e_t), "unit": "cell-updates/s",
           "h2d_bytes_per_step": 3 * H.nbytes, "d2h_bytes_per_step": d2h}
    head.close()

    # the pair's other side and the control, each warmed up on a short run
    fp64 = ValleyArm(stream, 0, False, 4, t_end=args.t_end)
    fp64.run(flush, t_end=2.0)
    fp64.autotune(0.25 * args.t_end)
    plain64 = fp64.summary([fp64.run(flush)])
    fp64.close()
    fp32p = ValleyArm(stream, 1, False, 4, t_end=args.t_end)
    fp32p.run(flush, t_end=2.0)
    fp32p.autotune(0.5 * args.t_end)
    plain32 = fp32p.summary([fp32p.run(flush) for _ in range(2)])
    fp32p.close()

    err = {"fp32_learned": compare_gauges(plain64, learned),
           "fp32_plain": compare_gauges(plain64, plain32)}
    for r in (learned, plain64, plain32):
        r.pop("_gauge_h")
        r.pop("_arrival")
    return dict(net=(net_prm, net_thr), value=value, sec=sec_max, runs=len(runs),
                launches=launches,
                clocks=clk.summary(), learned=learned, fp64=plain64, fp32_plain=plain32,
                err=err, train=train, roofline=roof, e2e=e2e,
                cells_per_run=cells / max(1, len(runs)))


def run_pair_only(args):
    """The metric's pair over a longer window: FP32 + learned tags (regrid
    every LEARNED_REGRID), plain FP64 and FP32 + plain tags (regrid every 4),
    each warmed up on the first 2 s and then run once over t = 0 -> t_end,
    timed with CUDA events around the run; gauge errors against plain FP64."""
    import torch
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    net_prm, net_thr, train = train_network(stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = {}
    for key, prec, learned, regrid in (("fp32_learned", 1, True, LEARNED_REGRID),
                                       ("fp64_plain", 0, False, 4),
                                       ("fp32_plain", 1, False, 4)):
        arm = ValleyArm(stream, prec, learned, regrid,
                        net=(net_prm, net_thr) if learned else None, t_end=args.t_end)
        arm.run(flush, t_end=2.0)
        out[key] = arm.summary([arm.run(flush)])
        arm.close()
    err = {"fp32_learned": compare_gauges(out["fp64_plain"], out["fp32_learned"]),
           "fp32_plain": compare_gauges(out["fp64_plain"], out["fp32_plain"])}
    for r in out.values():
        r.pop("_gauge_h")
        r.pop("_arrival")
    lr, f64 = out["fp32_learned"], out["fp64_plain"]
    print(json.dumps({
        "mode": "pair-only", "metric": "cell-updates/s", "unit": "cell-updates/s",
        "value": lr["value"], "dtype": "f32 (vs f64)", "data": "synthetic",
        "config": {"workload": VALLEY_WORKLOAD % args.t_end,
                   "timing": "one run per arm after a 2 s warm-up, CUDA events on the "
                             "library's stream, L2 flushed before each run"},
        "fp32_learned": lr, "fp64_plain": f64, "fp32_plain": out["fp32_plain"],
        "wall_clock_ratio_vs_fp64": f64["wall_s"] / lr["wall_s"],
        "network_gain_wall": out["fp32_plain"]["wall_s"] / lr["wall_s"],
        "error_vs_plain_fp64": err, "training": train}))


# ----------------------------------------------------------------------------
# secondary workloads
# ----------------------------------------------------------------------------

def measure_uniform(prec, args, dev, stream, gauges, peaks):
    """The 1024 x 1024 radial dam break (uniform grid, no regrid) to 60 s in
    one precision: warm-up runs, args.steps timed runs (L2 flushed before
    each), then one profiled run for the patch step's per-launch time."""
    import torch
    from paper_2403_15435_gb300 import geoflood, inputs

    prob = inputs.radial_dambreak(N_CELLS, PATCH, dx=2.0)
    prob.cfg.precision = prec
    f = geoflood.Forest(prob.cfg, prob.dem, stream=stream.cuda_stream)
    f.set_state(prob.ic)
    f.set_gauges(gauges)
    n = f.npatch
    cells = n * PATCH * PATCH
    h0, hu0, hv0, _ = f.read()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def reset():
        f.write(h0, hu0, hv0)
        f.set_time(0.0, prob.cfg.dt_initial)
        f.set_gauges(gauges)

    for _ in range(max(1, min(args.warmup, 3))):
        reset()
        f.step(T_UNIFORM)
    reset()
    f.step(T_UNIFORM * 0.5)
    variant, variant_ms = f.autotune(5)
    ev, steps = [], []
    for _ in range(max(1, min(args.steps, 5))):
        reset()
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, n_acc = f.step(T_UNIFORM)
        b.record(stream)
        ev.append((a, b))
        steps.append(n_acc)
    torch.cuda.synchronize(dev)
    sec = sum(a.elapsed_time(b) / 1e3 for a, b in ev)
    gauge_out, arrival = f.gauges()
    final = f.read()[:3]
    # profiled run
    reset()
    f.profile(True, every=4)
    cu0, wet0 = f.counters()
    f.step(T_UNIFORM)
    cu1, wet1 = f.counters()
    k_ms, k_n = f.profile_read("patch_step")
    k_cells = f.profile_cells("patch_step")
    g_ms, g_n = f.profile_read("ghost_fill")
    f.profile(False)
    f.close()
    traffic = TRAFFIC_PER_LAUNCH_FP64 if prec == 0 else TRAFFIC_PER_LAUNCH_FP32
    roof = roofline({"k_ms": k_ms, "k_n": k_n, "cells": k_cells, "wet": wet1 - wet0,
                     "updates": cu1 - cu0}, prec, peaks, traffic)
    return dict(value=sum(steps) * cells / sec, ms_per_run=1e3 * sec / len(steps),
                steps=steps[0], variant=variant,
                variant_ms=[float(x) for x in variant_ms if x == x], roofline=roof,
                gauges=gauge_out, arrival=arrival, final=final)


def measure_uniform_pair(args, dev, stream, peaks):
    import numpy as np
    ang = np.linspace(0.0, 2 * np.pi, 16, endpoint=False)
    rad = np.linspace(250.0, 900.0, 16)
    gauges = np.stack([1024.0 + rad * np.cos(ang), 1024.0 + rad * np.sin(ang)], 1)
    r32 = measure_uniform(1, args, dev, stream, gauges, peaks)
    r64 = measure_uniform(0, args, dev, stream, gauges, peaks)
    err = {"max_abs_depth_m": float(np.abs(r32["final"][0] - r64["final"][0]).max()),
           "max_abs_momentum_m2s": float(max(np.abs(r32["final"][1] - r64["final"][1]).max(),
                                             np.abs(r32["final"][2] - r64["final"][2]).max())),
           "gauge_depth_max_abs_m": float(np.abs(r32["gauges"][:, 1] - r64["gauges"][:, 1]).max()),
           "arrival_max_abs_s": float(np.abs(r32["arrival"] - r64["arrival"]).max())}
    out = {"workload": UNIFORM_WORKLOAD, "fp32_vs_fp64_error": err,
           "timing": "CUDA events around each whole run, L2 flushed before each"}
    for name, r in (("fp32", r32), ("fp64", r64)):
        out[name] = {"value": r["value"], "unit": "cell-updates/s", "ms_per_run": r["ms_per_run"],
                     "accepted_steps_per_run": r["steps"],
                     "kernel_variant": {"chosen": r["variant"], "ms_per_launch": r["variant_ms"]},
                     "roofline": r["roofline"]}
    return out


CANYON_T = 20.0


def measure_canyon(stream, net, patch=32):
    """The 17 km x 9 km canyon-to-plain dam break (55 m reservoir, five
    levels: 32 x 32 patches on levels 0-4, or 16 x 16 patches on levels 1-5,
    the same cell sizes), first CANYON_T seconds: FP32 with learned tags
    (regrid every LEARNED_REGRID; the network is the one trained on the plain
    criterion's flags from valley runs of 32 x 32 patches) against FP32 and
    FP64 with plain tags (regrid every 4).  Wall clock of the driver loop,
    second of two runs."""
    import numpy as np
    import torch
    from paper_2403_15435_gb300 import geoflood, inputs

    cap = 40000 if patch == 32 else 160000
    lmin, lmax = (0, 4) if patch == 32 else (1, 5)
    scale = CNN_SCALE
    prm, thr = net

    def run(prec, learned, regrid):
        prob = inputs.canyon_plain(patch=patch, minlevel=lmin, maxlevel=lmax, precision=prec,
                                   near_gauges=16)
        res = None
        for rep in range(2):
            g = geoflood.Forest(prob.cfg, prob.dem, max_patches=cap, stream=stream.cuda_stream)
            g.set_state(prob.ic)
            g.cnn_set_scale(scale)
            if learned:
                g.cnn_set_params(prm)
                g.set_tagger(geoflood.TAGGER_LEARNED, thr)
            g.set_gauges(prob.gauges)
            torch.cuda.synchronize()
            a = time.perf_counter()
            s = g.advance(CANYON_T if rep else 2.0, regrid_interval=regrid, check_interval=4,
                          regrid_on_miss=learned)
            torch.cuda.synchronize()
            wall = time.perf_counter() - a
            out, arr = g.gauges()
            res = {"value": s["patch_steps"] * patch * patch / wall, "unit": "cell-updates/s",
                   "wall_s": wall, "steps": s["steps"], "regrids": s["regrids"],
                   "patches_at_end": g.npatch, "levels": sorted(set(int(x) for x in g.patch_info()[0])),
                   "time_split_s": {"steps_and_checks": s["step_s"], "separate_checks": s["check_s"],
                                    "regrids": s["regrid_s"],
                                    "of_which_host_quadtree": s["regrid_host_s"]},
                   "_h": out[:, 1].copy(), "_a": arr.copy()}
            g.close()
        return res

    learned = run(1, True, LEARNED_REGRID)
    plain32 = run(1, False, 4)
    plain64 = run(0, False, 4)
    err = {}
    for name, r in (("fp32_learned", learned), ("fp32_plain", plain32)):
        both = (r["_a"] >= 0) & (plain64["_a"] >= 0)
        err[name] = {"gauge_depth_max_abs_m": float(np.abs(r["_h"] - plain64["_h"]).max()),
                     "arrival_max_abs_s": float(np.abs(r["_a"] - plain64["_a"])[both].max())
                     if both.any() else None,
                     "reached": int(both.sum())}
    for r in (learned, plain32, plain64):
        r.pop("_h")
        r.pop("_a")
    return {"workload": "canyon-to-plain 17 km x 9 km, 55 m reservoir, %dx%d patches, levels "
                        "%d-%d (finest dx 1.95 m), 32 gauges on the channel (16 within 2.05-2.8 km "
                        "of the upstream end), t 0->%g s" % (patch, patch, lmin, lmax, CANYON_T),
            "fp32_learned": learned, "fp32_plain_regrid4": plain32,
            "learned_regrid_interval": LEARNED_REGRID,
            "fp64_plain_regrid4": plain64, "error_vs_plain_fp64": err,
            "wall_clock_ratio_vs_fp64": plain64["wall_s"] / learned["wall_s"],
            "network_gain_wall": plain32["wall_s"] / learned["wall_s"],
            "training": {"threshold": thr,
                         "data": "the headline's network: plain-criterion flags of valley runs"},
            "timing": "wall clock around the whole driver loop, second of two runs"}


ENS_N = 64
ENS_T = 6.0


def measure_ensemble_full(stream):
    """64 scenarios of the full 4 km x 2 km valley (breach width U[50,400] m,
    reservoir depth U[10,30] m, n U[0.02,0.05], each with its own terrain and
    quadtree on levels 2-4, at least 2048 patches each) advanced together in
    one context, FP32, plain tags, regrid every 4 steps, t 0 -> ENS_T s; and
    four of them run alone (one context each) for their own times."""
    import torch
    from paper_2403_15435_gb300 import geoflood, inputs

    probs = inputs.valley_ensemble_full(ENS_N)
    cfg = probs[0].cfg

    def setup(ps):
        f = geoflood.Forest(cfg, None, num_scenarios=len(ps), max_patches=len(ps) * 8192,
                            max_gauges=16, stream=stream.cuda_stream)
        for k, p in enumerate(ps):
            f.set_scenario(k, p.cfg.manning_n, p.cfg.eta0)
            f.set_topo(p.dem, k)
            f.set_state(p.ic, k)
            f.set_gauges(p.gauges, k)
        return f

    def timed(f, n, t_end):
        torch.cuda.synchronize()
        a = time.perf_counter()
        st = f.advance(t_end, regrid_interval=4, check_interval=4)
        torch.cuda.synchronize()
        wall = time.perf_counter() - a
        cells = sum(f.counters(k)[0] for k in range(n))
        return st, wall, cells

    f = setup(probs[:2])  # warm-up: graphs, kernels
    f.advance(1.0, regrid_interval=4, check_interval=4)
    f.close()
    f = setup(probs)
    patches0 = sum(f.npatch_of(k) for k in range(ENS_N))
    st, wall, cells = timed(f, ENS_N, ENS_T)
    patches = [f.npatch_of(k) for k in range(ENS_N)]
    steps = [int(f.time(k)["steps"]) for k in range(ENS_N)]
    f.close()
    alone = []
    for k in (0, 21, 42, 63):
        g = setup([probs[k]])
        _, w, c = timed(g, 1, ENS_T)
        alone.append({"scenario": k, "wall_s": w, "cell_updates": int(c),
                      "value": c / w, "patches_at_end": g.npatch})
        g.close()
    return {"workload": "%d scenarios of the V-valley 4 km x 2 km (32x32 patches, levels 2-4, "
                        ">= 2048 patches each), breach width U[50,400] m, depth U[10,30] m, "
                        "n U[0.02,0.05], FP32, plain tags, regrid every 4, t 0->%g s"
                        % (ENS_N, ENS_T),
            "value": cells / wall, "unit": "cell-updates/s", "wall_s": wall,
            "patches_at_start": int(patches0),
            "patches_at_end": {"total": int(sum(patches)), "min": int(min(patches)),
                               "max": int(max(patches))},
            "steps_per_scenario": {"min": min(steps), "max": max(steps)},
            "regrids": st["regrids"],
            "time_split_s": {"steps_and_checks": st["step_s"], "separate_checks": st["check_s"],
                             "regrids": st["regrid_s"],
                             "of_which_host_quadtree": st["regrid_host_s"]},
            "time_to_t_end_s": {"all_scenarios_in_one_context": wall,
                                "scenarios_alone": alone},
            "timing": "wall clock around the whole driver loop (steps, checks, regrids)"}


VAR_STEPS = 96


def measure_variants(stream):
    """Scheme variants of Sec. 3.2 on the uniform workload (FP32 deviation
    form and FP64): the state at t = 20 s of the default method, then
    VAR_STEPS steps of each variant from it (two graph chunks of warm-up
    first), timed with CUDA events on the library's stream.  The
    no-transverse variant runs at its stability bound (CFL 0.45), which does
    not change the cost of a step."""
    import torch
    from paper_2403_15435_gb300 import geoflood, inputs

    out = {}
    flags = [("default", {}), ("first_order", dict(first_order=1)),
             ("no_transverse", dict(no_transverse=1, cfl_desired=0.45, cfl_max=0.5)),
             ("dim_split", dict(dim_split=1)), ("dim_split_first_order", dict(dim_split=1, first_order=1))]
    for prec in (1, 0):
        base = inputs.radial_dambreak(N_CELLS, PATCH, dx=2.0)
        base.cfg.precision = prec
        f = geoflood.Forest(base.cfg, base.dem, stream=stream.cuda_stream)
        f.set_state(base.ic)
        f.step(20.0)
        h, hu, hv, _ = f.read()
        t, dt = f.time()["t"], f.time()["dt_next"]
        f.close()
        res = {}
        for name, fl in flags:
            cfg = inputs.Config(**{**base.cfg.__dict__, **fl})
            g = geoflood.Forest(cfg, base.dem, stream=stream.cuda_stream)
            g.write(h, hu, hv)
            g.set_time(t, dt)
            g.step(1e9, 32)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            _, n = g.step(1e9, VAR_STEPS)
            b.record(stream)
            torch.cuda.synchronize()
            sec = a.elapsed_time(b) / 1e3
            cells = g.npatch * PATCH * PATCH
            res[name] = {"value": n * cells / sec, "unit": "cell-updates/s",
                         "us_per_step": 1e6 * sec / max(1, n), "steps": n}
            g.close()
        d = res["default"]["value"]
        for r in res.values():
            r["vs_default"] = r["value"] / d
        out["fp32" if prec else "fp64"] = res
    out["workload"] = UNIFORM_WORKLOAD.replace("t 0->60 s", "t 20 s + %d steps" % VAR_STEPS)
    return out


FS_T_END = 3600.0


def measure_flood_speed(stream):
    """Test Case 1 stand-in (Sec. 5.1): flat dry 1000 m x 2000 m plain fed
    by the inflow hydrograph through 20 m of its left side, 32x32 patches on
    levels 0-3 (finest dx 3.9 m), plain tagging with a regrid every 4 steps,
    FP32 deviation form, the first hour (the rising limb); wall clock of the
    driver loop, and the volume that entered against the integral of Q."""
    import torch
    from paper_2403_15435_gb300 import geoflood, inputs

    res = None
    for rep in range(2):  # the first run instantiates graphs and warms up
        prob = inputs.flood_speed(patch=32, minlevel=0, maxlevel=3, precision=1,
                                  t_end=FS_T_END)
        g = geoflood.Forest(prob.cfg, prob.dem, stream=stream.cuda_stream)
        g.set_state(prob.ic)
        v0 = g.mass()
        torch.cuda.synchronize()
        a = time.perf_counter()
        st = g.advance(FS_T_END if rep else 120.0, regrid_interval=4, check_interval=4)
        torch.cuda.synchronize()
        wall = time.perf_counter() - a
        cells = st["patch_steps"] * PATCH * PATCH
        vin = 0.5 * FS_T_END * 20.0 * min(FS_T_END, 3600.0) / 3600.0
        res = {"value": cells / wall, "unit": "cell-updates/s", "wall_s": wall,
               "steps": st["steps"], "regrids": st["regrids"], "cell_updates": cells,
               "patches_at_end": g.npatch,
               "time_split_s": {"steps_and_checks": st["step_s"], "separate_checks": st["check_s"],
                                "regrids": st["regrid_s"],
                                "of_which_host_quadtree": st["regrid_host_s"]},
               "volume_in_m3": g.mass() - v0 - g.time()["clipvol"],
               "integral_of_Q_m3": vin}
        g.close()
    res["workload"] = ("flood speed over a flat dry plain 1000 m x 2000 m, inflow 0->20 m3/s "
                       "over 20 m of the left side, 32x32 patches, levels 0-3, n 0.03, t 0->%g s"
                       % FS_T_END)
    res["timing"] = "wall clock around the whole driver loop (steps, checks, regrids), second run"
    return res


SUB_T = 90.0


def measure_subcycle(stream):
    """Level subcycling on the 2 km x 1 km valley (levels 0-3, FP32 deviation
    form, plain tagging, a regrid every 4 macro steps) against one time step
    for all levels, to the same end time: wall clock of the driver loop, cell
    updates actually computed, and the gauge depths' difference."""
    import numpy as np
    import torch
    from paper_2403_15435_gb300 import geoflood, inputs

    res = {}
    for sub in (0, 1):
        prob = inputs.valley_2km(precision=1)
        prob.cfg.subcycle = sub
        r = None
        for rep in range(2):  # the first run instantiates graphs and warms up
            g = geoflood.Forest(prob.cfg, prob.dem, stream=stream.cuda_stream)
            g.set_state(prob.ic)
            g.set_gauges(prob.gauges)
            torch.cuda.synchronize()
            a = time.perf_counter()
            st = g.advance(SUB_T if rep else 10.0, regrid_interval=4, check_interval=4)
            torch.cuda.synchronize()
            wall = time.perf_counter() - a
            cu = g.counters()[0]
            out, arr = g.gauges()
            r = {"wall_s": wall, "steps": st["steps"], "regrids": st["regrids"],
                 "cell_updates": int(cu), "cell_updates_per_s": cu / wall,
                 "simulated_s_per_wall_s": SUB_T / wall, "gauge_h": out[:, 1].copy()}
            g.close()
        res["subcycled" if sub else "global_step"] = r
    d = float(np.abs(res["subcycled"].pop("gauge_h") - res["global_step"].pop("gauge_h")).max())
    res["gauge_depth_max_abs_diff_m"] = d
    res["speedup_wall"] = res["global_step"]["wall_s"] / res["subcycled"]["wall_s"]
    res["workload"] = ("V-valley 2 km x 1 km, 4x2 blocks of 32x32 patches, levels 0-3 (finest dx "
                       "1.95 m), 12 m reservoir, full breach at x = 350 m, n = 0.033, FP32, plain "
                       "tags, t 0->%g s, 8 gauges" % SUB_T)
    res["timing"] = "wall clock around the whole driver loop, second of two runs"
    return res


def measure_topo(stream):
    """Bed evaluation from three nested DEMs (20 m over the whole domain,
    5 m and 2 m over nested boxes, Sec. 6.2) for a 2 km x 1 km forest of
    32x32 patches at uniform level 3 (512 patches, 1.95 m cells): seconds
    per geoflood_set_topos call (every tile cell, ghosts included) against
    the single 20 m DEM."""
    import torch
    from paper_2403_15435_gb300 import geoflood, inputs

    cfg = inputs.Config(mi=4, mj=2, mx=32, minlevel=3, maxlevel=3, xupper=2000.0,
                        yupper=1000.0, drytol=1e-3)
    dems = inputs.nested_dems(cfg, 12, [None, (400.0, 1200.0, 200.0, 800.0),
                                        (600.0, 900.0, 400.0, 600.0)], [20.0, 5.0, 2.0])
    g = geoflood.Forest(cfg, None, stream=stream.cuda_stream)
    out = {}
    for name, d in (("one_dem_20m", dems[:1]), ("nested_20_5_2m", dems)):
        g.set_topo(d)
        torch.cuda.synchronize()
        a = time.perf_counter()
        for _ in range(5):
            g.set_topo(d)
        torch.cuda.synchronize()
        sec = (time.perf_counter() - a) / 5
        tiles = g.npatch * (PATCH + 4) ** 2
        out[name] = {"seconds": sec, "tile_cells_per_s": tiles / sec}
    g.close()
    out["workload"] = "2 km x 1 km, 512 patches of 32x32 (level 3), every tile cell's bed"
    out["timing"] = "wall clock per set_topo call (DEM upload, bed kernel, ghost fill), mean of 5"
    return out


# ----------------------------------------------------------------------------
# CPU baselines: the oracle as it stands
# ----------------------------------------------------------------------------

CPU_STEPS = 20


def _oracle_valley(steps):
    """The oracle on the headline valley from t = 0: `steps` accepted steps
    with a regrid every 4 (the plain criterion), FP64.  Returns the cell
    updates and the seconds."""
    import oracle
    from paper_2403_15435_gb300 import inputs
    prob = inputs.v_valley()
    f = oracle.OracleForest(prob.cfg, prob.dem)
    f.set_state(prob.ic)
    t0 = time.perf_counter()
    cells = 0
    done = 0
    while done < steps:
        n0 = f.npatch
        _, n = f.step(1e9, min(4, steps - done))
        cells += n * n0 * PATCH * PATCH
        done += n
        if done < steps:
            f.regrid()
    return cells, time.perf_counter() - t0


def cpu_baseline():
    """The oracle on one host core over a bounded sample of the headline
    workload: the valley's first CPU_STEPS steps with their regrids."""
    cells, sec = _oracle_valley(CPU_STEPS)
    return {"value": cells / sec, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
            "sample": "the headline valley from t = 0, its first %d steps with a regrid every "
                      "4 (2048 -> ~6000 patches of 32x32), FP64, %.1f s" % (CPU_STEPS, sec)}


CPU_STEPS_UNIFORM = 40


def cpu_baseline_uniform(steps=CPU_STEPS_UNIFORM):
    """The oracle on one host core on the 1024 x 1024 radial dam break (the
    uniform workload) from t = 0: its first `steps` accepted steps of the
    299 that reach t = 60 s."""
    import oracle
    from paper_2403_15435_gb300 import inputs
    prob = inputs.radial_dambreak(N_CELLS, PATCH, dx=2.0, radius=200.0)
    f = oracle.OracleForest(prob.cfg, prob.dem)
    f.set_state(prob.ic)
    t0 = time.perf_counter()
    _, n = f.step(1e9, steps)
    sec = time.perf_counter() - t0
    cells = n * N_CELLS * N_CELLS
    f.close()
    return {"value": cells / sec, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
            "sample": "the 1024 x 1024 radial dam break from t = 0, its first %d steps "
                      "(of 299 to t = 60 s), FP64, %.1f s" % (n, sec)}


def cpu_baseline_all_cores(steps=12):
    """The same oracle, unchanged, on every host core at once: one spawned
    process per core, each stepping its own copy of the sample; the sum of
    their rates."""
    import multiprocessing as mp
    n = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(n) as pool:
        res = pool.map(_oracle_valley, [steps] * n)
    return {"value": sum(c / t for c, t in res), "unit": "cell-updates/s", "cores": n,
            "kind": "oracle",
            "sample": "%d processes, each the valley's first %d steps with regrids" % (n, steps)}


def run_reference(args):
    """The oracle on the headline workload: one bench step = one accepted
    time step of the valley (with the regrid every 4 steps that the method
    takes), on one host core, from t = 0 after the warm-up steps."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2403_15435_gb300 import inputs
    prob = inputs.v_valley()
    f = oracle.OracleForest(prob.cfg, prob.dem)
    f.set_state(prob.ic)
    taken = 0

    def one_step():
        nonlocal taken
        n0 = f.npatch
        _, n = f.step(1e9, 1)
        taken += n
        if taken % 4 == 0:
            f.regrid()
        return n * n0 * PATCH * PATCH

    for _ in range(args.warmup):
        one_step()
    t0 = time.perf_counter()
    cells = sum(one_step() for _ in range(args.steps))
    dt = time.perf_counter() - t0
    v = cells / dt
    sample = ("steps %d-%d of the valley from t = 0 (regrid every 4), one oracle time step per "
              "bench step" % (args.warmup + 1, args.warmup + args.steps))
    line = {"impl": "reference", "metric": "cell-updates/s", "value": v,
            "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": VALLEY_WORKLOAD % args.t_end, "sample": sample},
            "cpu_baseline": {"value": v, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # a stream of its own: the library captures its step chunks as CUDA
    # graphs, which the legacy default stream does not allow
    stream = torch.cuda.Stream(device=dev)
    peaks = measured_peaks()
    v = measure_valley(args, dev, stream, world, local, peaks)
    # the secondary workloads and the CPU baselines: one GPU only (with
    # replicas on several GPUs the headline is what scales)
    single = world == 1 and not args.headline_only
    uniform = measure_uniform_pair(args, dev, stream, peaks) if single else None
    canyon = measure_canyon(stream, v["net"]) if single else None
    canyon16 = measure_canyon(stream, v["net"], patch=16) if single else None
    ens = measure_ensemble_full(stream) if single else None
    variants = measure_variants(stream) if single else None
    flood = measure_flood_speed(stream) if single else None
    topo = measure_topo(stream) if single else None
    subcyc = measure_subcycle(stream) if single else None
    cpu = cpu_baseline() if (world == 1 and rank == 0) else None
    cpu_all = cpu_baseline_all_cores() if single else None
    cpu_uniform = cpu_baseline_uniform() if single else None
    lr, f64 = v["learned"], v["fp64"]
    line = {
        "metric": "cell-updates/s", "value": v["value"], "unit": "cell-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * v["sec"] / max(1, v["runs"]), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (vs f64)", "data": "synthetic",
        "config": {"workload": VALLEY_WORKLOAD % args.t_end,
                   "pair": "FP32 surface-deviation form + learned tags, regrid every %d "
                           "(value) vs plain FP64 + plain tags, regrid every 4 (fp64_plain)"
                           % LEARNED_REGRID,
                   "cell_updates_per_run": v["cells_per_run"],
                   "steps_per_run": lr["steps"], "patches_at_end": lr["patches_at_end"],
                   "l2": "flushed (256 MB write) before each timed run; the state (2-8k "
                         "patches, 70-250 MB per buffer) exceeds L2",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "fp64_plain": f64,
        "fp32_plain": v["fp32_plain"],
        "fp32_learned": lr,
        "wall_clock_ratio_vs_fp64": f64["wall_s"] / lr["wall_s"],
        "network_gain_wall": v["fp32_plain"]["wall_s"] / lr["wall_s"],
        "error_vs_plain_fp64": v["err"],
        "training": v["train"],
        "roofline": v["roofline"], "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all,
        "cpu_baseline_uniform_1024": cpu_uniform,
        "e2e": v["e2e"], "gpu_launches": v["launches"], "clocks": v["clocks"],
        "uniform_1024": uniform,
        "canyon_plain": canyon,
        "canyon_plain_16": canyon16,
        "ensemble_full": ens,
        "scheme_variants": variants,
        "flood_speed_inflow": flood,
        "nested_dem_topography": topo,
        "level_subcycling": subcyc,
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.profile_case:
        run_profile_case(args)
    elif args.profile_valley:
        run_profile_valley(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.pair_only:
        run_pair_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
