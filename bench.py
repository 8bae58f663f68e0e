"""Benchmark: cell-updates/s of the GeoFlood wave-propagation hot path.

Workload (one "step"): the 1024 x 1024 radial dam break of 32 x 32 patches
(dx = 2 m, 40-Gaussian seeded terrain, cylinder of radius 200 m at 5 m depth
onto a dry bed, drytol 1e-3 m, Manning 0.033, walls, CFL 0.9) run from t = 0
to t = 60 s in plain FP64: every accepted time step does the ghost fill, the
augmented Riemann solves, limited corrections, transverse terms, update,
Manning friction and the CFL control.  value = sum over accepted steps of the
interior cells updated / device time of the run, inputs resident in HBM; the
L2 is flushed (a 256 MB write) before every timed run.  e2e = the same run
through the C ABI from pinned host arrays (upload, run, read back).

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same
workload (there is no other implementation of the paper to run).
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

# DRAM bytes (read + write) of one patch_step launch on this workload, from
# the ncu captures summarised in profiles/ (launch 151 of --profile-case
# 1024, the same workload at t about 28 s, the middle of the timed run; ncu
# flushes the caches before each pass, so these are cold-cache figures).
# None when the kernel has changed since the capture.
TRAFFIC_PER_LAUNCH_FP64 = 24068864
N_CELLS = 1024
PATCH = 32
T_END = 60.0
WORKLOAD = "radial dam break 1024x1024, 32x32 patches, dx 2 m, t 0->60 s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--t-end", type=float, default=T_END)
    ap.add_argument("--profile-case", type=int, default=0,
                    help="run N x N cells of the workload for --profile-steps "
                         "steps and exit (for ncu captures; prints no JSON)")
    ap.add_argument("--profile-steps", type=int, default=20)
    ap.add_argument("--profile-precision", type=int, default=1, choices=[0, 1],
                    help="0 = FP64, 1 = FP32 deviation form")
    ap.add_argument("--profile-variant", type=int, default=0,
                    help="patch-step kernel variant (see geoflood_autotune)")
    return ap.parse_args()


def run_profile_case(args):
    """Fixed-length run of the same workload at another size (no timing)."""
    import torch
    from paper_2403_15435_gb300 import geoflood, inputs
    n = args.profile_case
    prob = inputs.radial_dambreak(n, PATCH, dx=2.0, radius=200.0 * n / N_CELLS)
    prob.cfg.precision = args.profile_precision
    f = geoflood.Forest(prob.cfg, prob.dem, max_patches=(n // PATCH) ** 2)
    f.set_state(prob.ic)
    f.set_variant(args.profile_variant)
    _, steps = f.step(1e9, args.profile_steps)
    print("profile case %d x %d: %d steps, t = %.3f s" % (n, n, steps, f.time()["t"]))


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


# FP32 deviation form: read w, hu, hv, b and the three compensation terms,
# write w, hu, hv and the compensation terms = 52 B per cell update; the
# operation count adds the compensated update (24) and the exact wet tests (8)
# to the scheme's 468.
BYTES_PER_CELL_FP32 = 52
OPS_PER_WET_CELL_FP32 = 500
FP32_LANES_PER_SM = 128
TRAFFIC_PER_LAUNCH_FP32 = 13558528
# Algorithmic work of the FP64 patch step, counted operation by operation
# from the scheme: a wet cell update takes two edge solves (74 operations
# each), two limited edge fluxes (81), two increments (9), two transverse
# splits (38), two transverse fluxes (9), the update (30) and Manning
# friction (16): 468 FP64 operations (add, sub, mul, div, sqrt, cbrt each
# counted once); a dry cell needs none.  Traffic: read h, hu, hv, b and write
# h, hu, hv = 56 B per cell update.
BYTES_PER_CELL_FP64 = 56
OPS_PER_WET_CELL_FP64 = 468
FP64_LANES_PER_SM = 2  # measured: DFMA throughput 1.20 TFLOP/s on 152 SMs
N_SM = 152


def measure(prec, args, dev, stream, world, local, gauges):
    """Time the workload in one precision: warm-up runs, then args.steps timed
    runs (L2 flushed before each), per-launch patch_step events, counters
    and the end-to-end runs through the C ABI with pinned host buffers."""
    import torch
    from paper_2403_15435_gb300 import geoflood, inputs

    prob = inputs.radial_dambreak(N_CELLS, PATCH, dx=2.0)
    prob.cfg.precision = prec
    f = geoflood.Forest(prob.cfg, prob.dem, stream=stream.cuda_stream)
    f.set_state(prob.ic)
    f.set_gauges(gauges)
    n = f.npatch
    m = prob.cfg.mx
    h0, hu0, hv0, _ = f.read()
    cells = n * m * m
    pin = lambda: torch.empty((n, m, m), dtype=torch.float64, pin_memory=True).numpy()
    H, HU, HV = pin(), pin(), pin()
    H[:], HU[:], HV[:] = h0, hu0, hv0
    OH, OHU, OHV = pin(), pin(), pin()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def reset():
        f.write(H, HU, HV)
        f.set_time(0.0, prob.cfg.dt_initial)
        f.set_gauges(gauges)

    for _ in range(args.warmup):
        reset()
        f.step(args.t_end)
    torch.cuda.synchronize(dev)
    # autotune the kernel shape on the state half way through the run (the
    # wet area grows with time; the middle is the average launch)
    reset()
    f.step(args.t_end * 0.5)
    variant, variant_ms = f.autotune(5)

    steps_list, ev = [], []
    launches0 = f.launch_count()
    cu0, wet0 = f.counters()
    # every 4th patch step and ghost fill of each captured chunk is bracketed
    # by CUDA events (every launch would add the cost of the event nodes to
    # the timed run)
    f.profile(True, every=4)
    with ClockSampler(local) as clk:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        for _ in range(args.steps):
            reset()
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            _, n_acc = f.step(args.t_end)
            b.record(stream)
            ev.append((a, b))
            steps_list.append(n_acc)
        torch.cuda.synchronize(dev)
    launches = f.launch_count() - launches0
    cu1, wet1 = f.counters()
    total_t = sum(a.elapsed_time(b) / 1e3 for a, b in ev)
    k_ms, k_n = f.profile_read("patch_step")
    g_ms, g_n = f.profile_read("ghost_fill")
    f.profile(False)
    value, total_t = replica_throughput(sum(steps_list) * cells, total_t, world, dev)
    gauge_out, arrival = f.gauges()
    final = f.read()[:3]

    e2e_t = []
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        f.write(H, HU, HV)
        f.set_time(0.0, prob.cfg.dt_initial)
        _, n_acc = f.step(args.t_end)
        f.read_into(OH, OHU, OHV)
        e2e_t.append(time.perf_counter() - t0)
    e2e = {"value": n_acc * cells * world / (sum(e2e_t) / len(e2e_t)),
           "unit": "cell-updates/s", "h2d_bytes_per_step": 3 * cells * 8,
           "d2h_bytes_per_step": 3 * cells * 8}
    f.close()
    return dict(value=value, ms_per_step=1e3 * total_t / args.steps, steps=steps_list,
                variant=variant, variant_ms=[float(x) for x in variant_ms if x == x],
                cells=cells, patches=n, launches=launches, clocks=clk.summary(),
                k_ms=k_ms, k_n=k_n, g_ms=g_ms, g_n=g_n, wet=wet1 - wet0, updates=cu1 - cu0, e2e=e2e,
                gauges=gauge_out, arrival=arrival, final=final)


AMR_T_END = 90.0
AMR_WORKLOAD = ("V-valley 2 km x 1 km, 4x2 blocks of 32x32 patches, levels 0-3 (finest dx 1.95 m), "
                "12 m reservoir, full breach at x = 350 m, n = 0.033, t 0->90 s, 8 gauges")
AMR4_T_END = 12.0
AMR4_CAP = 16 * 8 * 4 ** 4  # every patch on the finest level
AMR4_WORKLOAD = ("V-valley 4 km x 2 km, 16x8 blocks of 32x32 patches, levels 2-4 (finest dx 0.49 m), "
                 "20 m reservoir, full breach at x = 500 m, n = 0.033, first 12 s of the flood; "
                 "16 gauges on the thalweg at x = 520, 545, ..., 895 m (within the flood's reach)")
CNN_SCALE = (4.0, 8.0, 8.0, 4.0)


def measure_amr(stream):
    """The method with quadtree refinement: plain FP64 with the paper's
    regrid interval of 4 steps against the FP32 deviation form with learned
    tags and a regrid interval of 16 steps (the plain criterion checked every
    4 steps, regridding at once on a miss).  The network is trained first, on
    the plain criterion's flags from another valley.  Times are wall clock of
    the whole driver loop (steps, checks, regrids, host quadtree)."""
    import numpy as np
    import torch
    from paper_2403_15435_gb300 import geoflood, inputs

    def train_net(tr, t_end, capacity, epochs, cap=None):
        """Network trained on the plain criterion's flags from a run of tr."""
        t0 = time.perf_counter()
        f = geoflood.Forest(tr.cfg, tr.dem, max_patches=cap, stream=stream.cuda_stream)
        f.set_state(tr.ic)
        f.cnn_set_scale(CNN_SCALE)
        f.cnn_dataset(capacity)
        st = f.advance(t_end, regrid_interval=16, check_interval=4, collect=True)
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
        return prm, thr, {"samples": int(len(y)), "positives": npos, "epochs": epochs,
                          "pos_weight": pw, "threshold": thr,
                          "loss_first": float(loss[0]), "loss_last": float(loss[-1]),
                          "seconds": time.perf_counter() - t0}

    prm, thr, train = train_net(inputs.valley_2km(seed=inputs.SEED_BASE + 40, depth=10.0,
                                             breach_x=300.0, precision=1), 60.0, 60000, 40)

    def run(prec, learned, regrid, make=None, t_end=AMR_T_END, cap=None, net=None, gauges=None,
            threshold=None):
        if make is None:
            prob = inputs.valley_2km(precision=prec)
        else:
            prob = make()
            prob.cfg.precision = prec
        res = None
        for rep in range(2):  # the first run instantiates graphs and warms up
            g = geoflood.Forest(prob.cfg, prob.dem, max_patches=cap, stream=stream.cuda_stream)
            g.set_state(prob.ic)
            g.cnn_set_scale(CNN_SCALE)
            if learned:
                g.cnn_set_params(prm if net is None else net)
                g.set_tagger(geoflood.TAGGER_LEARNED, thr if threshold is None else threshold)
            g.set_gauges(prob.gauges if gauges is None else gauges)
            torch.cuda.synchronize()
            a = time.perf_counter()
            s = g.advance(t_end, regrid_interval=regrid, check_interval=4,
                          regrid_on_miss=learned)
            torch.cuda.synchronize()
            wall = time.perf_counter() - a
            out, arr = g.gauges()
            cells = s["patch_steps"] * prob.cfg.mx * prob.cfg.mx
            res = {"value": cells / wall, "unit": "cell-updates/s", "wall_s": wall,
                   "steps": s["steps"], "regrids": s["regrids"],
                   "regrids_on_miss": s["miss_regrids"], "criterion_misses": s["misses"],
                   "cell_updates": cells, "patches_at_end": g.npatch,
                   "gauge_h": out[:, 1].copy(), "arrival": arr.copy()}
            g.close()
        return res

    def compare(plain, learned):
        both = (plain["arrival"] >= 0) & (learned["arrival"] >= 0)
        err = {"gauge_depth_max_abs_m": float(np.abs(learned["gauge_h"] - plain["gauge_h"]).max()),
               "arrival_max_abs_s": float(np.abs(learned["arrival"] - plain["arrival"])[both].max())
               if both.any() else None,
               "gauges_reached": [int((plain["arrival"] >= 0).sum()),
                                  int((learned["arrival"] >= 0).sum())]}
        for r in (plain, learned):
            r.pop("gauge_h")
            r.pop("arrival")
        return err

    plain = run(0, False, 4)
    learned = run(1, True, 16)
    err = compare(plain, learned)
    # the full-size valley on three levels, over the first seconds of the
    # flood, with a network trained on the plain criterion's flags from
    # another seed of the same valley
    tr4 = inputs.v_valley(seed=inputs.SEED_BASE + 50)
    tr4.cfg.precision = 1
    prm4, thr4, train4 = train_net(tr4, AMR4_T_END, 120000, 10, cap=AMR4_CAP)
    thalweg = np.stack([520.0 + 25.0 * np.arange(16), np.full(16, 1000.0)], axis=1)
    plain4 = run(0, False, 4, make=inputs.v_valley, t_end=AMR4_T_END, cap=AMR4_CAP,
                 gauges=thalweg)
    learned4 = run(1, True, 16, make=inputs.v_valley, t_end=AMR4_T_END, cap=AMR4_CAP,
                   net=prm4, gauges=thalweg, threshold=thr4)
    err4 = compare(plain4, learned4)
    full = {"workload": AMR4_WORKLOAD, "plain_fp64_regrid4": plain4,
            "fp32_learned_regrid16": learned4,
            "speedup": learned4["value"] / plain4["value"],
            "wall_clock_ratio": plain4["wall_s"] / learned4["wall_s"],
            "error_vs_plain_fp64": err4, "training": train4,
            "timing": "wall clock around the whole driver loop, second of two runs"}
    return {"workload": AMR_WORKLOAD, "plain_fp64_regrid4": plain,
            "fp32_learned_regrid16": learned, "speedup": learned["value"] / plain["value"],
            "error_vs_plain_fp64": err, "training": train,
            "timing": "wall clock around the whole driver loop, second of two runs",
            "valley_4km_three_levels": full}


ENS_N = 64
ENS_T_END = 30.0


def measure_ensemble(stream):
    """Batched ensemble: ENS_N scenarios of the 2 km x 1 km valley (breach
    width, reservoir depth and Manning n drawn per scenario, each with its
    own terrain and quadtree) advanced together in one context, FP32
    deviation form, plain tagging with a regrid every 4 steps; against the
    same scenarios run one context at a time (8 of them, scaled)."""
    import numpy as np
    import torch
    from paper_2403_15435_gb300 import geoflood, inputs

    probs = inputs.valley_ensemble(ENS_N)
    cfg = probs[0].cfg

    def setup(ps, nscen):
        f = geoflood.Forest(cfg, None, num_scenarios=nscen, max_patches=nscen * 512,
                            max_gauges=8, stream=stream.cuda_stream)
        for k, p in enumerate(ps):
            f.set_scenario(k, p.cfg.manning_n, p.cfg.eta0)
            f.set_topo(p.dem, k)
            f.set_state(p.ic, k)
            f.set_gauges(p.gauges, k)
        return f

    def timed(f, nscen):
        torch.cuda.synchronize()
        a = time.perf_counter()
        st = f.advance(ENS_T_END, regrid_interval=4, check_interval=4)
        torch.cuda.synchronize()
        wall = time.perf_counter() - a
        cells = sum(f.counters(k)[0] for k in range(nscen))
        return st, wall, cells

    f = setup(probs[:2], 2)  # warm-up: graphs, kernels
    f.advance(2.0, regrid_interval=4, check_interval=4)
    f.close()
    f = setup(probs, ENS_N)
    st, wall, cells = timed(f, ENS_N)
    patches = [f.npatch_of(k) for k in range(ENS_N)]
    steps = [int(f.time(k)["steps"]) for k in range(ENS_N)]
    f.close()
    seq_wall, seq_cells = 0.0, 0
    for p in probs[:8]:
        g = setup([p], 1)
        _, w, c = timed(g, 1)
        seq_wall += w
        seq_cells += c
        g.close()
    return {"workload": "%d scenarios of the V-valley 2 km x 1 km (32x32 patches, levels 0-3), "
                        "breach width U[50,400] m, depth U[10,30] m, n U[0.02,0.05], t 0->%g s"
                        % (ENS_N, ENS_T_END),
            "value": cells / wall, "unit": "cell-updates/s", "wall_s": wall,
            "patches_at_end": {"total": int(sum(patches)), "min": int(min(patches)),
                               "max": int(max(patches))},
            "steps_per_scenario": {"min": min(steps), "max": max(steps)},
            "regrids": st["regrids"],
            "one_context_per_scenario": {"value": seq_cells / seq_wall, "unit": "cell-updates/s",
                                         "sample": "8 of the scenarios, one after another"},
            "timing": "wall clock around the whole driver loop (steps, checks, regrids)"}


VAR_STEPS = 96


def measure_variants(stream):
    """Scheme variants of Sec. 3.2 on the headline workload (FP32 deviation
    form and FP64): the state at t = 20 s of the default method, then
    VAR_STEPS steps of each variant from it (two graph chunks of warm-up
    first), timed with CUDA events on the library's stream; cell updates per
    second of the patch step loop.  The no-transverse variant runs at its
    stability bound (CFL 0.45), which does not change the cost of a step."""
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
    out["workload"] = WORKLOAD.replace("t 0->60 s", "t 20 s + %d steps" % VAR_STEPS)
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
               "volume_in_m3": g.mass() - v0 - g.time()["clipvol"],
               "integral_of_Q_m3": vin}
        g.close()
    res["workload"] = ("flood speed over a flat dry plain 1000 m x 2000 m, inflow 0->20 m3/s "
                       "over 20 m of the left side, 32x32 patches, levels 0-3, n 0.03, t 0->%g s"
                       % FS_T_END)
    res["timing"] = "wall clock around the whole driver loop (steps, checks, regrids), second run"
    return res


def measure_subcycle(stream):
    """Level subcycling on the AMR valley (levels 0-3, FP32 deviation form,
    plain tagging, a regrid every 4 macro steps) against one time step for
    all levels, to the same end time: wall clock of the driver loop, cell
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
            st = g.advance(AMR_T_END if rep else 10.0, regrid_interval=4, check_interval=4)
            torch.cuda.synchronize()
            wall = time.perf_counter() - a
            cu = g.counters()[0]
            out, arr = g.gauges()
            r = {"wall_s": wall, "steps": st["steps"], "regrids": st["regrids"],
                 "cell_updates": int(cu), "cell_updates_per_s": cu / wall,
                 "simulated_s_per_wall_s": AMR_T_END / wall, "gauge_h": out[:, 1].copy()}
            g.close()
        res["subcycled" if sub else "global_step"] = r
    d = float(np.abs(res["subcycled"].pop("gauge_h") - res["global_step"].pop("gauge_h")).max())
    res["gauge_depth_max_abs_diff_m"] = d
    res["speedup_wall"] = res["global_step"]["wall_s"] / res["subcycled"]["wall_s"]
    res["workload"] = AMR_WORKLOAD.replace("n = 0.033", "n = 0.033, FP32, plain tags")
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


def roofline(r, prec, peaks):
    """Roofline of the patch_step kernel from the live per-launch events:
    HBM side from the algorithmic bytes per cell update, ALU side from the
    counted operations per wet cell update; the binding side is reported."""
    avg = r["k_ms"] / 1e3 / max(1, r["k_n"])
    cells = r["cells"]
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
        traffic = TRAFFIC_PER_LAUNCH_FP64
    else:
        bytes_cell, ops_wet = BYTES_PER_CELL_FP32, OPS_PER_WET_CELL_FP32
        alu_peak = N_SM * FP32_LANES_PER_SM * mhz / 1e3            # GOP/s
        alu_src = "152 SMs x 128 FP32 lanes x %.0f MHz" % mhz
        traffic = TRAFFIC_PER_LAUNCH_FP32
    # work of an average launch: the wet fraction of all cell updates of the
    # timed runs times the cells of one launch
    ops = ops_wet * r["wet"] / max(1, r["updates"]) * cells
    alu = ops / avg / 1e9
    gbs = bytes_cell * cells / avg / 1e9
    out = {"kernel": "patch_step (%s)" % ("FP64" if prec == 0 else "FP32 deviation form"),
           "avg_launch_ms": avg * 1e3, "wet_fraction": r["wet"] / max(1, r["updates"]),
           "timed_launches": r["k_n"], "timing": "CUDA events around every 4th launch in the timed runs",
           "ghost_fill_avg_ms": r["g_ms"] / max(1, r["g_n"]),
           "alu": {"achieved": alu, "peak": alu_peak, "unit": "GOP/s", "frac": alu / alu_peak,
                   "ops_per_launch": ops, "peak_source": "derived: " + alu_src},
           "hbm": {"achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                   "frac_of_nominal_7900": gbs / 7900.0,
                   "bytes_per_launch": bytes_cell * cells, "peak_source": hbm_src}}
    side = "alu" if out["alu"]["frac"] >= out["hbm"]["frac"] else "hbm"
    out.update({"bound": side, "achieved": out[side]["achieved"], "peak": out[side]["peak"],
                "unit": out[side]["unit"], "frac": out[side]["frac"], "traffic": traffic})
    return out


def run_ours(args):
    import numpy as np
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
    # 16 gauges on rays from the cylinder centre (x, y in m)
    ang = np.linspace(0.0, 2 * np.pi, 16, endpoint=False)
    rad = np.linspace(250.0, 900.0, 16)
    gauges = np.stack([1024.0 + rad * np.cos(ang), 1024.0 + rad * np.sin(ang)], 1)

    peaks = measured_peaks()
    r32 = measure(1, args, dev, stream, world, local, gauges)
    r64 = measure(0, args, dev, stream, world, local, gauges)
    roof32 = roofline(r32, 1, peaks)
    roof64 = roofline(r64, 0, peaks)
    # error of the FP32 run against the FP64 run of the same workload
    err = {"max_abs_depth_m": float(np.abs(r32["final"][0] - r64["final"][0]).max()),
           "max_abs_momentum_m2s": float(max(np.abs(r32["final"][1] - r64["final"][1]).max(),
                                             np.abs(r32["final"][2] - r64["final"][2]).max())),
           "gauge_depth_max_abs_m": float(np.abs(r32["gauges"][:, 1] - r64["gauges"][:, 1]).max()),
           "arrival_max_abs_s": float(np.abs(r32["arrival"] - r64["arrival"]).max())}
    # the secondary workloads and the CPU baselines: one GPU only (with
    # replicas on several GPUs the headline is what scales)
    single = world == 1
    amr = measure_amr(stream) if single else None
    ens = measure_ensemble(stream) if single else None
    variants = measure_variants(stream) if single else None
    flood = measure_flood_speed(stream) if single else None
    topo = measure_topo(stream) if single else None
    subcyc = measure_subcycle(stream) if single else None
    cpu = cpu_baseline() if single else None
    cpu_all = cpu_baseline_all_cores() if single else None
    line = {
        "metric": "cell-updates/s", "value": r32["value"], "unit": "cell-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": r32["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": r32["cells"], "patches": r32["patches"],
                   "accepted_steps_per_run": r32["steps"][0],
                   "precision": "FP32 surface-deviation form (compensated update, exact wet tests)",
                   "kernel_variant": {"chosen": r32["variant"], "ms_per_launch": r32["variant_ms"],
                                      "variants": ["32x32 tile per 512-thread CTA, TMA bulk staging, 2 CTAs/SM",
                                                   "16x16 sub-tiles, 4 x 352-thread CTAs per patch",
                                                   "32x32 tile per 512-thread CTA, 1 CTA/SM (no spills)",
                                                   "32x32 tile per 1024-thread CTA, TMA bulk staging"][:len(r32["variant_ms"])]},
                   "tagging": "none: uniform single-level grid, no regrid in this workload",
                   "l2": "flushed (256 MB write) before each timed run; within a run the "
                         "working set stays in L2",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roof32, "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all,
        "e2e": r32["e2e"],
        "gpu_launches": r32["launches"], "clocks": r32["clocks"],
        "fp64": {"value": r64["value"], "ms_per_step": r64["ms_per_step"], "dtype": "f64",
                 "kernel_variant": {"chosen": r64["variant"], "ms_per_launch": r64["variant_ms"]},
                 "accepted_steps_per_run": r64["steps"][0], "roofline": roof64,
                 "e2e": r64["e2e"], "gpu_launches": r64["launches"], "clocks": r64["clocks"]},
        "fp32_vs_fp64_error": err,
        "amr_valley": amr,
        "ensemble": ens,
        "scheme_variants": variants,
        "flood_speed_inflow": flood,
        "nested_dem_topography": topo,
        "level_subcycling": subcyc,
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def cpu_baseline(budget_s=12.0):
    """The oracle as it stands on a bounded sample: a 128 x 128 window of
    the same workload (16 patches of 32 x 32 around the cylinder edge, same
    terrain and dx), stepped until the budget is spent."""
    import oracle
    from paper_2403_15435_gb300 import inputs
    prob = inputs.radial_dambreak(128, 32, dx=2.0, radius=100.0)
    f = oracle.OracleForest(prob.cfg, prob.dem)
    f.set_state(prob.ic)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < budget_s:
        _, n = f.step(1e9, 5)
        steps += n
    dt = time.perf_counter() - t0
    return {"value": steps * 128 * 128 / dt, "unit": "cell-updates/s", "cores": 1,
            "kind": "oracle", "sample": "128x128 window (16 patches of 32x32), same terrain/dx, %d steps in %.1f s" % (steps, dt)}


def _oracle_window(budget_s):
    """One host core's share of the all-cores baseline (a spawned process):
    the single-core sample, stepped until the budget is spent."""
    import oracle
    from paper_2403_15435_gb300 import inputs
    prob = inputs.radial_dambreak(128, 32, dx=2.0, radius=100.0)
    f = oracle.OracleForest(prob.cfg, prob.dem)
    f.set_state(prob.ic)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < budget_s:
        _, n = f.step(1e9, 5)
        steps += n
    return steps * 128 * 128, time.perf_counter() - t0


def cpu_baseline_all_cores(budget_s=8.0):
    """The same oracle, unchanged, on every host core at once: one spawned
    process per core, each stepping its own copy of the sample window;
    the sum of their rates."""
    import multiprocessing as mp
    n = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(n) as pool:
        res = pool.map(_oracle_window, [budget_s] * n)
    return {"value": sum(c / t for c, t in res), "unit": "cell-updates/s", "cores": n,
            "kind": "oracle", "sample": "%d processes, each the 128x128 window for %.0f s" % (n, budget_s)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2403_15435_gb300 import inputs
    prob = inputs.radial_dambreak(128, 32, dx=2.0, radius=100.0)
    f = oracle.OracleForest(prob.cfg, prob.dem)
    f.set_state(prob.ic)
    for _ in range(args.warmup):
        f.step(1e9, 2)
    t0 = time.perf_counter()
    steps = 0
    for _ in range(args.steps):
        _, n = f.step(1e9, 4)
        steps += n
    dt = time.perf_counter() - t0
    v = steps * 128 * 128 / dt
    line = {"impl": "reference", "metric": "cell-updates/s", "value": v,
            "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "128x128 window, 4 time steps per bench step"},
            "cpu_baseline": {"value": v, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                             "sample": "128x128 window (16 patches), 4 steps per bench step"},
            "e2e": {"value": v, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.profile_case:
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
