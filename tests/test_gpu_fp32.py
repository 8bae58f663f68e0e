"""FP32 surface-deviation path (GEOFLOOD_FP32_DEV) against the FP64 oracle.

Per step from identical inputs: |dh| <= 1e-4 m and |dhu|, |dhv| <= 1e-4 m^2/s
(the FP32 per-step bound).  Whole runs: the errors (depth, momentum, volume drift,
gauge arrival times, wet-mask and tag mismatches) are measured and bounded
loosely, since limiter switches amplify rounding differences over many
steps.  Lake at rest stays exactly at rest in FP32 (the deviation form)."""
import math

import numpy as np
import pytest

import oracle
from paper_2403_15435_gb300 import geoflood, inputs

pytestmark = pytest.mark.gpu

ABS = 1e-4


def f32(prob):
    cfg = inputs.Config(**{**prob.cfg.__dict__, "precision": 1})
    return inputs.Problem(prob.name, cfg, prob.dem, prob.ic, prob.t_end, prob.gauges)


def test_fp32_one_step_from_oracle_state():
    prob = inputs.radial_dambreak(128, 32, dx=4.0, radius=100.0)
    r = oracle.OracleForest(prob.cfg, prob.dem)
    r.set_state(prob.ic)
    r.step(8.0)
    h, hu, hv, _ = r.read()
    p32 = f32(prob)
    g = geoflood.Forest(p32.cfg, p32.dem)
    g.write(h, hu, hv)
    info = r.time()
    g.set_time(info["t"], info["dt_next"])
    r.step(info["t"] + 10.0, 1)
    g.step(info["t"] + 10.0, 1)
    a, b = g.read(), r.read()
    assert np.abs(a[0] - b[0]).max() <= ABS
    assert np.abs(a[1] - b[1]).max() <= ABS
    assert np.abs(a[2] - b[2]).max() <= ABS
    mism = int(np.count_nonzero((a[0] > prob.cfg.drytol) != (b[0] > prob.cfg.drytol)))
    assert mism <= 2, "wet masks differ in %d cells" % mism


@pytest.mark.parametrize("eta", [1.0, 0.3])
def test_fp32_lake_at_rest_is_exact(eta):
    prob = f32(inputs.lake_at_rest(128, patch=32, eta=eta))
    prob.cfg.eta0 = eta
    g = geoflood.Forest(prob.cfg, prob.dem)
    g.set_state(prob.ic)
    h0 = g.read()[0]
    g.step(1e9, 1000)
    h, hu, hv, b = g.read()
    assert np.abs(h - h0).max() <= 1e-6  # FP32 storage of w = 0 is exact
    assert np.all(hu == 0.0) and np.all(hv == 0.0)


def test_fp32_stoker_closed_form():
    from test_oracle_pins import stoker_exact
    prob = f32(inputs.stoker(128, patch=32))
    g = geoflood.Forest(prob.cfg, prob.dem)
    g.set_state(prob.ic)
    g.step(20.0)
    L, X, Y = g.patch_info()
    h = g.read()[0]
    row = np.zeros(128)
    for k in range(len(X)):
        if Y[k] == 0:
            row[X[k] * 32:(X[k] + 1) * 32] = h[k, 0]
    x = (np.arange(128) + 0.5) * 5.0
    he, *_ = stoker_exact(x, 20.0)
    assert np.abs(row - he).sum() / np.abs(he).sum() <= 0.02


def test_fp32_run_error_report_against_fp64():
    """Radial dam break on terrain for 12 s: FP32 vs the FP64 oracle."""
    prob = inputs.radial_dambreak(128, 32, dx=4.0, radius=100.0)
    r = oracle.OracleForest(prob.cfg, prob.dem)
    r.set_state(prob.ic)
    p32 = f32(prob)
    g = geoflood.Forest(p32.cfg, p32.dem)
    g.set_state(prob.ic)
    m0 = g.mass()
    r.step(12.0)
    g.step(12.0)
    a, b = g.read(), r.read()
    dh = np.abs(a[0] - b[0]).max()
    dm = max(np.abs(a[1] - b[1]).max(), np.abs(a[2] - b[2]).max())
    info = g.time()
    drift = abs(g.mass() - m0 - info["clipvol"]) / m0
    print("FP32 vs FP64 after 12 s: max |dh| %.2e m, max |dq| %.2e m2/s, volume drift %.2e"
          % (dh, dm, drift))
    assert dh <= 0.05 and dm <= 0.2
    assert drift <= 1e-6


def test_fp32_amr_valley_runs_and_tags_agree_mostly():
    prob = inputs.v_valley(mi=4, mj=2, patch=16, minlevel=0, maxlevel=2,
                           dem_spacing=8.0, Lx=1000.0, Ly=500.0, breach_x=300.0,
                           depth=8.0, n_gauges=6)
    prob.cfg.src_level = 1
    p32 = f32(prob)
    g = geoflood.Forest(p32.cfg, p32.dem)
    g.set_state(prob.ic)
    r = oracle.OracleForest(prob.cfg, prob.dem)
    r.set_state(prob.ic)
    g.set_gauges(prob.gauges)
    r.set_gauges(prob.gauges)
    mismatch = 0
    for cycle in range(4):
        tg, tr = g.tags(), r.tags()
        mismatch += int(np.count_nonzero(tg != tr))
        g.regrid()
        r.regrid()
        if len(g.patch_info()[0]) != len(r.patch_info()[0]):
            break
        g.step(1e9, 4)
        r.step(1e9, 4)
    print("FP32 tag mismatches over 4 regrids: %d" % mismatch)
    assert mismatch <= 2
    og, ag = g.gauges()
    orr, ar = r.gauges()
    assert np.abs(og[:, 1] - orr[:, 1]).max() <= 0.05


def _two_level(prob, box, precision):
    """The problem on a two-level forest: level 1 inside box, level 0 elsewhere."""
    cfg = inputs.Config(**{**prob.cfg.__dict__, "mi": prob.cfg.mi // 2,
                           "mj": prob.cfg.mj // 2, "minlevel": 0, "maxlevel": 1,
                           "src_box": box, "src_level": 1, "tag_depth": 1e9,
                           "precision": precision})
    return inputs.Problem(prob.name, cfg, prob.dem, prob.ic, prob.t_end)


RING = np.ones((36, 36), bool)  # the ghost ring of a 32 x 32 patch's tile
RING[2:-2, 2:-2] = False


def _ghost_gap(tg, tr):
    """Largest |difference| of (h, hu, hv) over the tiles, and over their ghost rings."""
    d = np.abs(tg[:, :3] - tr[:, :3])
    return float(d.max()), float(d[..., RING].max())


def test_fp32_ghost_cells_across_levels_match_oracle():
    """The FP32 ghost operators (copy, 2x2 mean and limited interpolation of
    the stored surface, in FP32) against the FP64 oracle's on the same
    stored state: after the full ghost fill that follows a host write, and
    after one step, whose level-change ghosts the per-step ghost kernel
    writes.  Smooth, partly dry state; within the FP32 per-step bound."""
    base = inputs.radial_dambreak(128, 32, dx=4.0, radius=150.0)
    box = (0.0, 200.0, 0.0, 300.0)
    p32, p64 = _two_level(base, box, 1), _two_level(base, box, 0)

    def ic(x, y, b):
        # the bed spans 4.5-19 m: a surface near 13 m leaves wet and dry
        # cells on both sides of the level interface
        h = np.maximum(0.0, 13.0 + 1.5 * np.sin(x / 40.0) * np.cos(y / 55.0) - b)
        return h, 0.2 * h * np.cos(y / 30.0), -0.1 * h
    g = geoflood.Forest(p32.cfg, p32.dem)
    r = oracle.OracleForest(p64.cfg, p64.dem)
    g.regrid()
    r.regrid()
    assert [list(a) for a in g.patch_info()] == [list(a) for a in r.patch_info()]
    assert len(set(int(x) for x in g.patch_info()[0])) == 2
    g.set_state(ic)
    for stage in ("host write", "one step"):
        if stage == "one step":
            g.step(1e9, 1)
        h, hu, hv, _ = g.read()
        r.write(h, hu, hv)
        r.ghost_fill()
        tr = r.read_tiles()
        wet = tr[:, 0][:, RING] > p64.cfg.drytol
        assert 0.2 <= wet.mean() <= 0.8, "the ghost rings must hold wet and dry cells"
        whole, ring = _ghost_gap(g.read_tiles(), tr)
        print("%s: max |d| %.2e over the tiles, %.2e over the ghost rings" % (stage, whole, ring))
        assert whole <= ABS


def test_fp32_lake_at_rest_across_levels_is_exact():
    """Still water over a submerged bump on a two-level forest (the level
    interface crosses the bump) stays exactly still in FP32 without
    subcycling: the level-change ghosts carry the stored surface, whose
    means and limited slopes are exactly zero."""
    prob = _two_level(inputs.lake_at_rest(128, patch=32, eta=1.0), (0.0, 300.0, 0.0, 300.0), 1)
    prob.cfg.eta0 = 1.0
    g = geoflood.Forest(prob.cfg, prob.dem)
    g.regrid()
    assert len(set(int(x) for x in g.patch_info()[0])) == 2
    g.set_state(prob.ic)
    h0 = g.read()[0]
    g.step(1e9, 200)
    h, hu, hv, _ = g.read()
    assert np.abs(h - h0).max() <= 1e-6
    assert np.all(hu == 0.0) and np.all(hv == 0.0)
