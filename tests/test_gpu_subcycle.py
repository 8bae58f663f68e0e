"""Level subcycling on the GPU against the FP64 oracle: two-level radial
dam break and Stoker band, a three-level valley through regrids, the inflow
boundary on a subcycled forest (ghost time of each substep), one macro step
with friction from the oracle's state, the single-level equivalence with
global stepping, and still water at rest in both precisions."""
import numpy as np
import pytest

import oracle
from paper_2403_15435_gb300 import geoflood, inputs
from test_gpu_parity import assert_same_state, rel

pytestmark = pytest.mark.gpu


def cfg_of(prob, **kw):
    return inputs.Config(**{**prob.cfg.__dict__, **kw})


def two_level(prob, box, **kw):
    return cfg_of(prob, mi=prob.cfg.mi // 2, mj=prob.cfg.mj // 2, minlevel=0, maxlevel=1,
                  src_box=box, src_level=1, tag_depth=1e9, **kw)


def pair(cfg, prob):
    g = geoflood.Forest(cfg, prob.dem)
    r = oracle.OracleForest(cfg, prob.dem)
    for f in (g, r):
        f.set_state(prob.ic)
        f.regrid()
        f.set_state(prob.ic)
    assert [list(a) for a in g.patch_info()] == [list(a) for a in r.patch_info()]
    return g, r


@pytest.mark.parametrize("patch", [16, 32])
def test_two_level_radial_dam_break_matches_oracle(patch):
    # level-0 patches of 128 m (16) or 256 m (32); the box refines the 2 x 2
    # around the dam
    n = 128 if patch == 16 else 256
    prob = inputs.radial_dambreak(n, patch, dx=4.0, radius=100.0)
    box = (200.0, 320.0, 200.0, 320.0) if patch == 16 else (400.0, 620.0, 400.0, 620.0)
    cfg = two_level(prob, box, subcycle=1, manning_n=0.0)
    g, r = pair(cfg, prob)
    assert set(g.patch_info()[0]) == {0, 1}
    tg, ng = g.step(12.0)
    tr, nr = r.step(12.0)
    assert ng == nr and tg == tr
    assert_same_state(g, r)
    gi, ri = g.time(), r.time()
    assert gi["rejects"] == ri["rejects"] and gi["nclip"] == ri["nclip"]
    assert abs(g.mass() - r.mass()) <= 1e-12 * r.mass()


def test_one_macro_step_with_friction_from_oracle_state():
    prob = inputs.radial_dambreak(128, 16, dx=4.0, radius=100.0)
    cfg = two_level(prob, (200.0, 320.0, 200.0, 320.0), subcycle=1)
    g, r = pair(cfg, prob)
    r.step(6.0)
    h, hu, hv, _ = r.read()
    g.write(h, hu, hv)
    info = r.time()
    g.set_time(info["t"], info["dt_next"])
    r.step(info["t"] + 10.0, 1)
    g.step(info["t"] + 10.0, 1)
    assert_same_state(g, r)
    assert g.time()["dt_next"] == pytest.approx(r.time()["dt_next"], rel=1e-12)


def test_three_level_valley_through_regrids_matches_oracle():
    prob = inputs.v_valley(mi=4, mj=2, patch=16, minlevel=0, maxlevel=2, dem_spacing=8.0,
                           Lx=1000.0, Ly=500.0, breach_x=300.0, depth=8.0, n_gauges=6)
    cfg = cfg_of(prob, src_level=1, subcycle=1, manning_n=0.0)
    g = geoflood.Forest(cfg, prob.dem)
    r = oracle.OracleForest(cfg, prob.dem)
    g.set_state(prob.ic)
    r.set_state(prob.ic)
    g.set_gauges(prob.gauges)
    r.set_gauges(prob.gauges)
    for cycle in range(4):
        g.regrid()
        r.regrid()
        assert [list(a) for a in g.patch_info()] == [list(a) for a in r.patch_info()]
        g.step(1e9, 3)
        r.step(1e9, 3)
        assert_same_state(g, r)
    assert set(g.patch_info()[0]) == {0, 1, 2}
    og, ag = g.gauges()
    orr, ar = r.gauges()
    assert rel(og, orr) <= 1e-11
    assert np.array_equal(ag, ar)


def test_inflow_on_a_subcycled_forest_matches_oracle():
    prob = inputs.flood_speed(patch=16, minlevel=0, maxlevel=2)
    cfg = cfg_of(prob, subcycle=1)
    g = geoflood.Forest(cfg, prob.dem)
    r = oracle.OracleForest(cfg, prob.dem)
    for f in (g, r):
        f.set_state(prob.ic)
    for cycle in range(5):
        g.regrid()
        r.regrid()
        assert [list(a) for a in g.patch_info()] == [list(a) for a in r.patch_info()]
        g.step(1e9, 4)
        r.step(1e9, 4)
        assert_same_state(g, r, tol=1e-11)
    assert g.read()[0].max() > 0.0


def test_single_level_forest_equals_global_stepping():
    prob = inputs.radial_dambreak(128, 16, dx=4.0, radius=100.0)
    whole = (0.0, 1e9, 0.0, 1e9)
    a_cfg = two_level(prob, whole, dt_max=0.25, dt_initial=0.25)
    b_cfg = two_level(prob, whole, dt_max=0.5, dt_initial=0.5, subcycle=1)
    out = []
    for c in (a_cfg, b_cfg):
        g = geoflood.Forest(c, prob.dem)
        g.set_state(prob.ic)
        g.regrid()
        g.set_state(prob.ic)
        assert set(g.patch_info()[0]) == {1}
        g.step(10.0)
        out.append((g.read(), g.time()["steps"]))
    assert out[0][1] == 2 * out[1][1]
    for k in range(3):
        assert np.array_equal(out[0][0][k], out[1][0][k])


@pytest.mark.parametrize("prec", [0, 1])
def test_still_water_across_levels(prec):
    prob = inputs.lake_at_rest(64, patch=16, eta=1.0)
    cfg = two_level(prob, (0.0, 300.0, 0.0, 300.0), subcycle=1, precision=prec, eta0=1.0)
    g = geoflood.Forest(cfg, prob.dem)
    g.set_state(prob.ic)
    g.regrid()
    g.set_state(prob.ic)
    assert set(g.patch_info()[0]) == {0, 1}
    g.step(1e9, 40)
    h, hu, hv, b = g.read()
    tol = 1e-13 if prec == 0 else 2e-6
    assert np.abs(h + b - 1.0).max() <= tol
    assert np.abs(hu).max() <= (1e-13 if prec == 0 else 0.0)
    assert np.abs(hv).max() <= (1e-13 if prec == 0 else 0.0)
