"""Checkpoint and resume (geoflood_save / geoflood_load): a context resumed
from a checkpoint continues bit for bit as the saved one, in both
precisions, on a uniform grid with gauges, on a refined forest over nested
DEMs through regrids, with several scenarios, and with the learned tagger;
checkpoints of another configuration or cut short are refused."""
import numpy as np
import pytest

from paper_2403_15435_gb300 import geoflood, inputs

pytestmark = pytest.mark.gpu

ANG = np.linspace(0.0, 2 * np.pi, 8, endpoint=False)
GAUGES = np.stack([256.0 + 150.0 * np.cos(ANG), 256.0 + 150.0 * np.sin(ANG)], 1)


def same(a, b):
    ra, rb = a.read(), b.read()
    for x, y in zip(ra, rb):
        assert np.array_equal(x, y)
    for x, y in zip(a.gauges(), b.gauges()):
        assert np.array_equal(x, y)
    ta, tb = a.time(), b.time()
    # the clipped volume is summed with atomic additions in any order
    assert ta.pop("clipvol") == pytest.approx(tb.pop("clipvol"), rel=1e-12, abs=1e-12)
    assert ta == tb
    assert [list(v) for v in a.patch_info()] == [list(v) for v in b.patch_info()]


@pytest.mark.parametrize("prec", [0, 1])
def test_resume_on_a_uniform_grid(prec):
    prob = inputs.radial_dambreak(128, 32, dx=4.0, radius=100.0)
    prob.cfg.precision = prec
    a = geoflood.Forest(prob.cfg, prob.dem)
    a.set_state(prob.ic)
    a.set_gauges(GAUGES)
    a.step(6.0)
    blob = a.save()
    a.step(12.0)
    b = geoflood.Forest(prob.cfg, None)
    b.load(blob)
    b.step(12.0)
    same(a, b)


@pytest.mark.parametrize("prec", [0, 1])
def test_resume_through_regrids_over_nested_dems(prec):
    cfg = inputs.Config(mi=4, mj=2, mx=16, minlevel=0, maxlevel=2, xupper=1000.0,
                        yupper=500.0, drytol=1e-3, dt_initial=0.5, manning_n=0.03,
                        src_box=(250.0, 550.0, 150.0, 350.0), src_level=2,
                        tag_depth=1e-3, tag_speed=0.05, tag_deta=1e9, precision=prec)
    dems = inputs.nested_dems(cfg, 11, [None, (200.0, 600.0, 100.0, 400.0),
                                        (300.0, 400.0, 200.0, 300.0)], [20.0, 5.0, 2.0], relief=2.0)

    def ic(x, y, b):
        h = np.where(x < 350.0, np.maximum(12.0 - b, 0.0), 0.0)
        return h, np.zeros_like(h), np.zeros_like(h)

    a = geoflood.Forest(cfg, dems)
    a.set_state(ic)
    for _ in range(3):
        a.regrid()
        a.step(1e9, 5)
    blob = a.save()

    def more(f):
        for _ in range(3):
            f.regrid()
            f.step(1e9, 5)

    more(a)
    b = geoflood.Forest(cfg, None)
    b.load(blob)
    more(b)
    same(a, b)


def test_resume_with_several_scenarios():
    probs = inputs.valley_ensemble(3, precision=1)
    cfg = probs[0].cfg

    def build():
        f = geoflood.Forest(cfg, None, num_scenarios=3, max_patches=3 * 512, max_gauges=8)
        return f

    a = build()
    for k, p in enumerate(probs):
        a.set_scenario(k, p.cfg.manning_n, p.cfg.eta0)
        a.set_topo(p.dem, k)
        a.set_state(p.ic, k)
        a.set_gauges(p.gauges, k)
    a.advance(6.0, regrid_interval=4, check_interval=4)
    blob = a.save()
    a.advance(12.0, regrid_interval=4, check_interval=4)
    b = build()
    b.load(blob)
    b.advance(12.0, regrid_interval=4, check_interval=4)
    for k in range(3):
        for x, y in zip(a.read(k), b.read(k)):
            assert np.array_equal(x, y)
        ta, tb = a.time(k), b.time(k)
        assert ta.pop("clipvol") == pytest.approx(tb.pop("clipvol"), rel=1e-12, abs=1e-12)
        assert ta == tb
        for x, y in zip(a.gauges(k), b.gauges(k)):
            assert np.array_equal(x, y)


def test_resume_keeps_the_network_and_the_learned_tagger():
    prob = inputs.v_valley(mi=4, mj=2, patch=16, minlevel=0, maxlevel=2, dem_spacing=8.0,
                           Lx=1000.0, Ly=500.0, breach_x=300.0, depth=8.0, n_gauges=6)
    prob.cfg.src_level = 1
    prob.cfg.precision = 1
    prm = inputs.cnn_init(4).astype(np.float32)
    a = geoflood.Forest(prob.cfg, prob.dem)
    a.set_state(prob.ic)
    a.cnn_set_scale((4.0, 8.0, 8.0, 4.0))
    a.cnn_set_params(prm)
    a.set_tagger(geoflood.TAGGER_LEARNED, 0.5)
    a.advance(10.0, regrid_interval=8, check_interval=4, regrid_on_miss=True)
    blob = a.save()
    a.advance(25.0, regrid_interval=8, check_interval=4, regrid_on_miss=True)
    b = geoflood.Forest(prob.cfg, None)
    b.load(blob)
    assert np.array_equal(b.cnn_get_params(), prm)
    b.advance(25.0, regrid_interval=8, check_interval=4, regrid_on_miss=True)
    same(a, b)


def test_foreign_or_cut_checkpoints_are_refused():
    prob = inputs.radial_dambreak(128, 32, dx=4.0, radius=100.0)
    a = geoflood.Forest(prob.cfg, prob.dem)
    a.set_state(prob.ic)
    blob = a.save()
    other = inputs.Config(**{**prob.cfg.__dict__, "drytol": 2e-3})
    b = geoflood.Forest(other, prob.dem)
    with pytest.raises(geoflood.GeoFloodError):
        b.load(blob)
    c = geoflood.Forest(prob.cfg, prob.dem)
    with pytest.raises(geoflood.GeoFloodError):
        c.load(blob[:-17])
    with pytest.raises(geoflood.GeoFloodError):
        c.load(b"not a checkpoint")
