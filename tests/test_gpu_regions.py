"""Refinement regions (Sec. 4.1 criterion 4: regions refined between
user-given minimum and maximum levels; Sec. 6.4: places and times of
interest) on the GPU against the FP64 oracle through the C ABI.

Tolerances: FP64 tags and patch lists bit-exact, states within 1e-11 of the
field's largest magnitude after steps and regrids (the FP64 bound, as in the
other trajectory tests); FP32 (its own single-precision criterion, the
regions' geometry in FP64 like the oracle's) at most three tag mismatches
over the run."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2403_15435_gb300 import geoflood, inputs

pytestmark = pytest.mark.gpu

# (x0, x1, y0, y1, t0, t1, minlevel, maxlevel); edges off the patch lines so
# that patches of every level are crossed as well as covered
REGIONS = (
    (612.3, 811.7, 141.9, 352.4, 0.0, 3.5, 2, 3),   # dry ground refined early on
    (0.0, 251.3, 0.0, 500.0, -1e30, 1e30, 0, 1),    # the reservoir held at level <= 1
    (703.1, 1000.0, 0.0, 247.7, 2.5, 100.0, 1, 2),  # overlaps the first one
)


def valley(patch, prec=0, regions=REGIONS):
    prob = inputs.v_valley(mi=4, mj=2, patch=patch, minlevel=0, maxlevel=3,
                           dem_spacing=8.0, Lx=1000.0, Ly=500.0, breach_x=300.0,
                           depth=8.0, n_gauges=6)
    prob.cfg.src_level = 1
    prob.cfg.regions = tuple(regions)
    prob.cfg.precision = prec
    return prob


def rel(a, b):
    return float(np.abs(a - b).max()) / max(1.0, float(np.abs(b).max()))


@pytest.mark.parametrize("patch", [16, 32])
def test_region_tags_and_regrids_match_oracle(patch):
    """FP64: tags bit-exact, leaf lists identical and states equal through
    step/regrid cycles across the regions' time windows (the first region
    ends at 3.5 s, the third starts at 2.5 s)."""
    prob = valley(patch)
    g = geoflood.Forest(prob.cfg, prob.dem)
    r = oracle.OracleForest(prob.cfg, prob.dem)
    g.set_state(prob.ic)
    r.set_state(prob.ic)
    seen = set()
    times = []
    for cycle in range(12):
        tg, tr = g.tags(), r.tags()
        seen.update(int(x) for x in tr)
        assert np.array_equal(tg, tr), "tags differ in cycle %d" % cycle
        g.regrid()
        r.regrid()
        assert [list(a) for a in g.patch_info()] == [list(a) for a in r.patch_info()]
        g.step(1e9, 4)
        r.step(1e9, 4)
        times.append(r.time()["t"])
        a, b = g.read(), r.read()
        for k in range(3):
            assert rel(a[k], b[k]) <= 1e-11
    assert times[0] < 2.5 and times[-1] > 3.5     # both window edges crossed
    assert {oracle.REFINE, oracle.KEEP, oracle.COARSEN} <= seen
    # the reservoir stays at level <= 1 away from the region's edge (where
    # the 2:1 balance with the refined breach may step the levels down)
    L, X, Y = r.patch_info()
    w = 1000.0 / (4 << L)
    assert np.all(L[(X + 1) * w <= 251.3 - 125.0] <= 1)


def test_region_tags_fp32():
    """FP32 deviation form: the same run, tags against the oracle's at most
    three mismatches (single-precision criterion at threshold ties)."""
    prob = valley(16)
    p32 = valley(16, prec=1)
    g = geoflood.Forest(p32.cfg, p32.dem)
    r = oracle.OracleForest(prob.cfg, prob.dem)
    g.set_state(prob.ic)
    r.set_state(prob.ic)
    mismatch = 0
    for cycle in range(8):
        tg, tr = g.tags(), r.tags()
        mismatch += int(np.count_nonzero(tg != tr))
        g.regrid()
        r.regrid()
        if [list(a) for a in g.patch_info()] != [list(a) for a in r.patch_info()]:
            break
        g.step(1e9, 4)
        r.step(1e9, 4)
    assert cycle >= 2
    assert mismatch <= 3


@pytest.mark.parametrize("prec", [0, 1])
def test_learned_tags_are_bounded_by_regions(prec):
    """A network that asks for refinement everywhere refines every patch to
    the finest level except where a region caps the level: inside the
    reservoir region (level <= 1) no patch goes beyond level 1 away from the
    region's edge (next to it the 2:1 balance with the level-3 patches
    outside forces level 2), while every patch outside reaches level 3."""
    prob = valley(16, prec=prec, regions=(REGIONS[1],))
    g = geoflood.Forest(prob.cfg, prob.dem)
    g.set_state(prob.ic)
    prm = np.zeros(geoflood.cnn_nparam(), np.float32)
    prm[-1] = 10.0                                  # head bias: logit 10
    g.cnn_set_params(prm)
    g.set_tagger(geoflood.TAGGER_LEARNED, 0.5)
    for _ in range(5):
        g.regrid()
    L, X, Y = g.patch_info()
    w = 1000.0 / (4 << L)
    x_hi = (X + 1) * w
    inside = x_hi <= 251.3 - 125.0     # a level-1 patch away from the edge
    assert np.any(inside) and np.all(L[inside] <= 1)
    assert np.all(L[X * w >= 251.3] == 3)
    # without the region the same network refines the reservoir as well
    free = valley(16, prec=prec, regions=())
    h = geoflood.Forest(free.cfg, free.dem)
    h.set_state(free.ic)
    h.cnn_set_params(prm)
    h.set_tagger(geoflood.TAGGER_LEARNED, 0.5)
    for _ in range(5):
        h.regrid()
    assert set(h.patch_info()[0]) == {3}


def test_invalid_regions_are_refused():
    base = valley(16)
    for bad in [(0.0, 1.0, 0.0, 1.0, 0.0, 1.0, 2, 1),     # minimum above maximum
                (0.0, 1.0, 0.0, 1.0, 0.0, 1.0, 0, 4),     # beyond the forest's maxlevel
                (1.0, 0.0, 0.0, 1.0, 0.0, 1.0, 0, 1),     # empty box
                (0.0, 1.0, 0.0, 1.0, 2.0, 1.0, 0, 1)]:    # empty window
        cfg = inputs.Config(**{**base.cfg.__dict__, "regions": (bad,)})
        with pytest.raises(geoflood.GeoFloodError):
            geoflood.Forest(cfg, base.dem)
    c = geoflood.config_struct(base.cfg)
    c.nregions = 9
    h = ctypes.c_void_p()
    assert geoflood.lib().geoflood_init_forest(ctypes.byref(c), None, ctypes.byref(h)) == -1
