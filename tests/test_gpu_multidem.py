"""Composite topography from several overlapping DEMs (Sec. 6.2) on the GPU
against the FP64 oracle: beds of every tile cell (ghost cells included) on
three levels through regrids, independence of the DEMs' order, a dam break
over the composite bed through regrids, and still water at rest in both
precisions."""
import numpy as np
import pytest

import oracle
from paper_2403_15435_gb300 import geoflood, inputs
from test_gpu_parity import assert_same_state, rel

pytestmark = pytest.mark.gpu

BOXES = [None, (200.0, 600.0, 100.0, 400.0), (300.0, 400.0, 200.0, 300.0)]
SPACINGS = [20.0, 5.0, 2.0]


def valley(mx=16, maxlevel=2, precision=0, eta0=0.0):
    cfg = inputs.Config(mi=4, mj=2, mx=mx, minlevel=0, maxlevel=maxlevel, xupper=1000.0,
                        yupper=500.0, drytol=1e-3, dt_initial=0.5, manning_n=0.03,
                        src_box=(250.0, 550.0, 150.0, 350.0), src_level=maxlevel,
                        tag_depth=1e-3, tag_speed=0.05, tag_deta=1e9,
                        precision=precision, eta0=eta0)
    dems = inputs.nested_dems(cfg, 11, BOXES, SPACINGS, relief=2.0)
    return cfg, dems


def pond(x, y, b):
    h = np.where(x < 350.0, np.maximum(12.0 - b, 0.0), 0.0)
    return h, np.zeros_like(h), np.zeros_like(h)


@pytest.mark.parametrize("mx", [16, 32])
def test_beds_match_oracle_on_three_levels(mx):
    cfg, dems = valley(mx)
    g = geoflood.Forest(cfg, dems)
    r = oracle.OracleForest(cfg, dems)
    g.set_state(pond)
    r.set_state(pond)
    for _ in range(2):
        g.regrid()
        r.regrid()
    assert [list(a) for a in g.patch_info()] == [list(a) for a in r.patch_info()]
    assert set(g.patch_info()[0]) == {0, 1, 2}
    tg, tr = g.read_tiles(), r.read_tiles()
    assert rel(tg[:, 3], tr[:, 3]) <= 1e-14


def test_dem_order_does_not_matter():
    cfg, dems = valley(16, 1)
    a = geoflood.Forest(cfg, dems)
    b = geoflood.Forest(cfg, dems[::-1])
    assert np.array_equal(a.read_tiles()[:, 3], b.read_tiles()[:, 3])


def test_dam_break_over_nested_dems_matches_oracle():
    cfg, dems = valley(16, 2)
    g = geoflood.Forest(cfg, dems)
    r = oracle.OracleForest(cfg, dems)
    g.set_state(pond)
    r.set_state(pond)
    for cycle in range(4):
        g.regrid()
        r.regrid()
        assert [list(a) for a in g.patch_info()] == [list(a) for a in r.patch_info()]
        g.step(1e9, 8)
        r.step(1e9, 8)
        assert_same_state(g, r, tol=1e-11)
    assert g.read()[1].max() > 0.1


@pytest.mark.parametrize("prec", [0, 1])
def test_still_water_over_nested_dems(prec):
    eta = 30.0
    cfg, dems = valley(16, 2, precision=prec, eta0=eta)
    g = geoflood.Forest(cfg, dems)

    def ic(x, y, b):
        h = eta - b
        return h, np.zeros_like(h), np.zeros_like(h)

    g.set_state(ic)
    for _ in range(3):
        g.regrid()
        g.step(1e9, 10)
    h, hu, hv, b = g.read()
    tol = 1e-12 if prec == 0 else 2e-5
    assert np.abs(h + b - eta).max() <= tol
    assert np.abs(hu).max() <= (1e-12 if prec == 0 else 0.0)
    assert np.abs(hv).max() <= (1e-12 if prec == 0 else 0.0)
