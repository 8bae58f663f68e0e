"""Pins of the oracle's composite topography from several overlapping DEMs
(Sec. 6.2): cell averages of nested bilinear surfaces against their closed
form (the integral of a bilinear function over a rectangle is its area times
the value at its centre; the composite is split by inclusion and exclusion
of the DEM extents); additivity of the cell integral (a cell's average is
the mean of its four quarters' averages, hence a coarse bed is the mean of
its children's beds); the choice of DEM by resolution, not by list order;
and a lake at rest over the composite bed through regrids."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2403_15435_gb300 import inputs
from test_oracle_pins import assemble


def bilinear_dem(coef, box, sp):
    a, b, c, d = coef
    x0, x1, y0, y1 = box
    X, Y = np.meshgrid(np.arange(x0, x1 + 0.5 * sp, sp), np.arange(y0, y1 + 0.5 * sp, sp))
    return inputs.Dem(a + b * X + c * Y + d * X * Y, x0, y0, sp, sp)


def integral(coef, r):
    """Integral of the bilinear surface over rectangle r (empty: 0)."""
    x0, x1, y0, y1 = r
    if x1 <= x0 or y1 <= y0:
        return 0.0
    a, b, c, d = coef
    xc, yc = 0.5 * (x0 + x1), 0.5 * (y0 + y1)
    return (x1 - x0) * (y1 - y0) * (a + b * xc + c * yc + d * xc * yc)


def meet(*rs):
    return (max(r[0] for r in rs), min(r[1] for r in rs),
            max(r[2] for r in rs), min(r[3] for r in rs))


CA, CB, CC = (1.0, 0.01, -0.02, 1e-4), (3.0, -0.03, 0.005, -2e-4), (-2.0, 0.02, 0.04, 3e-4)
BA, BB, BC = (0.0, 400.0, 0.0, 300.0), (100.0, 260.0, 50.0, 210.0), (180.0, 300.0, 120.0, 200.0)
DEMS = [bilinear_dem(CA, BA, 20.0), bilinear_dem(CB, BB, 5.0), bilinear_dem(CC, BC, 2.0)]


def closed_form(r):
    """C on its extent, B on its extent outside C, A elsewhere."""
    rc, rb = meet(r, BC), meet(r, BB)
    rbc = meet(r, BB, BC)
    return (integral(CC, rc) + integral(CB, rb) - integral(CB, rbc) +
            integral(CA, r) - integral(CA, rb) - integral(CA, rc) + integral(CA, rbc))


def test_composite_average_of_nested_bilinear_surfaces():
    rng = np.random.default_rng(17)
    for _ in range(300):
        xa = rng.uniform(0, 380)
        ya = rng.uniform(0, 280)
        w = rng.choice([1.3, 7.0, 31.0, 95.0]) * rng.uniform(0.5, 1.0)
        r = (xa, min(400.0, xa + w), ya, min(300.0, ya + w * rng.uniform(0.5, 1.5)))
        area = (r[1] - r[0]) * (r[3] - r[2])
        got = oracle.dems_average(DEMS, *r)
        ref = closed_form(r) / area
        assert got == pytest.approx(ref, rel=1e-12, abs=1e-12), r


def test_priority_is_by_resolution_not_by_order():
    rng = np.random.default_rng(3)
    cells = [(rng.uniform(0, 300), rng.uniform(0, 200)) for _ in range(40)]
    for perm in itertools.permutations(range(3)):
        dems = [DEMS[k] for k in perm]
        for x, y in cells:
            r = (x, x + 40.0, y, y + 40.0)
            assert oracle.dems_average(dems, *r) == oracle.dems_average(DEMS, *r)


def test_cell_integral_is_additive():
    cfg = inputs.Config(xupper=1000.0, yupper=500.0)
    dems = inputs.nested_dems(cfg, 5, [None, (200, 600, 100, 400), (300, 400, 200, 300)],
                              [20.0, 5.0, 2.0])
    rng = np.random.default_rng(8)
    for _ in range(200):
        s = rng.choice([2.0, 8.0, 31.25, 125.0])
        x = rng.uniform(0, 1000 - 2 * s)
        y = rng.uniform(0, 500 - 2 * s)
        whole = oracle.dems_average(dems, x, x + 2 * s, y, y + 2 * s)
        q = [oracle.dems_average(dems, x + i * s, x + (i + 1) * s, y + j * s, y + (j + 1) * s)
             for i in (0, 1) for j in (0, 1)]
        assert whole == pytest.approx(0.25 * ((q[0] + q[1]) + (q[2] + q[3])), rel=1e-13, abs=1e-12)


def test_single_dem_is_the_one_dem_average():
    cfg = inputs.Config(xupper=1000.0, yupper=500.0)
    d = inputs.nested_dems(cfg, 5, [None], [20.0])
    rng = np.random.default_rng(2)
    for _ in range(50):
        x, y = rng.uniform(-50, 1000), rng.uniform(-50, 500)
        r = (x, x + 17.0, y, y + 9.0)
        assert oracle.dems_average(d, *r) == oracle.dem_average(d[0], *r)


def valley_cfg(mx=16, maxlevel=1):
    return inputs.Config(mi=4, mj=2, mx=mx, minlevel=0, maxlevel=maxlevel, xupper=1000.0,
                         yupper=500.0, drytol=1e-3, dt_initial=0.5,
                         src_box=(250.0, 550.0, 150.0, 350.0), src_level=maxlevel,
                         tag_depth=1e9)


def test_coarse_bed_is_mean_of_fine_beds_with_nested_dems():
    cfg = valley_cfg(16, 1)
    dems = inputs.nested_dems(cfg, 5, [None, (200, 600, 100, 400), (300, 400, 200, 300)],
                              [20.0, 5.0, 2.0])
    c0 = inputs.Config(**{**cfg.__dict__, "minlevel": 0, "maxlevel": 0})
    c1 = inputs.Config(**{**cfg.__dict__, "minlevel": 1, "maxlevel": 1})
    bc = assemble(oracle.OracleForest(c0, dems), 3)
    bf = assemble(oracle.OracleForest(c1, dems), 3)
    mean = 0.25 * ((bf[0::2, 0::2] + bf[1::2, 0::2]) + (bf[0::2, 1::2] + bf[1::2, 1::2]))
    assert np.abs(bc - mean).max() <= 1e-12 * (1 + np.abs(bc).max())
    # the finest DEM shows: beds inside its box differ from the coarse DEM's
    bcoarse = assemble(oracle.OracleForest(c1, dems[:1]), 3)
    assert np.abs(bf - bcoarse).max() > 0.05


def test_lake_at_rest_over_nested_dems_through_regrids():
    """Still water over the composite bed stays at rest to round-off on three
    levels through regrids (the beds of every level are averages of one
    interpolant, so refinement and coarsening keep the surface flat)."""
    cfg = valley_cfg(16, 2)
    dems = inputs.nested_dems(cfg, 9, [None, (200, 600, 100, 400), (300, 400, 200, 300)],
                              [20.0, 5.0, 2.0], relief=2.0)
    eta = 30.0  # above the whole composite bed: no shoreline
    f = oracle.OracleForest(cfg, dems)

    def ic(x, y, b):
        h = np.maximum(eta - b, 0.0)
        return h, np.zeros_like(h), np.zeros_like(h)

    f.set_state(ic)
    for _ in range(3):
        f.regrid()
        f.step(1e9, 10)
    L = f.patch_info()[0]
    assert set(L) == {0, 1, 2}
    h, hu, hv, b = f.read()
    wet = h > cfg.drytol
    assert wet.all()
    assert np.abs((h + b)[wet] - eta).max() < 1e-12
    assert np.abs(hu).max() < 1e-12 and np.abs(hv).max() < 1e-12
