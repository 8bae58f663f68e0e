"""Pins of the oracle's level subcycling (level L takes 2^(L - minlevel)
steps per macro step, coarser levels interpolated in time for the ghost
cells): equivalence with single-level stepping where the two must agree bit
for bit (a forest whose leaves all sit on one level, stepped with the fixed
fine time step both ways), still water and uniform flow kept exactly across
level changes, the volume change bounded by the flux mismatch at level
changes, the Stoker dam break's closed form with a refined band, and
agreement with global stepping on a two-level radial dam break."""
import math

import numpy as np
import pytest

import oracle
from paper_2403_15435_gb300 import inputs
from test_oracle_pins import stoker_exact


def forest(prob, **kw):
    cfg = inputs.Config(**{**prob.cfg.__dict__, **kw})
    f = oracle.OracleForest(cfg, prob.dem)
    f.set_state(prob.ic)
    f.regrid()
    f.set_state(prob.ic)
    return f


def two_level(prob, box, **kw):
    return forest(prob, mi=prob.cfg.mi // 2, mj=prob.cfg.mj // 2, minlevel=0, maxlevel=1,
                  src_box=box, src_level=1, tag_depth=1e9, **kw)


def test_single_level_forest_steps_like_global_stepping():
    """All leaves on level 1 of a 0..1 forest: a macro step is two fine steps
    of DT / 2; with the time step fixed (dt_max below the CFL limit) that is
    global stepping with dt = DT / 2, bit for bit."""
    prob = inputs.radial_dambreak(128, 32, dx=4.0, radius=100.0)
    whole = (0.0, 1e9, 0.0, 1e9)
    a = two_level(prob, whole, dt_max=0.25, dt_initial=0.25)
    b = two_level(prob, whole, dt_max=0.5, dt_initial=0.5, subcycle=1)
    assert set(a.patch_info()[0]) == {1}
    a.step(10.0)
    b.step(10.0)
    assert a.time()["steps"] == 2 * b.time()["steps"]
    ra, rb = a.read(), b.read()
    for k in range(3):
        assert np.array_equal(ra[k], rb[k])


@pytest.mark.parametrize("eta", [1.0])
def test_still_water_stays_still_across_levels(eta):
    prob = inputs.lake_at_rest(64, patch=16, eta=eta)
    f = two_level(prob, (0.0, 300.0, 0.0, 300.0), subcycle=1)
    assert set(f.patch_info()[0]) == {0, 1}
    h0 = f.read()[0]
    f.step(1e9, 40)
    h, hu, hv, b = f.read()
    assert np.abs(h + b - eta).max() < 1e-13
    assert np.abs(hu).max() < 1e-13 and np.abs(hv).max() < 1e-13


def test_uniform_flow_is_steady_across_levels():
    prob = inputs.stoker(128, patch=16)
    prob.cfg.bc = (inputs.BC_EXTRAP,) * 4
    prob.ic = lambda x, y, b: (np.full_like(x, 1.5), np.full_like(x, 0.9), np.full_like(x, -0.6))
    f = two_level(prob, (170.0, 310.0, 170.0, 310.0), subcycle=1)
    assert set(f.patch_info()[0]) == {0, 1}
    f.step(1e9, 30)
    h, hu, hv, _ = f.read()
    assert np.abs(h - 1.5).max() < 1e-13
    assert np.abs(hu - 0.9).max() < 1e-13 and np.abs(hv + 0.6).max() < 1e-13


def test_stoker_with_a_refined_band_matches_closed_form():
    """The refined band (level 1) spans the shock's path; with walls and
    rows kept identical, the depth along a row approaches Stoker's solution
    like global stepping does, and the volume error from the level changes
    is small."""
    errs = {}
    for sub in (0, 1):
        prob = inputs.stoker(128, patch=16)
        f = two_level(prob, (300.0, 460.0, 0.0, 640.0), subcycle=sub)
        assert set(f.patch_info()[0]) == {0, 1}
        m0 = f.mass()
        f.step(20.0)
        L, X, Y = f.patch_info()
        h = f.read()[0]
        x, row = [], []
        for k in range(len(L)):
            if Y[k] != 0:
                continue
            dx = 5.0 * (2 ** (1 - L[k]))
            for i in range(16):
                x.append((X[k] * 16 + i + 0.5) * dx)
                row.append(h[k, 0, i])
        x, row = np.array(x), np.array(row)
        o = np.argsort(x)
        x, row = x[o], row[o]
        w = np.gradient(x)
        he, *_ = stoker_exact(x, 20.0)
        errs[sub] = np.sum(w * np.abs(row - he)) / np.sum(w * he)
        assert abs(f.mass() - m0) <= 2e-3 * m0
    assert errs[1] <= 0.02
    assert errs[1] <= 1.3 * errs[0] + 1e-3


def _coarse_depths(f, n0, m):
    """Depths of a 0..1 forest on the level-0 grid (level-1 patches averaged
    2x2): n0 x n0 coarse cells in patches of m."""
    L, X, Y = f.patch_info()
    h = f.read()[0]
    out = np.zeros((n0, n0))
    for k in range(len(L)):
        c = h[k] if L[k] == 0 else h[k].reshape(m // 2, 2, m // 2, 2).mean(axis=(1, 3))
        w = m if L[k] == 0 else m // 2
        out[Y[k] * w:(Y[k] + 1) * w, X[k] * w:(X[k] + 1) * w] = c
    return out


def test_radial_dam_break_close_to_global_stepping():
    """Two-level radial dam break over terrain onto a dry bed: against the
    same problem refined everywhere, the subcycled forest's error is of the
    order of the globally stepped one's (the fronts cross the coarse/fine
    interface, where the two place a front up to a coarse cell apart)."""
    prob = inputs.radial_dambreak(128, 16, dx=4.0, radius=100.0)
    box = (160.0, 352.0, 160.0, 352.0)
    a = two_level(prob, box)
    b = two_level(prob, box, subcycle=1)
    c = two_level(prob, (0.0, 1e9, 0.0, 1e9))
    assert set(a.patch_info()[0]) == {0, 1}
    for f in (a, b, c):
        f.step(12.0)
    ha, hb, hc = (_coarse_depths(f, 64, 16) for f in (a, b, c))
    ea, eb = np.abs(ha - hc), np.abs(hb - hc)
    assert eb.mean() <= 2.0 * ea.mean()
    assert eb.mean() <= 0.025 * hc.mean()
    assert eb.max() <= 0.15 * hc.max()
    assert np.abs(ha - hb).mean() <= 0.015 * hc.mean()
    # fewer coarse updates: the coarse level took half as many steps
    assert b.time()["steps"] < a.time()["steps"]
