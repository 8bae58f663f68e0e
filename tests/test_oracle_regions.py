"""Pins of the oracle's refinement regions (Sec. 4.1 criterion 4: regions
refined to a desired resolution between user-given minimum and maximum
levels; Sec. 6.4: places and times of interest).  Each case is built so that
the expected levels or flags follow by hand from that statement: a region's
minimum forces refinement even of dry water, its maximum caps what the other
criteria ask for, overlapping regions take the largest minimum and the
largest maximum, a region outside its time window or spanning every level
changes nothing."""
import numpy as np

import oracle
from paper_2403_15435_gb300 import inputs

INF = 1e30


def cfg_with(regions=(), **kw):
    base = dict(mi=2, mj=2, mx=4, minlevel=0, maxlevel=3, xupper=64.0, yupper=64.0,
                drytol=1e-3, dt_initial=0.1, tag_depth=1e-3, tag_speed=0.01,
                tag_deta=10.0, eta0=0.0, regions=tuple(regions))
    base.update(kw)
    return inputs.Config(**base)


def level_at(f, cfg, x, y):
    """Level of the leaf holding the point (x, y)."""
    L, X, Y = f.patch_info()
    for l, px, py in zip(L, X, Y):
        w = (cfg.xupper - cfg.xlower) / (cfg.mi << l)
        h = (cfg.yupper - cfg.ylower) / (cfg.mj << l)
        if px * w <= x < (px + 1) * w and py * h <= y < (py + 1) * h:
            return int(l)
    raise AssertionError("no leaf holds (%g, %g)" % (x, y))


def settle(f, state=None, n=6):
    """Regrid n times; state(n) gives (h, hu, hv) for n patches, rewritten
    after each regrid so the criteria see the same water everywhere."""
    for _ in range(n):
        if state is not None:
            f.write(*state(f.npatch))
        f.regrid()
    if state is not None:
        f.write(*state(f.npatch))


def moving(n, m=4):
    return (np.full((n, m, m), 1.0), np.full((n, m, m), 0.5), np.zeros((n, m, m)))


def still(n, m=4):
    return (np.full((n, m, m), 1.0), np.zeros((n, m, m)), np.zeros((n, m, m)))


def test_minimum_level_refines_dry_cells_inside_its_window():
    """Dry bed: the criteria ask for nothing, but the cells whose centres lie
    in [0, 10]^2 must reach level 2 while t is in [0, 5]; after the window
    every patch coarsens back to level 0."""
    cfg = cfg_with([(0.0, 10.0, 0.0, 10.0, 0.0, 5.0, 2, 3)])
    f = oracle.OracleForest(cfg)
    tags = f.tags()
    L, X, Y = f.patch_info()
    k0 = int(np.nonzero((X == 0) & (Y == 0))[0][0])
    assert tags[k0] == oracle.REFINE
    assert all(tags[k] == oracle.KEEP for k in range(len(tags)) if k != k0)
    settle(f)
    # level-2 cells are 2 m wide: the centres at 1, 3, ..., 9 lie in the box,
    # so the level-2 patches over [0, 16]^2 hold region cells
    for x, y in [(1.0, 1.0), (9.0, 9.0), (15.0, 1.0), (1.0, 15.0), (5.0, 12.0)]:
        assert level_at(f, cfg, x, y) == 2
    assert max(f.patch_info()[0]) == 2                     # nothing asks for 3
    before = [a.copy() for a in f.patch_info()]
    f.regrid()                                             # settled: no change
    assert all(np.array_equal(a, b) for a, b in zip(before, f.patch_info()))
    f.set_time(6.0, 0.1)                                   # the window is over
    settle(f)
    assert set(f.patch_info()[0]) == {0}


def test_window_bounds_are_inclusive():
    cfg = cfg_with([(0.0, 10.0, 0.0, 10.0, 2.0, 3.0, 1, 3)])
    f = oracle.OracleForest(cfg)
    L, X, Y = f.patch_info()
    k0 = int(np.nonzero((X == 0) & (Y == 0))[0][0])
    for t, want in [(1.999, oracle.KEEP), (2.0, oracle.REFINE), (3.0, oracle.REFINE),
                    (3.001, oracle.KEEP)]:
        f.set_time(t, 0.1)
        assert f.tags()[k0] == want, t


def test_maximum_level_caps_the_criteria():
    """Fast water everywhere asks for refinement everywhere; a region with
    maximum level 1 over the left half holds its cells at level 1: a level-1
    patch there is kept, a level-2 one coarsens, while the right half
    refines to the forest's maximum."""
    cap = [(0.0, 31.0, 0.0, 64.0, -INF, INF, 0, 1)]
    cfg = cfg_with(cap)
    f = oracle.OracleForest(cfg)
    f.write(*moving(f.npatch))
    f.regrid_flags(np.full(f.npatch, oracle.REFINE, np.uint8))   # all level 1
    f.write(*moving(f.npatch))
    L, X, Y = f.patch_info()
    tags = f.tags()
    left = X < 2                       # level-1 patches are 16 m wide
    assert set(tags[left]) == {oracle.KEEP}
    assert set(tags[~left]) == {oracle.REFINE}
    f.regrid_flags(np.full(f.npatch, oracle.REFINE, np.uint8))   # all level 2
    f.write(*moving(f.npatch))
    L, X, Y = f.patch_info()
    tags = f.tags()
    left = X < 4                       # level-2 patches are 8 m wide
    assert set(tags[left]) == {oracle.COARSEN}
    assert set(tags[~left]) == {oracle.REFINE}
    # settled: the far left at the cap, the right at maxlevel, the 2:1
    # balance bridging the two
    f2 = oracle.OracleForest(cfg)
    settle(f2, moving)
    assert level_at(f2, cfg, 2.0, 30.0) == 1
    assert level_at(f2, cfg, 60.0, 30.0) == 3
    assert level_at(f2, cfg, 40.0, 30.0) == 3
    without = oracle.OracleForest(cfg_with())
    settle(without, moving)
    assert set(without.patch_info()[0]) == {3}


def test_overlapping_regions_take_the_largest_minimum_and_maximum():
    """Dry bed, region A over the whole domain with levels [1, 1], region B
    over [0, 20]^2 with [2, 3]: the cells in both ask for level 2 (the larger
    minimum); moving water there may refine to 3 (the larger maximum) while
    A alone holds the rest at 1."""
    regs = [(0.0, 64.0, 0.0, 64.0, -INF, INF, 1, 1), (0.0, 20.0, 0.0, 20.0, -INF, INF, 2, 3)]
    cfg = cfg_with(regs)
    f = oracle.OracleForest(cfg)
    settle(f)
    assert level_at(f, cfg, 3.0, 3.0) == 2
    assert level_at(f, cfg, 50.0, 50.0) == 1
    assert max(f.patch_info()[0]) == 2
    g = oracle.OracleForest(cfg)
    settle(g, moving)
    assert level_at(g, cfg, 3.0, 3.0) == 3
    assert level_at(g, cfg, 50.0, 50.0) == 1
    assert level_at(g, cfg, 60.0, 3.0) == 1


def test_flow_grade_is_capped_by_a_region():
    """A depth grade asking for level 3 inside a region whose maximum is 2:
    refine below 2, keep at 2, coarsen from 3."""
    cfg = cfg_with([(0.0, 64.0, 0.0, 64.0, -INF, INF, 0, 2)], grades=((0, 0.5, 3),),
                   tag_speed=1e9)
    f = oracle.OracleForest(cfg)
    for lvl, want in [(0, oracle.REFINE), (1, oracle.REFINE), (2, oracle.KEEP),
                      (3, oracle.COARSEN)]:
        f.write(*still(f.npatch))
        assert set(f.patch_info()[0]) == {lvl}
        assert set(f.tags()) == {want}, lvl
        if lvl < 3:
            f.regrid_flags(np.full(f.npatch, oracle.REFINE, np.uint8))


def test_inactive_or_all_level_regions_change_nothing():
    """On a wet state of calm, moving, deep and dry patches on two levels:
    regions whose windows exclude t, and a region spanning every level over
    the whole domain, give the tags of no region at all, flag for flag."""
    rng = np.random.default_rng(5)
    base = cfg_with(grades=((0, 1.5, 2), (1, 0.3, 1)), tag_flux=0.8)

    def forest(cfg):
        f = oracle.OracleForest(cfg)
        f.regrid_flags(np.array([oracle.REFINE, oracle.KEEP, oracle.REFINE, oracle.KEEP],
                                np.uint8))
        return f

    f0 = forest(base)
    n = f0.npatch
    mode = np.array([0, 1, 2, 3, 0, 1, 2, 3, 0, 2])[:n]
    h = np.where(mode[:, None, None] == 2, 1.7, 1.0) + rng.uniform(0.0, 0.1, (n, 4, 4))
    h[mode == 3] = 1e-4
    hu = np.where(mode[:, None, None] == 1, 0.4, 0.0) * rng.uniform(0.5, 1.0, (n, 4, 4))
    hv = np.zeros((n, 4, 4))
    f0.write(h, hu, hv)
    ref = f0.tags()
    assert set(ref) == {oracle.REFINE, oracle.KEEP, oracle.COARSEN}
    for regs in ([(0.0, 64.0, 0.0, 64.0, 1.0, 2.0, 3, 3)],
                 [(0.0, 64.0, 0.0, 64.0, -INF, -1.0, 3, 3), (10.0, 20.0, 0.0, 64.0, 5.0, 9.0, 0, 0)],
                 [(0.0, 64.0, 0.0, 64.0, -INF, INF, 0, 3)]):
        f = forest(inputs.Config(**{**base.__dict__, "regions": tuple(regs)}))
        f.write(h, hu, hv)
        assert np.array_equal(f.tags(), ref), regs


def test_too_many_regions_are_refused():
    import ctypes
    reg = (0.0, 1.0, 0.0, 1.0, 0.0, 1.0, 0, 1)
    oracle.OracleForest(cfg_with([reg] * 8)).close()
    c = oracle._cfg_struct(cfg_with([reg] * 8))
    c.nregions = 9
    assert not oracle.lib().oracle_forest_new(ctypes.byref(c))
