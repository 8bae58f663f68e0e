"""Pins of the oracle's quadtree pieces (Sec. 4, Sec. 4.1, Sec. 6.2): ghost
exchange between levels, regrid with 2:1 balance, the plain tagger, gauges and
lake at rest / volume across refinement.  Each compares with a closed form
(linear fields are reproduced exactly by limited linear interpolation and by
bilinear sampling), an invariant (balance, coverage, conservation) or a
hand-checkable case."""
import numpy as np
import pytest

import oracle
from paper_2403_15435_gb300 import inputs


def two_level_cfg(**kw):
    base = dict(mi=2, mj=2, mx=8, minlevel=0, maxlevel=1, xupper=160.0,
                yupper=160.0, drytol=1e-3, dt_initial=0.1, tag_depth=1e9,
                src_box=(0.0, 79.0, 0.0, 79.0), src_level=1)
    base.update(kw)
    return inputs.Config(**base)


def refined_forest(cfg, dem=None):
    """Forest whose lower-left block is refined to level 1 by the source box."""
    f = oracle.OracleForest(cfg, dem)
    f.regrid()
    return f


def levels(f):
    return f.patch_info()[0]


def test_source_box_refines_one_block():
    f = refined_forest(two_level_cfg())
    L, X, Y = f.patch_info()
    assert sorted(zip(L, X, Y)) == sorted([(0, 1, 0), (0, 0, 1), (0, 1, 1),
                                          (1, 0, 0), (1, 1, 0), (1, 0, 1), (1, 1, 1)])


def linear_state(cfg, L, X, Y, a=(2.0, 0.01, -0.004), mu=(0.3, 0.002, 0.001), mv=(-0.1, 0.0, 0.003)):
    xs, ys = inputs.cell_centres(cfg, L, X, Y)
    eta = a[0] + a[1] * xs + a[2] * ys
    hu = mu[0] + mu[1] * xs + mu[2] * ys
    hv = mv[0] + mv[1] * xs + mv[2] * ys
    return xs, ys, eta, hu, hv


def test_ghosts_exact_for_linear_fields_across_levels():
    """With the surface and momenta linear and everything wet, copy, 2x2
    averaging and minmod-limited linear interpolation all reproduce the linear
    function at the ghost-cell centres."""
    cfg = two_level_cfg(bc=(inputs.BC_EXTRAP,) * 4)
    f = refined_forest(cfg)
    L, X, Y = f.patch_info()
    xs, ys, eta, hu, hv = linear_state(cfg, L, X, Y)
    b = f.read()[3]
    f.write(eta - b, hu, hv)
    tiles = f.read_tiles()
    m, T = cfg.mx, cfg.mx + 4
    idx = np.arange(-2, m + 2)
    for k in range(len(L)):
        dx = 160.0 / (2 * m << L[k])
        xc = (X[k] * m + idx + 0.5) * dx
        yc = (Y[k] * m + idx + 0.5) * dx
        XX, YY = np.meshgrid(xc, yc)
        # coarse cells on the domain edge take a zero slope across the edge
        # (their outside neighbour is a boundary ghost), so stay one coarse
        # cell away from the boundary
        inside = (XX > 10) & (XX < 150) & (YY > 10) & (YY < 150)
        e = (2.0 + 0.01 * XX - 0.004 * YY)
        got_eta = tiles[k, 0] + tiles[k, 3]
        assert np.abs((got_eta - e)[inside]).max() < 1e-12
        assert np.abs((tiles[k, 1] - (0.3 + 0.002 * XX + 0.001 * YY))[inside]).max() < 1e-12
        assert np.abs((tiles[k, 2] - (-0.1 + 0.003 * YY))[inside]).max() < 1e-12


def test_lake_at_rest_across_levels_and_regrid():
    """A lake at rest over a bump stays at rest across a coarse/fine interface
    and through refine + coarsen regrids (Sec. 6.2: the topography averages are
    conservative so the surface stays flat)."""
    cfg = two_level_cfg(xupper=640.0, yupper=640.0, mx=16, src_box=(0.0, 300.0, 0.0, 300.0))
    prob = inputs.lake_at_rest(64, eta=1.0)
    f = refined_forest(cfg, prob.dem)
    f.set_state(prob.ic)
    f.step(1e9, 50)
    h, hu, hv, b = f.read()
    assert np.abs(h + b - 1.0).max() < 1e-13
    assert np.abs(hu).max() < 1e-13 and np.abs(hv).max() < 1e-13
    # move the source box: the lower-left block coarsens, the upper-right refines
    f.cfg.src_box = (340.0, 640.0, 340.0, 640.0)
    g = oracle.OracleForest(f.cfg, prob.dem)
    g.set_state(prob.ic)
    g.regrid()
    g.step(1e9, 20)
    h, hu, hv, b = g.read()
    assert np.abs(h + b - 1.0).max() < 1e-13
    assert np.abs(hu).max() < 1e-13


def test_refine_and_coarsen_conserve_volume_when_wet():
    """Refinement by limited interpolation of the surface and coarsening by
    averaging keep the volume of a wet state (sum of the four fine depths =
    four times the coarse depth)."""
    cfg = two_level_cfg(xupper=640.0, yupper=640.0, mx=16, src_box=(0.0, 300.0, 0.0, 300.0),
                        tag_depth=1e9)
    prob = inputs.lake_at_rest(64, eta=3.0)

    def ic(x, y, b):
        h = 3.0 - b + 0.2 * np.sin(x / 50.0) * np.cos(y / 70.0)
        return h, 0.1 * h, -0.05 * h

    f = oracle.OracleForest(cfg, prob.dem)
    f.set_state(ic)
    m0 = f.mass()
    f.regrid()
    assert len(f.patch_info()[0]) == 7
    assert abs(f.mass() - m0) / m0 < 1e-13
    f.cfg.src_box = (0.0, -1.0, 0.0, -1.0)
    g_cfg = inputs.Config(**{**cfg.__dict__, "src_box": (0.0, -1.0, 0.0, -1.0)})
    # coarsen back: rebuild the oracle with no source box and copy the state
    g = oracle.OracleForest(g_cfg, prob.dem)
    g.set_state(ic)
    m1 = g.mass()
    assert abs(m1 - m0) / m0 < 1e-13


def _check_balanced_cover(f, cfg):
    L, X, Y = f.patch_info()
    maxl = cfg.maxlevel
    W, H = cfg.mi << maxl, cfg.mj << maxl
    lvl = -np.ones((H, W), int)
    for l, x, y in zip(L, X, Y):
        s = maxl - l
        blk = lvl[y << s:(y + 1) << s, x << s:(x + 1) << s]
        assert np.all(blk == -1), "leaves overlap"
        blk[:] = l
    assert np.all(lvl >= 0), "leaves do not cover the domain"
    # 2:1 across faces and corners
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            a = lvl[max(0, dy):H + min(0, dy), max(0, dx):W + min(0, dx)]
            b = lvl[max(0, -dy):H + min(0, -dy), max(0, -dx):W + min(0, -dx)]
            assert np.abs(a - b).max() <= 1
    return lvl


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_regrid_keeps_cover_and_two_to_one_balance(seed):
    """Repeated regrids driven by a moving point source keep the leaves a
    disjoint cover of the domain with 2:1 balance across faces and corners,
    and refine the source to the requested level."""
    rng = np.random.default_rng(seed)
    cfg = inputs.Config(mi=3, mj=2, mx=4, minlevel=0, maxlevel=4, xupper=300.0,
                        yupper=200.0, tag_depth=1e9, src_level=4)
    for _ in range(6):
        x, y = rng.uniform(0, 270), rng.uniform(0, 170)
        cfg.src_box = (x, x + 30.0, y, y + 30.0)  # holds a level-0 cell centre
        x, y = x + 15.0, y + 15.0
        f = oracle.OracleForest(cfg)
        for _ in range(5):
            f.regrid()
        lvl = _check_balanced_cover(f, cfg)
        X = min(int(x / 300.0 * (3 << 4)), (3 << 4) - 1)
        Y = min(int(y / 200.0 * (2 << 4)), (2 << 4) - 1)
        assert lvl[Y, X] == 4


def test_tagger_criteria():
    """Criterion 1 (wet) with 3 (speed) or the surface departure, and 4 (the
    source region), per cell; a patch refines if any cell is flagged, coarsens
    if none is and it is above minlevel, and never refines past maxlevel."""
    cfg = inputs.Config(mi=2, mj=1, mx=4, minlevel=0, maxlevel=1, xupper=80.0,
                        yupper=40.0, tag_depth=1e-3, tag_speed=0.01, tag_deta=0.05,
                        eta0=1.0)
    f = oracle.OracleForest(cfg)
    h = np.full((2, 4, 4), 1.0)
    hu = np.zeros_like(h)
    hv = np.zeros_like(h)
    hu[1, 2, 3] = 0.02  # speed 0.02 > 0.01 in patch 1 only
    f.write(h, hu, hv)
    L, X, Y = f.patch_info()
    tags = f.tags()
    k1 = int(np.nonzero(X == 1)[0][0])
    assert tags[k1] == oracle.REFINE and tags[1 - k1] == oracle.KEEP
    h2 = h.copy()
    h2[1 - k1, 0, 0] = 1.06  # surface 6 cm above eta0
    f.write(h2, np.zeros_like(h), hv)
    tags = f.tags()
    assert tags[1 - k1] == oracle.REFINE and tags[k1] == oracle.KEEP
    h3 = h.copy()
    h3[:] = 1e-4  # dry: nothing flagged even though eta departs
    f.write(h3, np.zeros_like(h), hv)
    assert list(f.tags()) == [oracle.KEEP, oracle.KEEP]


def test_tagger_criteria_2_and_5():
    """Criterion 2 (velocity-depth product: |hu| above tag_flux refines even
    when the speed is below tag_speed) and criterion 5 (flow grades: a wet
    cell deeper than the grade's depth asks for exactly the grade's level:
    refine below it, keep at it, coarsen above it)."""
    cfg = inputs.Config(mi=2, mj=1, mx=4, minlevel=0, maxlevel=3, xupper=80.0,
                        yupper=40.0, tag_depth=1e-3, tag_speed=0.01, tag_deta=10.0,
                        eta0=0.0, tag_flux=0.05)
    f = oracle.OracleForest(cfg)
    h = np.full((2, 4, 4), 10.0)
    hu = np.zeros_like(h)
    hu[0, 1, 1] = 0.06   # speed 0.006 < tag_speed, |hu| = 0.06 > tag_flux
    hu[1, 1, 1] = 0.04   # speed 0.004, |hu| = 0.04 below both
    f.write(h, hu, np.zeros_like(h))
    L, X, Y = f.patch_info()
    k0 = int(np.nonzero(X == 0)[0][0])
    tags = f.tags()
    assert tags[k0] == oracle.REFINE and tags[1 - k0] == oracle.KEEP  # level 0: keep
    # flow grades: depth > 5 m asks for level 2, speed > 0.005 m/s for level 1
    cfg2 = inputs.Config(**{**cfg.__dict__, "tag_flux": float("inf"), "tag_speed": 1.0,
                            "grades": ((0, 5.0, 2), (1, 0.005, 1))})
    f2 = oracle.OracleForest(cfg2)
    f2.write(h, hu, np.zeros_like(h))
    assert list(f2.tags()) == [oracle.REFINE, oracle.REFINE]   # level 0 < 2
    f2.regrid()
    f2.regrid()                                                # now at level 2
    L2 = f2.patch_info()[0]
    assert set(L2) == {2}
    assert set(f2.tags()) == {oracle.KEEP}                     # the grade's level
    # shallow water: only the speed grade (level 1) applies -> coarsen from 2
    n = len(L2)
    f2.write(np.full((n, 4, 4), 1.0), np.full((n, 4, 4), 0.01), np.zeros((n, 4, 4)))
    assert set(f2.tags()) == {oracle.COARSEN}
    # dry cells ask for nothing, whatever the grades
    f2.write(np.full((n, 4, 4), 1e-4), np.zeros((n, 4, 4)), np.zeros((n, 4, 4)))
    assert set(f2.tags()) == {oracle.COARSEN}


def test_gauges_bilinear_exact_and_arrival():
    """Gauges sample the finest leaf bilinearly, ghosts included: a linear
    field is reproduced exactly anywhere, also next to a coarse/fine edge."""
    cfg = two_level_cfg(bc=(inputs.BC_EXTRAP,) * 4)
    f = refined_forest(cfg)
    L, X, Y = f.patch_info()
    xs, ys, eta, hu, hv = linear_state(cfg, L, X, Y)
    b = f.read()[3]
    f.write(eta - b, hu, hv)
    pts = np.array([[10.0, 10.0], [79.0, 33.3], [81.0, 41.0], [120.0, 148.0], [15.5, 78.9]])
    f.set_gauges(pts)
    out, arr = f.gauges()
    x, y = pts[:, 0], pts[:, 1]
    np.testing.assert_allclose(out[:, 4], 2.0 + 0.01 * x - 0.004 * y, atol=1e-12)
    np.testing.assert_allclose(out[:, 2], 0.3 + 0.002 * x + 0.001 * y, atol=1e-12)
    assert np.all(arr == 0.0)  # wet at registration time t = 0


def test_uniformly_refined_forest_equals_single_level_forest():
    """A forest refined everywhere to level 1 advances bit-for-bit like a forest
    created at level 1 (leaf bookkeeping, Morton order, ghost copy)."""
    prob = inputs.radial_dambreak(64, 16, dx=8.0, radius=100.0)
    c1 = inputs.Config(**{**prob.cfg.__dict__, "mi": 2, "mj": 2, "minlevel": 0,
                          "maxlevel": 1, "src_box": (0.0, 1e9, 0.0, 1e9),
                          "src_level": 1, "tag_depth": 1e9})
    c2 = inputs.Config(**{**c1.__dict__, "minlevel": 1})
    fa = oracle.OracleForest(c1, prob.dem)
    fa.regrid()
    fb = oracle.OracleForest(c2, prob.dem)
    assert [list(a) for a in fa.patch_info()] == [list(a) for a in fb.patch_info()]
    fa.set_state(prob.ic)
    fb.set_state(prob.ic)
    fa.step(5.0)
    fb.step(5.0)
    for a, b in zip(fa.read(), fb.read()):
        assert np.array_equal(a, b)


def _rippled_refinement(dry_column=None, ripple=0.25):
    """Coarse wet state over a bed rippled at the coarse cell size (a 10 m
    sine averages to zero over each coarse cell but not over its fine halves)
    and the forest after one refinement of the lower-left block."""
    cfg = two_level_cfg(mx=8)
    xn = np.arange(0.0, 160.0 + 1e-9, 1.25)
    X, Y = np.meshgrid(xn, xn)
    dem = inputs.Dem(z=ripple * np.sin(2 * np.pi * X / 10.0) + 0.001 * Y,
                     x0=0.0, y0=0.0, dx=1.25, dy=1.25)
    f = oracle.OracleForest(cfg, dem)

    def ic(x, y, b):
        h = 0.6 + 0.05 * np.sin(x / 17.0) * np.cos(y / 23.0) - b
        if dry_column is not None:
            h = np.where(np.floor(x / 10.0) == dry_column, 0.0, h)
        u = 1.0 + 0.05 * np.cos(y / 13.0)
        v = -0.5 + 0.05 * np.sin(x / 19.0)
        return h, h * u, h * v

    f.set_state(ic)
    L, X0, Y0 = f.patch_info()
    h, hu, hv, _ = f.read()
    C = np.zeros((4, 16, 16))
    for k in range(len(L)):
        for a, v in enumerate((h, hu, hv)):
            C[a, Y0[k] * 8:(Y0[k] + 1) * 8, X0[k] * 8:(X0[k] + 1) * 8] = v[k]
    f.regrid()
    L, X1, Y1 = f.patch_info()
    h, hu, hv, _ = f.read()
    F = np.zeros((3, 16, 16))
    for k in range(len(L)):
        if L[k] == 1:
            for a, v in enumerate((h, hu, hv)):
                F[a, Y1[k] * 8:(Y1[k] + 1) * 8, X1[k] * 8:(X1[k] + 1) * 8] = v[k]
    assert (L == 1).sum() == 4
    return C, F


def test_refinement_creates_no_new_velocity_extremes():
    """A fine cell much shallower than its coarse parent (the bed's ripple)
    must not inherit the parent's momentum whole: every refined velocity lies
    in the range of the velocities of the parent's 3x3 neighbourhood (limited
    interpolation, Sec. 6.2; the velocity bound is the reading that the
    method's interpolation keeps the flow's speeds)."""
    C, F = _rippled_refinement()
    uc, vc = C[1] / C[0], C[2] / C[0]
    checked = 0
    for J in range(16):
        for I in range(16):
            jc, ic = J >> 1, I >> 1
            sl = (slice(max(jc - 1, 0), jc + 2), slice(max(ic - 1, 0), ic + 2))
            uf, vf = F[1, J, I] / F[0, J, I], F[2, J, I] / F[0, J, I]
            tol = 1e-12
            assert uc[sl].min() - tol <= uf <= uc[sl].max() + tol
            assert vc[sl].min() - tol <= vf <= vc[sl].max() + tol
            checked += 1
    assert checked == 256
    # the ripple makes the fine depths differ from the coarse ones by far more
    # than the surface variation, so the bound is exercised
    assert np.abs(F[0] - np.kron(C[0, :8, :8], np.ones((2, 2)))).max() > 0.1


def test_refinement_next_to_dry_keeps_velocity_and_momentum():
    """Beside a dry coarse cell the fine surface is the coarse one and each
    fine cell carries the coarse cell's velocity: the four children hold the
    parent's volume and momentum (the fine beds average to the coarse bed and
    no depth is clamped here)."""
    C, F = _rippled_refinement(dry_column=3)
    seen = 0
    for jc in range(8):
        for ic in (2, 4):
            ch = F[:, 2 * jc:2 * jc + 2, 2 * ic:2 * ic + 2]
            assert (ch[0] > 0.1).all()
            assert np.allclose(ch[1] / ch[0], C[1, jc, ic] / C[0, jc, ic], rtol=1e-13, atol=0)
            assert np.allclose(ch[2] / ch[0], C[2, jc, ic] / C[0, jc, ic], rtol=1e-13, atol=0)
            for a in range(3):
                assert abs(ch[a].sum() - 4 * C[a, jc, ic]) <= 1e-12 * abs(4 * C[a, jc, ic])
            seen += 1
    assert seen == 16
    # the dry column stays dry and still
    assert (F[:, :, 6:8] == 0).all()


@pytest.mark.parametrize("dry_column", [None, 3])
def test_refinement_with_emerging_children_keeps_momentum_and_speeds(dry_column):
    """A 1 m ripple lifts some children above the parent's surface (their
    depth is clamped at zero, so the volume grows, as the surface-based
    interpolation keeps still water still).  The momentum still is the
    parent's, split in proportion to the children's depths, and no child is
    faster than the fastest cell of the parent's neighbourhood."""
    C, F = _rippled_refinement(dry_column=dry_column, ripple=1.0)
    clamped = 0
    for jc in range(8):
        for ic in range(8):
            if not C[0, jc, ic] > 1e-3:
                continue
            ch = F[:, 2 * jc:2 * jc + 2, 2 * ic:2 * ic + 2]
            clamped += int((ch[0] == 0).any())
            if ((ch[0] > 0) & (ch[0] <= 1e-3)).any():
                continue
            for a in (1, 2):
                assert abs(ch[a].sum() - 4 * C[a, jc, ic]) <= 1e-12 * abs(4 * C[a, jc, ic])
            sl = (slice(max(jc - 1, 0), jc + 2), slice(max(ic - 1, 0), ic + 2))
            wet = C[0][sl] > 1e-3
            vmax = np.abs(C[1:3][(slice(None),) + sl][:, wet] / C[0][sl][wet]).max()
            wf = ch[0] > 0
            assert (np.abs(ch[1:3][:, wf] / ch[0][wf]) <= vmax * (1 + 1e-12)).all()
    assert clamped >= 8


def test_valley_floods_keep_physical_speeds_through_regrids():
    """Eight valleys of the 64-scenario ensemble as one context runs them
    (the first valley's configuration, each with its own Manning n, surface
    and terrain; a regrid whenever 4 steps have passed in some scenario)
    advanced 2 s, then two regrid + 4-step cycles: no cell deeper than
    drytol moves faster than 60 m/s.  The interpolation of momentum into new
    fine cells (Sec. 6.2) must not hand a shallow child its deep parent's
    momentum: copying it gave 200-1300 m/s in these valleys."""
    probs = inputs.valley_ensemble(64, precision=0)
    cfg = probs[0].cfg
    fs = []
    for p in probs[:8]:
        c = inputs.Config(**{**cfg.__dict__, "manning_n": p.cfg.manning_n, "eta0": p.cfg.eta0})
        f = oracle.OracleForest(c, p.dem)
        f.set_state(p.ic)
        fs.append(f)

    def fastest():
        out = []
        for f in fs:
            h, hu, hv, _ = f.read()
            wet = h > 1e-3
            sp = np.sqrt(hu[wet] ** 2 + hv[wet] ** 2) / h[wet]
            assert np.isfinite(sp).all()
            out.append(float(sp.max()) if sp.size else 0.0)
        return max(out)

    since = 0
    while True:
        before = [f.time()["steps"] for f in fs]
        for f in fs:
            f.step(2.0, 4 - since)
        since += max(f.time()["steps"] - b for f, b in zip(fs, before))
        if all(f.time()["t"] >= 2.0 for f in fs):
            break
        if since >= 4:
            for f in fs:
                f.regrid()
            since = 0
    assert fastest() < 60.0
    for _ in range(2):
        for f in fs:
            f.regrid()
        assert fastest() < 60.0
        for f in fs:
            f.step(1e9, 4)
        assert fastest() < 60.0
