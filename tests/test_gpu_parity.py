"""GPU (sm_103a) vs the FP64 oracle through the C ABI.

Tolerance (FP64): max-norm difference per field <= 1e-12 relative to the
field's largest magnitude (the FP64 bound); wet masks (h > drytol), tags and
patch lists bit-exact.  Both sides run without fused multiply-add, so most
results agree to the last bit; the bound leaves room for the one libm
difference (cbrt in the friction term)."""
import numpy as np
import pytest

import oracle
from paper_2403_15435_gb300 import geoflood, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12


def rel(a, b):
    return float(np.abs(a - b).max()) / max(1.0, float(np.abs(b).max()))


def pair(prob, **kw):
    g = geoflood.Forest(prob.cfg, prob.dem, **kw)
    r = oracle.OracleForest(prob.cfg, prob.dem)
    g.set_state(prob.ic)
    r.set_state(prob.ic)
    return g, r


def assert_same_state(g, r, tol=TOL, s=0):
    a = g.read(s)
    b = r.read()
    for k, name in enumerate(("h", "hu", "hv", "b")):
        e = rel(a[k], b[k])
        assert e <= tol, "%s differs by %.3e" % (name, e)
    drytol = g.cfg.drytol
    assert np.array_equal(a[0] > drytol, b[0] > drytol), "wet masks differ"


def test_one_step_from_dumped_oracle_state():
    prob = inputs.radial_dambreak(128, 32, dx=4.0, radius=100.0)
    g, r = pair(prob)
    r.step(8.0)
    h, hu, hv, _ = r.read()
    g.write(h, hu, hv)
    info = r.time()
    g.set_time(info["t"], info["dt_next"])
    r.step(info["t"] + 10.0, 1)
    g.step(info["t"] + 10.0, 1)
    assert_same_state(g, r)
    gi = g.time()
    ri = r.time()
    assert gi["t"] == pytest.approx(ri["t"], rel=1e-14)
    assert gi["dt_next"] == pytest.approx(ri["dt_next"], rel=TOL)


def test_trajectory_parity_radial_dam_break_on_terrain():
    prob = inputs.radial_dambreak(128, 32, dx=4.0, radius=100.0)
    g, r = pair(prob)
    tg, ng = g.step(12.0)
    tr, nr = r.step(12.0)
    assert ng == nr and tg == tr
    assert_same_state(g, r, tol=1e-11)
    assert g.time()["rejects"] == r.time()["rejects"]
    m_g, m_r = g.mass(), r.mass()
    assert abs(m_g - m_r) <= 1e-12 * m_r


def test_stoker_on_gpu_matches_oracle():
    prob = inputs.stoker(128, patch=32)
    g, r = pair(prob)
    g.step(20.0)
    r.step(20.0)
    assert_same_state(g, r)
    h = g.read()[0]
    assert np.all(g.read()[2] == 0.0)


def test_lake_at_rest_on_gpu():
    prob = inputs.lake_at_rest(128, patch=32, eta=0.3)
    g = geoflood.Forest(prob.cfg, prob.dem)
    g.set_state(prob.ic)
    h0 = g.read()[0]
    g.step(1e9, 1000)
    h, hu, hv, b = g.read()
    wet = h > prob.cfg.drytol
    assert np.abs((h + b)[wet] - 0.3).max() <= 1e-13
    assert np.abs(h - h0).max() <= 1e-13
    assert np.abs(hu).max() <= 1e-13 and np.abs(hv).max() <= 1e-13


def test_mass_on_gpu_equals_clipped_volume():
    prob = inputs.radial_dambreak(128, 32, dx=4.0, radius=100.0)
    g = geoflood.Forest(prob.cfg, prob.dem)
    g.set_state(prob.ic)
    m0 = g.mass()
    g.step(15.0)
    info = g.time()
    assert abs(g.mass() - m0 - info["clipvol"]) <= 1e-13 * m0


def two_level(prob, box):
    cfg = inputs.Config(**{**prob.cfg.__dict__, "mi": prob.cfg.mi // 2,
                           "mj": prob.cfg.mj // 2, "minlevel": 0, "maxlevel": 1,
                           "src_box": box, "src_level": 1, "tag_depth": 1e9})
    return inputs.Problem(prob.name, cfg, prob.dem, prob.ic, prob.t_end)


def test_ghost_fill_across_levels_matches_oracle():
    """Ghost cells of every patch (copy, 2x2 average, limited interpolation,
    walls, corners) after a regrid, compared cell by cell."""
    base = inputs.radial_dambreak(128, 32, dx=4.0, radius=150.0)
    prob = two_level(base, (0.0, 200.0, 0.0, 300.0))

    def ic(x, y, b):
        # the bed spans 4.5-19 m: a surface near 13 m leaves wet and dry
        # cells on both sides of the level interface
        h = np.maximum(0.0, 13.0 + 1.5 * np.sin(x / 40.0) * np.cos(y / 55.0) - b)
        return h, 0.2 * h * np.cos(y / 30.0), -0.1 * h
    prob.ic = ic
    g = geoflood.Forest(prob.cfg, prob.dem)
    r = oracle.OracleForest(prob.cfg, prob.dem)
    g.regrid()
    r.regrid()
    assert [list(a) for a in g.patch_info()] == [list(a) for a in r.patch_info()]
    g.set_state(ic)
    r.set_state(ic)
    tg, tr = g.read_tiles(), r.read_tiles()
    ring = np.ones(tr.shape[-2:], bool)
    ring[2:-2, 2:-2] = False
    wet = tr[:, 0][:, ring] > prob.cfg.drytol
    assert 0.2 <= wet.mean() <= 0.8, "the ghost rings must hold wet and dry cells"
    assert rel(tg, tr) <= 1e-14


@pytest.mark.parametrize("patch", [16, 32])
def test_regrid_and_tags_match_oracle(patch):
    """Tags bit-exact, identical leaf lists (2:1 balance, Morton order) and the
    same data after repeated step/regrid cycles on a V-valley breach."""
    prob = inputs.v_valley(mi=4, mj=2, patch=patch, minlevel=0, maxlevel=2,
                           dem_spacing=8.0, Lx=1000.0, Ly=500.0, breach_x=300.0,
                           depth=8.0, n_gauges=6)
    prob.cfg.src_level = 1
    g, r = pair(prob)
    g.set_gauges(prob.gauges)
    r.set_gauges(prob.gauges)
    for cycle in range(4):
        assert np.array_equal(g.tags(), r.tags()), "tags differ in cycle %d" % cycle
        g.regrid()
        r.regrid()
        assert [list(a) for a in g.patch_info()] == [list(a) for a in r.patch_info()]
        g.step(1e9, 4)
        r.step(1e9, 4)
        assert_same_state(g, r, tol=1e-11)
    og, ag = g.gauges()
    orr, ar = r.gauges()
    assert rel(og, orr) <= 1e-11
    assert np.array_equal(ag, ar)


@pytest.mark.parametrize("prec", [0, 1])
def test_criteria_2_and_5_match_oracle(prec):
    """Refinement criteria 2 (|hu| above tag_flux) and 5 (flow grades by
    depth and by speed) on the valley breach: FP64 tags bit-exact with the
    oracle through step/regrid cycles; FP32 (its own single-precision
    criterion) at most a few tag mismatches."""
    prob = inputs.v_valley(mi=4, mj=2, patch=16, minlevel=0, maxlevel=3,
                           dem_spacing=8.0, Lx=1000.0, Ly=500.0, breach_x=300.0,
                           depth=8.0, n_gauges=6)
    prob.cfg.src_level = 1
    prob.cfg.tag_speed = 0.5       # leave room for the other criteria
    prob.cfg.tag_deta = 0.5
    prob.cfg.tag_flux = 0.2
    prob.cfg.grades = ((0, 3.0, 2), (1, 0.1, 1))
    g, r = pair(prob)
    if prec:
        p32 = inputs.Problem(prob.name, inputs.Config(**{**prob.cfg.__dict__, "precision": 1}),
                             prob.dem, prob.ic, prob.t_end, prob.gauges)
        g = geoflood.Forest(p32.cfg, p32.dem)
        g.set_state(prob.ic)
    mismatch = 0
    seen = set()
    for cycle in range(5):
        tg, tr = g.tags(), r.tags()
        seen.update(int(x) for x in tr)
        if prec:
            mismatch += int(np.count_nonzero(tg != tr))
        else:
            assert np.array_equal(tg, tr), "tags differ in cycle %d" % cycle
        g.regrid()
        r.regrid()
        if [list(a) for a in g.patch_info()] != [list(a) for a in r.patch_info()]:
            assert prec, "patch lists differ"
            break
        g.step(1e9, 6)
        r.step(1e9, 6)
    assert mismatch <= 3
    # the depth grade (> 3 m: level 2) refines the still reservoir, which the
    # source box alone keeps at level 1
    L, X, Y = r.patch_info()
    x_lo = X * (1000.0 / (4 * 2 ** L))  # left edge of each patch
    assert np.any((L == 2) & (x_lo < 250.0))
    assert oracle.REFINE in seen


def test_all_dry_domain_is_a_fixed_point():
    prob = inputs.radial_dambreak(64, 32, dx=8.0, radius=0.0)
    g = geoflood.Forest(prob.cfg, prob.dem)
    g.set_state(prob.ic)
    g.set_time(0.0, 0.25)
    t, n = g.step(1.0)
    assert n == 4 and t == 1.0
    h, hu, hv, _ = g.read()
    assert np.all(h == 0) and np.all(hu == 0) and np.all(hv == 0)
    assert g.time()["dt_next"] == 0.25


def test_ragged_forest_and_extrapolation_boundaries():
    """Non-square block arrangement (3x2 blocks of 16), open boundaries."""
    prob = inputs.radial_dambreak(96, 16, dx=5.0, radius=80.0)
    prob.cfg.mi, prob.cfg.mj = 6, 4
    prob.cfg.yupper = 320.0
    prob.cfg.bc = (inputs.BC_EXTRAP, inputs.BC_WALL, inputs.BC_EXTRAP, inputs.BC_WALL)
    g, r = pair(prob)
    g.step(6.0)
    r.step(6.0)
    assert_same_state(g, r, tol=1e-11)


def test_batched_scenarios_match_independent_oracle_runs():
    """Three scenarios with different Manning coefficients advance in the
    same launches, each with its own dt."""
    prob = inputs.radial_dambreak(64, 32, dx=8.0, radius=120.0)
    g = geoflood.Forest(prob.cfg, prob.dem, num_scenarios=3)
    ns = [0.0, 0.03, 0.06]
    for s, n in enumerate(ns):
        g.set_scenario(s, n, 0.0)
        g.set_state(prob.ic, s)
    g.step(6.0)
    for s, n in enumerate(ns):
        cfg = inputs.Config(**{**prob.cfg.__dict__, "manning_n": n})
        r = oracle.OracleForest(cfg, prob.dem)
        r.set_state(prob.ic)
        r.step(6.0)
        a = g.read(s)
        b = r.read()
        for k in range(3):
            assert rel(a[k], b[k]) <= 1e-11
        assert g.time(s)["steps"] == r.time()["steps"]


def test_full_size_1024_sampled_patches():
    """The 1024x1024 radial dam break (32x32 patches, dx = 2 m, 40-Gaussian
    terrain) in the benchmark's launch configuration: after 40 steps, one more
    step is checked patch by patch on a sample, the oracle stepping each
    sampled tile (ghosts included) with the same dt."""
    prob = inputs.radial_dambreak(1024, 32, dx=2.0)
    g = geoflood.Forest(prob.cfg, prob.dem)
    g.set_state(prob.ic)
    g.step(1e9, 40)
    info = g.time()
    tiles = g.read_tiles()
    L, X, Y = g.patch_info()
    g.step(info["t"] + 1e9, 1)
    assert g.time()["rejects"] == info["rejects"]
    after = g.read()
    rng = np.random.default_rng(7)
    c = 16  # patches around the cylinder edge and random ones
    ring = [k for k in range(len(X)) if 12 <= X[k] <= 19 and 12 <= Y[k] <= 19]
    sample = list(rng.choice(ring, 8, replace=False)) + list(rng.choice(len(X), 8, replace=False))
    dx = 2.0
    for k in sample:
        t = tiles[k]
        hn, hun, hvn, cm, nc = oracle.step_grid(t[0], t[1], t[2], t[3], dx, dx,
                                                info["dt_next"], drytol=prob.cfg.drytol,
                                                manning_n=prob.cfg.manning_n)
        for f, ref in enumerate((hn, hun, hvn)):
            e = rel(after[f][k], ref[2:-2, 2:-2])
            assert e <= TOL, "patch %d field %d differs by %.3e" % (k, f, e)


@pytest.mark.parametrize("prec", [0, 1])
def test_kernel_variants_agree_bitwise(prec):
    """The autotuner's variants (whole 32x32 tile per CTA with TMA staging,
    16x16 sub-tiles, other thread counts and register budgets) compute every
    cell with the same operations, so the states agree bit for bit."""
    prob = inputs.radial_dambreak(128, 32, dx=4.0, radius=100.0)
    prob.cfg.precision = prec
    g = geoflood.Forest(prob.cfg, prob.dem)
    g.set_state(prob.ic)
    best, ms = g.autotune(3)
    nvar = int(np.count_nonzero(np.isfinite(ms)))
    assert nvar >= 3 and 0 <= best < nvar and np.all(ms[:nvar] > 0)
    states = []
    for variant in range(nvar):
        g = geoflood.Forest(prob.cfg, prob.dem)
        g.set_state(prob.ic)
        g.set_variant(variant)
        g.step(10.0)
        states.append(g.read())
    for v in range(1, nvar):
        for a, b in zip(states[0], states[v]):
            assert np.array_equal(a, b), "variant %d differs" % v


@pytest.mark.parametrize("prec", [0, 1])
def test_kernel_variants_agree_on_the_full_workload(prec):
    """Every variant on the 1024 x 1024 radial dam break for 60 s (300
    steps: water reaching tiles that were dry and unchanged, sub-tiles, the
    wet-first launch order), bit for bit against variant 0."""
    prob = inputs.radial_dambreak(1024, 32, dx=2.0)
    prob.cfg.precision = prec
    g = geoflood.Forest(prob.cfg, prob.dem)
    nvar = int(np.count_nonzero(np.isfinite(g.autotune(1)[1])))
    ang = np.linspace(0.0, 2 * np.pi, 16, endpoint=False)
    rad = np.linspace(250.0, 900.0, 16)
    gauges = np.stack([1024.0 + rad * np.cos(ang), 1024.0 + rad * np.sin(ang)], 1)
    ref = None
    for variant in range(nvar):
        g = geoflood.Forest(prob.cfg, prob.dem)
        g.set_state(prob.ic)
        g.set_gauges(gauges)
        g.set_variant(variant)
        # several calls: the work list restarts at each
        g.step(20.0)
        g.step(60.0)
        st = list(g.read()) + list(g.gauges()) + [np.array([g.time()["steps"]])]
        if ref is None:
            ref = st
            continue
        for a, b in zip(st, ref):
            assert np.array_equal(a, b), "variant %d differs" % variant


@pytest.mark.parametrize("prec", [0, 1])
def test_regrid_with_scenarios_at_different_buffer_parities(prec):
    """Scenarios that took odd and even numbers of steps hold their latest
    states in different buffers of the shared patch slots; regrids and
    steps after that leave every scenario as it is when run alone (bit for
    bit), and equal to the oracle in FP64."""
    prob = inputs.v_valley(mi=4, mj=2, patch=16, minlevel=0, maxlevel=2,
                           dem_spacing=8.0, Lx=1000.0, Ly=500.0, breach_x=300.0,
                           depth=8.0, n_gauges=6)
    prob.cfg.src_level = 1
    prob.cfg.precision = prec
    ns = [0.0, 0.03, 0.1]

    def start(forest, s, n):
        forest.set_scenario(s, n, prob.cfg.eta0)
        forest.set_state(prob.ic, s)

    g = geoflood.Forest(prob.cfg, prob.dem, num_scenarios=len(ns))
    alone = [geoflood.Forest(prob.cfg, prob.dem) for _ in ns]
    refs = []
    for s, n in enumerate(ns):
        start(g, s, n)
        start(alone[s], 0, n)
        cfg = inputs.Config(**{**prob.cfg.__dict__, "manning_n": n, "precision": 0})
        r = oracle.OracleForest(cfg, prob.dem)
        r.set_state(prob.ic)
        refs.append(r)
    for f in [g] + alone + refs:
        f.regrid()
    for s in range(len(ns)):
        g.set_state(prob.ic, s)
        alone[s].set_state(prob.ic)
        refs[s].set_state(prob.ic)
    ops = [("step", 2.0, 1 << 30), ("regrid",), ("step", 1e9, 4), ("regrid",),
           ("step", 1e9, 3), ("regrid",), ("step", 1e9, 2)]
    for k, op in enumerate(ops):
        for f in [g] + alone + refs:
            f.regrid() if op[0] == "regrid" else f.step(op[1], op[2])
        if k == 0:
            parities = {g.time(s)["steps"] % 2 for s in range(len(ns))}
            assert parities == {0, 1}, "the scenarios must end on both buffer parities"
        for s in range(len(ns)):
            assert [list(a) for a in g.patch_info(s)] == [list(a) for a in alone[s].patch_info()]
            a, b = g.read(s), alone[s].read()
            for x, y in zip(a, b):
                assert np.array_equal(x, y), "scenario %d differs from its lone run after %s" % (s, op)
            assert g.time(s)["steps"] == alone[s].time()["steps"]
            if prec == 0:
                assert [list(a) for a in g.patch_info(s)] == [list(a) for a in refs[s].patch_info()]
                c = refs[s].read()
                for x, y in zip(a, c):
                    assert rel(x, y) <= 1e-11


def test_regrid_beyond_capacity_fails_and_leaves_the_forest_usable():
    """A regrid that needs more patches than the context holds returns
    GEOFLOOD_ERR_CAPACITY and changes nothing: the context keeps its forest
    and then steps exactly as the oracle does on the unrefined forest."""
    base = inputs.radial_dambreak(64, 16, dx=8.0, radius=120.0)
    prob = two_level(base, (0.0, 1e9, 0.0, 1e9))  # every patch asks to refine
    g, r = pair(prob, max_patches=4)
    before = [list(a) for a in g.patch_info()]
    assert len(before[0]) == 4
    with pytest.raises(geoflood.GeoFloodError) as e:
        g.regrid()
    assert e.value.code == -8
    assert [list(a) for a in g.patch_info()] == before
    g.step(1e9, 6)
    r.step(1e9, 6)
    assert g.time()["steps"] == r.time()["steps"]
    assert_same_state(g, r, tol=1e-11)


@pytest.mark.parametrize("bad", [{"mx": 24}, {"minlevel": 2, "maxlevel": 1}, {"drytol": 0.0},
                                 {"cfl_desired": 0.9, "cfl_max": 0.5}, {"precision": 7}])
def test_invalid_configuration_is_refused(bad):
    """Patch sizes other than 16 and 32, an inverted level range, a
    non-positive dry tolerance, cfl_max below cfl_desired and unknown
    precisions are refused at creation with GEOFLOOD_ERR_ARG."""
    prob = inputs.radial_dambreak(64, 16, dx=8.0, radius=120.0)
    cfg = inputs.Config(**{**prob.cfg.__dict__, **bad})
    with pytest.raises(geoflood.GeoFloodError) as e:
        geoflood.Forest(cfg, prob.dem)
    assert e.value.code == -1


def test_bad_call_arguments_are_refused_and_the_context_still_steps():
    """A scenario index out of range and a negative Manning coefficient are
    refused with GEOFLOOD_ERR_ARG; the context then steps as the oracle."""
    prob = inputs.radial_dambreak(64, 16, dx=8.0, radius=120.0)
    g, r = pair(prob)
    for call in (lambda: g.read(1), lambda: g.set_scenario(1, 0.03, 0.0),
                 lambda: g.set_scenario(0, -0.01, 0.0)):
        with pytest.raises(geoflood.GeoFloodError) as e:
            call()
        assert e.value.code == -1
    g.step(1e9, 4)
    r.step(1e9, 4)
    assert g.time()["steps"] == r.time()["steps"]
    assert_same_state(g, r)


def test_single_patch_forest_and_a_target_already_reached():
    """Degenerate sizes: a forest of one 32 x 32 patch (all four sides
    physical boundaries) steps as the oracle; a call whose target time is
    already reached takes no step and leaves the state as it was."""
    prob = inputs.radial_dambreak(32, 32, dx=4.0, radius=40.0)
    g, r = pair(prob)
    assert g.npatch == 1
    g.step(1e9, 10)
    r.step(1e9, 10)
    assert g.time()["steps"] == r.time()["steps"] == 10
    assert_same_state(g, r)
    t = g.time()["t"]
    before = g.read()
    _, n = g.step(t, 5)
    assert n == 0 and g.time()["t"] == t and g.time()["steps"] == 10
    for a, b in zip(g.read(), before):
        assert np.array_equal(a, b)
