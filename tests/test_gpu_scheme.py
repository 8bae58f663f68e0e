"""Scheme variants of Sec. 3.2 on the GPU against the FP64 oracle: the
first-order method, the unsplit method without transverse terms and
dimensional splitting, alone and combined, on both patch sizes.

FP64: within 1e-12 relative per step from identical inputs, wet masks
bit-exact.  Whole trajectories are compared without bottom friction: both
sides then take the same operations in the same order and agree to the last
bit, whereas with friction the one libm difference (cbrt) is amplified by
the no-transverse and split variants (a 1e-15 perturbation of the oracle's
own initial state grows to 1e-7 in 12 s of the radial dam break; the
unsplit method with transverse terms keeps it at 1e-15).  FP32: within
1e-4 m and 1e-4 m^2/s per step from identical inputs."""
import numpy as np
import pytest

import oracle
from paper_2403_15435_gb300 import geoflood, inputs
from test_gpu_parity import assert_same_state, pair, rel

pytestmark = pytest.mark.gpu

# without transverse terms the unsplit method is stable up to a Courant
# number of 1/2 only
NO_TR = dict(no_transverse=1, cfl_desired=0.45, cfl_max=0.5)
FLAGS = [dict(first_order=1), NO_TR, dict(dim_split=1),
         dict(dim_split=1, first_order=1), dict(first_order=1, **NO_TR)]
IDS = ["first_order", "no_transverse", "dim_split", "dim_split+first_order",
       "first_order+no_transverse"]
ABS = 1e-4


def with_flags(prob, flags, **extra):
    cfg = inputs.Config(**{**prob.cfg.__dict__, **flags, **extra})
    return inputs.Problem(prob.name, cfg, prob.dem, prob.ic, prob.t_end, prob.gauges)


@pytest.mark.parametrize("patch", [16, 32])
@pytest.mark.parametrize("flags", FLAGS, ids=IDS)
def test_variant_one_step_from_oracle_state(flags, patch):
    """One step with friction from the oracle's state at 8 s."""
    prob = with_flags(inputs.radial_dambreak(128, patch, dx=4.0, radius=100.0), flags)
    g, r = pair(prob)
    r.step(8.0)
    h, hu, hv, _ = r.read()
    g.write(h, hu, hv)
    info = r.time()
    g.set_time(info["t"], info["dt_next"])
    r.step(info["t"] + 10.0, 1)
    g.step(info["t"] + 10.0, 1)
    assert_same_state(g, r)
    assert g.time()["dt_next"] == pytest.approx(r.time()["dt_next"], rel=1e-12)


@pytest.mark.parametrize("patch", [16, 32])
@pytest.mark.parametrize("flags", FLAGS, ids=IDS)
def test_variant_trajectory_matches_oracle(flags, patch):
    """Radial dam break over terrain with wet/dry fronts, 12 s, no friction."""
    prob = with_flags(inputs.radial_dambreak(128, patch, dx=4.0, radius=100.0), flags,
                      manning_n=0.0)
    g, r = pair(prob)
    tg, ng = g.step(12.0)
    tr, nr = r.step(12.0)
    assert ng == nr and tg == tr
    assert_same_state(g, r)
    gi, ri = g.time(), r.time()
    assert gi["rejects"] == ri["rejects"] and gi["nclip"] == ri["nclip"]


@pytest.mark.parametrize("flags", [dict(dim_split=1), dict(first_order=1)],
                         ids=["dim_split", "first_order"])
def test_variant_on_refined_forest_matches_oracle(flags):
    """Valley breach on three levels: ghost cells across level changes feed
    the sweeps (the split x sweep runs on the ghost rows too)."""
    base = inputs.v_valley(mi=4, mj=2, patch=16, minlevel=0, maxlevel=2,
                           dem_spacing=8.0, Lx=1000.0, Ly=500.0, breach_x=300.0,
                           depth=8.0, n_gauges=6)
    prob = with_flags(base, flags, src_level=1, manning_n=0.0)
    g, r = pair(prob)
    for cycle in range(3):
        g.regrid()
        r.regrid()
        assert [list(a) for a in g.patch_info()] == [list(a) for a in r.patch_info()]
        g.step(1e9, 6)
        r.step(1e9, 6)
        assert_same_state(g, r)


@pytest.mark.parametrize("flags", FLAGS, ids=IDS)
def test_fp32_variant_one_step_from_oracle_state(flags):
    prob = with_flags(inputs.radial_dambreak(128, 32, dx=4.0, radius=100.0), flags)
    r = oracle.OracleForest(prob.cfg, prob.dem)
    r.set_state(prob.ic)
    r.step(8.0)
    h, hu, hv, _ = r.read()
    p32 = with_flags(prob, {}, precision=1)
    g = geoflood.Forest(p32.cfg, p32.dem)
    g.write(h, hu, hv)
    info = r.time()
    g.set_time(info["t"], info["dt_next"])
    r.step(info["t"] + 10.0, 1)
    g.step(info["t"] + 10.0, 1)
    a, b = g.read(), r.read()
    for k in range(3):
        assert np.abs(a[k] - b[k]).max() <= ABS, k
    mism = int(np.count_nonzero((a[0] > prob.cfg.drytol) != (b[0] > prob.cfg.drytol)))
    assert mism <= 2, "wet masks differ in %d cells" % mism


@pytest.mark.parametrize("prec", [0, 1])
def test_dim_split_lake_at_rest_and_volume(prec):
    """A lake at rest over an emerged bump stays at rest under dimensional
    splitting, and a dam break keeps its volume up to the clipped depth."""
    lake = with_flags(inputs.lake_at_rest(128, patch=32, eta=0.3), dict(dim_split=1),
                      precision=prec, eta0=0.3)
    g = geoflood.Forest(lake.cfg, lake.dem)
    g.set_state(lake.ic)
    h0 = g.read()[0]
    g.step(1e9, 200)
    h, hu, hv, _ = g.read()
    if prec == 0:
        assert np.abs(h - h0).max() <= 1e-13
        assert np.abs(hu).max() <= 1e-13 and np.abs(hv).max() <= 1e-13
    else:  # deviation form: w = 0 is stored exactly
        assert np.abs(h - h0).max() <= 1e-6
        assert np.all(hu == 0.0) and np.all(hv == 0.0)
    dam = with_flags(inputs.radial_dambreak(128, 32, dx=4.0, radius=100.0),
                     dict(dim_split=1), precision=prec)
    g = geoflood.Forest(dam.cfg, dam.dem)
    g.set_state(dam.ic)
    m0 = g.mass()
    g.step(10.0)
    info = g.time()
    assert abs(g.mass() - m0 - info["clipvol"]) <= (1e-13 if prec == 0 else 1e-6) * m0


def test_bad_scheme_flags_are_rejected():
    prob = with_flags(inputs.stoker(64, patch=32), dict(dim_split=2))
    with pytest.raises(Exception):
        geoflood.Forest(prob.cfg, prob.dem)
