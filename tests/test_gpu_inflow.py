"""Inflow-hydrograph boundary (Sec. 5.1) on the GPU against the FP64 oracle:
trajectories of a dry basin fed through a segment of one side (each side in
turn, both patch sizes), every tile cell (ghost cells and corners included),
a bore entering a channel, a refined forest through regrids, and the FP32
form within 1e-4 per step."""
import numpy as np
import pytest

import oracle
from paper_2403_15435_gb300 import geoflood, inputs
from test_gpu_parity import assert_same_state, pair, rel
from test_oracle_inflow import flood

pytestmark = pytest.mark.gpu


def rotate(prob, side):
    """The basin with its inflow on another side (a square domain)."""
    cfg = inputs.Config(**{**prob.cfg.__dict__, "inflow_side": side})
    return inputs.Problem(prob.name, cfg, prob.dem, prob.ic, prob.t_end)


@pytest.mark.parametrize("side", [0, 1, 2, 3])
@pytest.mark.parametrize("patch", [16, 32])
def test_inflow_trajectory_matches_oracle(patch, side):
    prob = rotate(flood(64, patch), side)
    g, r = pair(prob)
    tg, ng = g.step(150.0)
    tr, nr = r.step(150.0)
    assert ng == nr and tg == tr
    assert_same_state(g, r, tol=1e-11)
    assert rel(g.read_tiles(), r.read_tiles()) <= 1e-11
    m_g, m_r = g.mass(), r.mass()
    assert abs(m_g - m_r) <= 1e-11 * m_r


def test_inflow_ghosts_after_set_state_and_across_hydrograph_end():
    """Tiles right after the initial fill (wet interior next to the inlet),
    then through the end of the inflow (Q falls to 0: the wall again)."""
    prob = flood(64, 16, hydrograph=((0.0, 6.0), (40.0, 6.0), (50.0, 0.0)))

    def ic(x, y, b):
        h = 0.2 + 0.1 * np.exp(-((y - 320.0) / 60.0) ** 2)
        return h, 0.05 * h, np.zeros_like(h)

    prob.ic = ic
    g, r = pair(prob)
    assert rel(g.read_tiles(), r.read_tiles()) <= 1e-14
    for t in (20.0, 45.0, 70.0):
        g.step(t)
        r.step(t)
        assert rel(g.read_tiles(), r.read_tiles()) <= 1e-11, t


def test_bore_channel_matches_oracle():
    prob = inputs.inflow_channel(128, 32, q=2.0, h0=1.0, t_end=30.0)
    g, r = pair(prob)
    g.step(30.0)
    r.step(30.0)
    assert_same_state(g, r, tol=1e-11)


def test_flood_speed_forest_matches_oracle_through_regrids():
    """Test Case 1 stand-in, coarsened (16-cell patches, levels 0..2) and
    shortened: regrid every 8 steps for 6 cycles, patch lists and states
    compared after each."""
    prob = inputs.flood_speed(patch=16, minlevel=0, maxlevel=2)
    g, r = pair(prob)
    for cycle in range(6):
        g.regrid()
        r.regrid()
        assert [list(a) for a in g.patch_info()] == [list(a) for a in r.patch_info()]
        g.step(1e9, 8)
        r.step(1e9, 8)
        assert_same_state(g, r, tol=1e-11)
    assert g.read()[0].max() > 0.0


def test_fp32_inflow_one_step_from_oracle_state():
    prob = flood(64, 32)
    r = oracle.OracleForest(prob.cfg, prob.dem)
    r.set_state(prob.ic)
    r.step(100.0)
    h, hu, hv, _ = r.read()
    cfg32 = inputs.Config(**{**prob.cfg.__dict__, "precision": 1})
    g = geoflood.Forest(cfg32, prob.dem)
    info = r.time()
    g.set_time(info["t"], info["dt_next"])
    g.write(h, hu, hv)
    r.step(info["t"] + 10.0, 1)
    g.step(info["t"] + 10.0, 1)
    a, b = g.read(), r.read()
    for k in range(3):
        assert np.abs(a[k] - b[k]).max() <= 1e-4, k


def test_bad_inflow_is_rejected():
    for kw in (dict(inflow_side=4), dict(inflow_hi=0.0), dict(inflow_tau=0.0),
               dict(hydrograph=((0.0, 1.0), (0.0, 2.0))),
               dict(hydrograph=((0.0, -1.0),))):
        with pytest.raises(Exception):
            p = flood(64, 32, **kw)
            geoflood.Forest(p.cfg, p.dem)
