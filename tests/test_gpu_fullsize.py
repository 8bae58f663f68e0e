"""The larger workloads at their full sizes, checked on sampled outputs the
oracle computes one by one: after some steps and regrids, one more step is
taken and, for a sample of patches, the oracle steps each tile as the GPU
held it (ghost cells included) with the same dt; FP64 within 1e-12
relative, FP32 within 1e-4 m and 1e-4 m^2/s.  Workloads: the 4 km x 2 km
V-valley on three levels (about 2-6k patches of 32 x 32), the 17 km x 9 km
canyon-to-plain on five levels with 16 x 16 or 32 x 32 patches and the
learned tagger, and 64 full-size valleys in one context."""
import numpy as np
import pytest

import oracle
from paper_2403_15435_gb300 import geoflood, inputs

pytestmark = pytest.mark.gpu


def sampled_step(g, cfg, s, rng, n_wet=16, n_any=8, prec=0, manning=None):
    """Take one more step of scenario s and check sampled patches."""
    info = g.time(s)
    tiles = g.read_tiles(s)
    L, X, Y = g.patch_info(s)
    g.step(info["t"] + 1e9, 1)
    assert g.time(s)["rejects"] == info["rejects"], "the checked step was retaken"
    after = g.read(s)
    wet = [k for k in range(len(L)) if tiles[k][0].max() > 10 * cfg.drytol]
    assert len(wet) >= n_wet
    sample = list(rng.choice(wet, n_wet, replace=False)) + \
        list(rng.choice(len(L), n_any, replace=False))
    for k in sample:
        nx = cfg.mi * cfg.mx << int(L[k])
        ny = cfg.mj * cfg.mx << int(L[k])
        dx = (cfg.xupper - cfg.xlower) / nx
        dy = (cfg.yupper - cfg.ylower) / ny
        t = tiles[k]
        ref = oracle.step_grid(t[0], t[1], t[2], t[3], dx, dy, info["dt_next"],
                               drytol=cfg.drytol,
                               manning_n=cfg.manning_n if manning is None else manning)[:3]
        for f in range(3):
            got, want = after[f][k], ref[f][2:-2, 2:-2]
            if prec == 0:
                e = float(np.abs(got - want).max()) / max(1.0, float(np.abs(want).max()))
                assert e <= 1e-12, "patch %d field %d: %.3e" % (k, f, e)
            else:
                e = float(np.abs(got - want).max())
                assert e <= 1e-4, "patch %d field %d: %.3e" % (k, f, e)
    return len(L)


@pytest.mark.parametrize("prec", [0, 1])
def test_valley_4km_three_levels(prec):
    prob = inputs.v_valley()
    prob.cfg.precision = prec
    g = geoflood.Forest(prob.cfg, prob.dem)
    g.set_state(prob.ic)
    g.set_gauges(prob.gauges)
    for _ in range(3):
        g.regrid()
        g.step(1e9, 4)
    assert set(g.patch_info()[0]) == {2, 3, 4}
    n = sampled_step(g, prob.cfg, 0, np.random.default_rng(3), prec=prec)
    assert 2000 <= n <= 8000


@pytest.mark.parametrize("patch,maxlevel", [(32, 4), (16, 5)])
def test_canyon_plain_five_levels_learned_tagger(patch, maxlevel):
    prob = inputs.canyon_plain(patch=patch, minlevel=maxlevel - 4, maxlevel=maxlevel)
    g = geoflood.Forest(prob.cfg, prob.dem, max_patches=40000)
    g.set_state(prob.ic)
    g.cnn_set_scale((10.0, 20.0, 20.0, 10.0))
    g.cnn_set_params(inputs.cnn_init(3).astype(np.float32))
    g.set_tagger(geoflood.TAGGER_LEARNED, 0.5)
    g.advance(20.0, regrid_interval=8, check_interval=4, regrid_on_miss=True)
    L = g.patch_info()[0]
    assert len(set(L)) >= 4
    n = sampled_step(g, prob.cfg, 0, np.random.default_rng(5), prec=1)
    assert 1000 <= n <= 40000


def test_ensemble_of_64_full_valleys():
    probs = inputs.valley_ensemble_full(64)
    cfg = probs[0].cfg
    g = geoflood.Forest(cfg, None, num_scenarios=64, max_patches=64 * 8192, max_gauges=16)
    for k, p in enumerate(probs):
        g.set_scenario(k, p.cfg.manning_n, p.cfg.eta0)
        g.set_topo(p.dem, k)
        g.set_state(p.ic, k)
    g.advance(6.0, regrid_interval=4, check_interval=4)
    counts = [g.npatch_of(k) for k in range(64)]
    assert min(counts) >= 2048 and sum(counts) <= 64 * 8192
    rng = np.random.default_rng(11)
    for s in (0, 31, 63):
        sampled_step(g, probs[s].cfg, s, rng, n_wet=8, n_any=4, prec=1)
