"""Parity at the configurations the benchmark times, on sampled outputs the
oracle computes one by one.  The GPU runs the workload in the bench's launch
configuration; at several times one more step is taken and, for at least
64 patches -- half of them on the wet front (tiles holding both wet and dry
cells), the rest drawn from all patches -- the oracle steps each tile as the
GPU held it (ghost cells included) with the same dt.  (Early in the
uniform run the front crosses fewer than 32 patches; then all of them are
taken and the rest drawn from all patches.)  FP64 within 1e-12
relative, FP32 within 1e-4 m and 1e-4 m^2/s (the deviation form's bound).

Workloads: the 1024 x 1024 radial dam break (the uniform secondary
workload) at t = 5, 30 and 60 s in both precisions, and the 4 km x 2 km
valley on levels 2-4 (the headline workload) in FP32 with the learned
tagger and regrid every 64 steps, and in FP64 with plain tags and regrid
every 4, at t = 5 and 20 s."""
import numpy as np
import pytest

import oracle
from paper_2403_15435_gb300 import geoflood, inputs

pytestmark = pytest.mark.gpu


def check_step(g, cfg, prec, rng, n_total=64):
    """One more step of the forest; 64 sampled patches against the oracle:
    up to half of them on the wet front (at least 16 must exist), the rest
    drawn from all patches.  Returns the number of front patches found."""
    info = g.time()
    tiles = g.read_tiles()
    L, X, Y = g.patch_info()
    g.step(info["t"] + 1e9, 1)
    assert g.time()["rejects"] == info["rejects"], "the checked step was retaken"
    after = g.read()
    h = tiles[:, 0, 2:-2, 2:-2]
    wet = h > cfg.drytol
    front = np.flatnonzero(wet.any(axis=(1, 2)) & ~wet.all(axis=(1, 2)))
    assert len(front) >= 16, "only %d patches on the wet front" % len(front)
    n_front = min(n_total // 2, len(front))
    sample = list(rng.choice(front, n_front, replace=False)) + \
        list(rng.choice(len(L), n_total - n_front, replace=False))
    worst = 0.0
    for k in sample:
        nx = cfg.mi * cfg.mx << int(L[k])
        ny = cfg.mj * cfg.mx << int(L[k])
        dx = (cfg.xupper - cfg.xlower) / nx
        dy = (cfg.yupper - cfg.ylower) / ny
        t = tiles[k]
        ref = oracle.step_grid(t[0], t[1], t[2], t[3], dx, dy, info["dt_next"],
                               drytol=cfg.drytol, manning_n=cfg.manning_n)[:3]
        for f in range(3):
            got, want = after[f][k], ref[f][2:-2, 2:-2]
            if prec == 0:
                e = float(np.abs(got - want).max()) / max(1.0, float(np.abs(want).max()))
                assert e <= 1e-12, "patch %d field %d: %.3e" % (k, f, e)
            else:
                e = float(np.abs(got - want).max())
                assert e <= 1e-4, "patch %d field %d: %.3e" % (k, f, e)
            worst = max(worst, e)
    print("t = %.2f s: %d front patches, %d checked, worst %.2e"
          % (info["t"], len(front), len(sample), worst))
    return len(front)


@pytest.mark.parametrize("prec", [1, 0])
def test_uniform_1024_at_three_times(prec):
    """The 1024 x 1024 radial dam break, in the bench's kernel variant
    (chosen by the autotuner half way through the run)."""
    prob = inputs.radial_dambreak(1024, 32, dx=2.0)
    prob.cfg.precision = prec
    g = geoflood.Forest(prob.cfg, prob.dem)
    g.set_state(prob.ic)
    g.step(30.0)
    variant, _ = g.autotune(2)
    g.close()
    g = geoflood.Forest(prob.cfg, prob.dem)
    g.set_state(prob.ic)
    g.set_variant(variant)
    rng = np.random.default_rng(21 + prec)
    for t in (5.0, 30.0, 60.0):
        g.step(t)
        check_step(g, prob.cfg, prec, rng)
    g.close()


def _valley_net(stream=None):
    """A network for the valley's learned tags: trained briefly on the plain
    criterion's flags from another seed of the valley (as the bench does)."""
    tr = inputs.v_valley(seed=inputs.SEED_BASE + 50)
    tr.cfg.precision = 1
    f = geoflood.Forest(tr.cfg, tr.dem, max_patches=16 * 8 * 4 ** 4)
    f.set_state(tr.ic)
    f.cnn_set_scale((4.0, 8.0, 8.0, 4.0))
    f.cnn_dataset(60000)
    st = f.advance(8.0, regrid_interval=64, check_interval=4, collect=True)
    _, y = f.cnn_dataset_read(0, st["samples"])
    pw = float(np.clip((len(y) - y.sum()) / max(y.sum(), 1), 1.0, 20.0))
    f.cnn_set_params(inputs.cnn_init(3))
    f.cnn_train(3, 64, lr=2e-3, pos_weight=pw, seed=7)
    prm = f.cnn_get_params()
    f.close()
    return prm, pw / (1.0 + pw)


@pytest.mark.parametrize("prec,learned,regrid", [(1, True, 64), (0, False, 4)])
def test_headline_valley_in_bench_configuration(prec, learned, regrid):
    prob = inputs.v_valley()
    prob.cfg.precision = prec
    g = geoflood.Forest(prob.cfg, prob.dem, max_patches=16 * 8 * 4 ** 4, max_gauges=32)
    g.set_state(prob.ic)
    g.cnn_set_scale((4.0, 8.0, 8.0, 4.0))
    if learned:
        prm, thr = _valley_net()
        g.cnn_set_params(prm)
        g.set_tagger(geoflood.TAGGER_LEARNED, thr)
    g.set_gauges(prob.gauges)
    rng = np.random.default_rng(31 + prec)
    for t in (5.0, 20.0):
        g.advance(t, regrid_interval=regrid, check_interval=4, regrid_on_miss=learned)
        check_step(g, prob.cfg, prec, rng)
    L = g.patch_info()[0]
    levels = set(int(x) for x in L)
    assert levels <= {2, 3, 4} and len(levels) >= 2
    g.close()


@pytest.mark.parametrize("prec", [1, 0])
def test_valley_variants_agree_bitwise(prec):
    """The headline valley through its regrids (plain tags, regrid every 4,
    to t = 20 s) with the whole-tile kernel, which lets isolated dry tiles
    skip the step, and with the 16 x 16 sub-tile kernel, which runs every
    tile: states, forests, gauges and step counts agree bit for bit."""
    out = []
    for variant in (0, 1):
        prob = inputs.v_valley()
        prob.cfg.precision = prec
        g = geoflood.Forest(prob.cfg, prob.dem, max_patches=16 * 8 * 4 ** 4)
        g.set_state(prob.ic)
        g.set_gauges(prob.gauges)
        g.set_variant(variant)
        st = g.advance(20.0 if prec else 6.0, regrid_interval=4, check_interval=4)
        out.append([np.array([st["steps"], st["regrids"]])] + list(g.patch_info()) +
                   list(g.read()) + list(g.gauges()))
        g.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
