"""Learned refinement predictor on the GPU against the FP64 oracle of
oracle/cnn.py: input features, forward and backward passes, the Adam step,
training on the plain criterion's own flags, and what the trained network
gains over plain tagging when regridding less often."""
import time

import numpy as np
import pytest

from oracle import cnn as ocnn
from paper_2403_15435_gb300 import geoflood, inputs

pytestmark = pytest.mark.gpu

SCALE = (4.0, 8.0, 8.0, 4.0)


def small_valley(patch=16, seed=inputs.SEED_BASE + 2, depth=8.0, breach_x=300.0,
                 precision=0, maxlevel=2, mi=4, mj=2, Lx=1000.0, Ly=500.0):
    prob = inputs.v_valley(mi=mi, mj=mj, patch=patch, minlevel=0, maxlevel=maxlevel,
                           dem_spacing=8.0, Lx=Lx, Ly=Ly, breach_x=breach_x,
                           depth=depth, n_gauges=8, seed=seed)
    prob.cfg.src_level = 1
    prob.cfg.precision = precision
    return prob


def valley(seed, depth, breach_x, precision=0):
    """2 km x 1 km valley, 16 x 16 patches on levels 0..3 (finest dx 1.95 m)."""
    return small_valley(16, seed=seed, depth=depth, breach_x=breach_x, precision=precision,
                        maxlevel=3, mi=8, mj=4, Lx=2000.0, Ly=1000.0)


def forest(prob, **kw):
    g = geoflood.Forest(prob.cfg, prob.dem, **kw)
    g.set_state(prob.ic)
    g.cnn_set_scale(SCALE)
    return g


def params(seed):
    rng = np.random.default_rng(seed)
    prm = ocnn.init_params(rng)
    for l in range(3):
        off = l * (16 * 144 + 16) + 16 * 144
        prm[off:off + 16] = rng.normal(0, 0.05, 16)
    prm[-1] = -0.5
    return prm.astype(np.float32)


def ulp_bf16(x):
    e = np.floor(np.log2(np.maximum(np.abs(x), 1e-30)))
    return 2.0 ** (e - 7)


@pytest.mark.parametrize("patch,precision", [(16, 0), (32, 0), (16, 1), (32, 1)])
def test_features_match_oracle(patch, precision):
    """FP64 forests: FP64 sums, as the oracle.  FP32 forests: FP32 sums of
    the stored values; the oracle takes the same state read out in FP64."""
    prob = small_valley(patch, precision=precision)
    g = forest(prob)
    for _ in range(3):
        g.regrid()
        g.step(1e9, 6)
    L, X, Y = g.patch_info()
    assert len(set(L)) > 1  # several levels present
    gpu = geoflood.bf16_to_float(g.cnn_features()).astype(np.float64).reshape(-1, 18, 18, 16)
    c = prob.cfg
    ref = ocnn.bf16_round(ocnn.features(L, X, Y, *g.read(), c.mi, c.mj, c.mx, SCALE))
    d = np.abs(gpu - ref)
    # every feature within one BF16 unit in the last place of the larger of
    # the two (both round the same FP64 means; only summation order differs)
    assert np.all(d <= ulp_bf16(np.maximum(np.abs(ref), np.abs(gpu)))), d.max()
    exact = np.mean(d == 0)
    print("features: %d patches, %.4f%% bit-exact" % (len(L), 100 * exact))
    assert exact >= 0.999


def test_forward_backward_match_oracle():
    prob = small_valley(16)
    g = forest(prob)
    g.regrid()
    g.step(1e9, 20)
    x = g.cnn_features()[:64]
    n = len(x)
    rng = np.random.default_rng(11)
    y = (rng.random(n) < 0.4).astype(np.float32)
    prm = params(5)
    g.cnn_set_params(prm)
    z, grad, loss = g.cnn_grad(x, y, pos_weight=2.5)
    xf = ocnn.bf16_bits_to_float(x)
    l_ref, g_ref, f = ocnn.loss_and_grad(xf, y, prm.astype(np.float64), 2.5, rounding=True)
    l_ex, g_ex, f_ex = ocnn.loss_and_grad(xf, y, prm.astype(np.float64), 2.5, rounding=False)
    dz = np.abs(z - f["z"]).max()
    print("logits: max |dz| %.2e vs the BF16-point oracle, %.2e vs exact FP64"
          % (dz, np.abs(z - f_ex["z"]).max()))
    # measured 3.7e-7: FP32 summation order only
    assert dz <= 1e-5 * max(1.0, np.abs(f["z"]).max())
    assert abs(loss - l_ref) <= 1e-4 * max(1.0, l_ref)
    # per parameter block: relative L2 error of the gradient
    blocks = {"W1": (0, 2304), "b1": (2304, 2320), "W2": (2320, 4624), "b2": (4624, 4640),
              "W3": (4640, 6944), "b3": (6944, 6960), "wh": (6960, 6976), "bh": (6976, 6977)}
    for name, (a, b) in blocks.items():
        ref = g_ref[a:b]
        err = np.linalg.norm(grad[a:b] - ref) / max(np.linalg.norm(ref), 1e-30)
        err_ex = np.linalg.norm(grad[a:b] - g_ex[a:b]) / max(np.linalg.norm(g_ex[a:b]), 1e-30)
        print("grad %s: rel L2 %.2e (BF16-point oracle), %.2e (exact FP64)" % (name, err, err_ex))
        assert err <= 1e-4, name  # measured at most 1.4e-6


def collect_dataset(prob, t_end, capacity=20000, regrid=16, check=4):
    g = forest(prob)
    g.cnn_dataset(capacity)
    st = g.advance(t_end, regrid_interval=regrid, check_interval=check, collect=True)
    x, y = g.cnn_dataset_read(0, st["samples"])
    return g, x, y, st


def test_adam_step_matches_oracle():
    prob = small_valley(16)
    g, x, y, st = collect_dataset(prob, 30.0, capacity=512)
    assert st["samples"] > 0
    n = len(y)
    prm = params(9)
    g.cnn_set_params(prm)
    lr = 1e-3
    g.cnn_train(1, n, lr=lr, pos_weight=2.0, seed=1)
    p1 = g.cnn_get_params().astype(np.float64)
    _, g_ref, _ = ocnn.loss_and_grad(ocnn.bf16_bits_to_float(x), y, prm.astype(np.float64),
                                     2.0, rounding=True)
    ref, _, _ = ocnn.adam_step(prm.astype(np.float64), g_ref, 0 * g_ref, 0 * g_ref, 1, lr)
    big = np.abs(g_ref) > 1e-3 * np.abs(g_ref).max()  # sign of the step well defined
    d = np.abs((p1 - prm) - (ref - prm))[big]
    print("Adam step: %d of %d parameters compared, max |d| %.2e (lr %.0e)"
          % (big.sum(), len(big), d.max(), lr))
    assert np.mean(d <= 1e-2 * lr) >= 0.999


@pytest.fixture(scope="module")
def trained():
    """Network trained on the plain criterion's flags of one valley."""
    prob = valley(inputs.SEED_BASE + 40, depth=10.0, breach_x=300.0)
    g, x, y, st = collect_dataset(prob, 60.0, capacity=60000)
    npos = int(y.sum())
    print("dataset: %d samples, %d positive" % (len(y), npos))
    g.cnn_set_params(params(3))
    pw = float(np.clip((len(y) - npos) / max(npos, 1), 1.0, 20.0))
    loss = g.cnn_train(40, 64, lr=2e-3, pos_weight=pw, seed=7)
    return g.cnn_get_params(), loss, pw


def test_training_reduces_loss(trained):
    prm, loss, pw = trained
    print("epoch loss: first %.4f, last %.4f" % (loss[0], loss[-1]))
    assert loss[-1] < 0.6 * loss[0]


def run_mode(prob, prm, regrid, tagger, on_miss, t_end, thr=0.5):
    g = forest(prob)
    if prm is not None:
        g.cnn_set_params(prm)
        g.set_tagger(tagger, thr)
    g.set_gauges(prob.gauges)
    t0 = time.perf_counter()
    st = g.advance(t_end, regrid_interval=regrid, check_interval=4, regrid_on_miss=on_miss)
    st["wall"] = time.perf_counter() - t0
    out, arr = g.gauges()
    st["gauge_h"] = out[:, 1].copy()
    st["arrival"] = arr.copy()
    return st


def test_learned_tags_let_regridding_run_less_often(trained):
    prm = trained[0]
    prob = valley(inputs.SEED_BASE + 41, depth=12.0, breach_x=350.0)
    t_end = 90.0
    plain4 = run_mode(prob, None, 4, geoflood.TAGGER_PLAIN, False, t_end)
    plain16 = run_mode(prob, None, 16, geoflood.TAGGER_PLAIN, True, t_end)
    learned16 = run_mode(prob, prm, 16, geoflood.TAGGER_LEARNED, True, t_end)
    for name, st in (("plain/4", plain4), ("plain/16+miss", plain16), ("learned/16+miss", learned16)):
        print("%-16s steps %4d regrids %3d (on miss %3d) misses %4d patch-steps %7d "
              "max gauge |dh| vs plain/4 %.3f m"
              % (name, st["steps"], st["regrids"], st["miss_regrids"], st["misses"],
                 st["patch_steps"], np.abs(st["gauge_h"] - plain4["gauge_h"]).max()))
    for thr in (0.3, 0.7):
        st = run_mode(prob, prm, 16, geoflood.TAGGER_LEARNED, True, t_end, thr)
        print("learned thr %.1f   steps %4d regrids %3d (on miss %3d) misses %4d patch-steps %7d "
              "wall %.2f s" % (thr, st["steps"], st["regrids"], st["miss_regrids"], st["misses"],
                               st["patch_steps"], st["wall"]))
    for name, st in (("plain/4", plain4), ("plain/16+miss", plain16), ("learned/16+miss", learned16)):
        print("%-16s wall %.2f s, arrival times %s" % (name, st["wall"], np.round(st["arrival"], 2)))
    assert learned16["regrids"] < plain4["regrids"]
    assert learned16["regrids"] < plain16["regrids"]
    assert learned16["misses"] <= plain16["misses"]
