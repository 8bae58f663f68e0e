"""Pins of the learned-tagger oracle (oracle/cnn.py) against facts that do not
come from the oracle itself: library routines (torch's BF16 conversion,
scipy's 2-D cross-correlation), finite differences of the loss, closed forms
(zero network, constant and linear fields, the first Adam step)."""
import numpy as np
import pytest

from oracle import cnn

rng0 = np.random.default_rng(20240322)


def test_bf16_round_matches_torch_and_ties_to_even():
    torch = pytest.importorskip("torch")
    x = np.concatenate([rng0.normal(0, 1, 4000), rng0.normal(0, 1e3, 1000),
                        rng0.normal(0, 1e-3, 1000)]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cnn.bf16_round(x), ref)
    # halfway cases: 1 + 2^-8 lies between 1 and 1 + 2^-7 (ties to the even 1),
    # 1 + 3 * 2^-8 between 1 + 2^-7 and 1 + 2^-6 (ties to the even 1 + 2^-6)
    assert cnn.bf16_round(1 + 2.0 ** -8) == 1.0
    assert cnn.bf16_round(1 + 3 * 2.0 ** -8) == 1 + 2.0 ** -6
    assert cnn.bf16_round(-(1 + 3 * 2.0 ** -8)) == -(1 + 2.0 ** -6)
    bits = cnn.float_to_bf16_bits(np.array([1.0, -2.0, 0.15625]))
    assert list(bits) == [0x3F80, 0xC000, 0x3E20]


def test_conv_matches_scipy_correlate2d():
    signal = pytest.importorskip("scipy.signal")
    x = rng0.normal(size=(1, 18, 18, 16))
    W = rng0.normal(size=(16, 144))
    out = cnn.conv3x3(x, W)
    for co in (0, 5, 15):
        ref = np.zeros((16, 16))
        for ci in range(16):
            k = np.zeros((3, 3))
            for tap in range(9):
                k[tap // 3, tap % 3] = W[co, tap * 16 + ci]  # row = dy + 1
            ref += signal.correlate2d(x[0, :, :, ci], k, mode="valid")
        assert np.allclose(out[0, :, :, co], ref, rtol=1e-12, atol=1e-12)


def test_adjoint_and_weight_gradient_are_the_transposes():
    # <conv(x; W), d> = <x, conv_adjoint(d; W)> = <W, wgrad(d, x)>
    x = rng0.normal(size=(2, 18, 18, 16))
    W = rng0.normal(size=(16, 144))
    d = rng0.normal(size=(2, 16, 16, 16))
    lhs = np.sum(cnn.conv3x3(x, W) * d)
    assert np.isclose(lhs, np.sum(x * cnn.conv3x3_adjoint(d, W)), rtol=1e-12)
    assert np.isclose(lhs, np.sum(W * cnn.conv3x3_wgrad(d, x)), rtol=1e-12)


def _sample(n, rng):
    x = np.zeros((n, 18, 18, 16))
    x[..., :5] = rng.normal(size=(n, 18, 18, 5))
    y = (rng.random(n) < 0.5).astype(np.float64)
    return x, y


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(7)
    prm = cnn.init_params(rng)
    prm[cnn.NPARAM - 17:cnn.NPARAM - 1] = rng.normal(0, 1.0, 16)
    for l in range(3):  # non-zero biases so that relu boundaries move
        off = l * (16 * 144 + 16) + 16 * 144
        prm[off:off + 16] = rng.normal(0, 0.1, 16)
    x, y = _sample(3, rng)
    loss, g, _ = cnn.loss_and_grad(x, y, prm, pos_weight=3.0, rounding=False)
    idx = np.concatenate([rng.choice(cnn.NPARAM - 17, 60, replace=False),
                          np.arange(cnn.NPARAM - 17, cnn.NPARAM)])
    for layer_off in (0, 16 * 144 + 16, 2 * (16 * 144 + 16)):
        idx = np.concatenate([idx, layer_off + 16 * 144 + np.arange(3)])  # biases
    eps = 1e-6
    for k in idx:
        p1, p2 = prm.copy(), prm.copy()
        p1[k] += eps
        p2[k] -= eps
        l1 = cnn.loss_and_grad(x, y, p1, 3.0, rounding=False)[0]
        l2 = cnn.loss_and_grad(x, y, p2, 3.0, rounding=False)[0]
        fd = (l1 - l2) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])) + 1e-9, (k, fd, g[k])


def test_zero_network_closed_form():
    prm = np.zeros(cnn.NPARAM)
    prm[-1] = 0.3  # bh
    x, y = _sample(5, np.random.default_rng(3))
    loss, g, f = cnn.loss_and_grad(x, y, prm, pos_weight=2.0)
    assert np.all(f["z"] == 0.3)
    s = 1 / (1 + np.exp(-0.3))
    w = np.where(y > 0.5, 2.0, 1.0)
    assert np.isclose(g[-1], np.mean(w * (s - y)), rtol=1e-14)
    assert np.isclose(loss, np.mean(w * (np.log1p(np.exp(0.3)) - 0.3 * y)), rtol=1e-14)
    assert np.all(g[:-17] == 0)


def test_features_closed_forms():
    # uniform forest of 2 x 2 patches of 32 x 32 cells at level 1 over 2 x 1
    # blocks; h constant, bed and hu linear in the cell indices
    mx, mi, mj = 32, 2, 1
    L = np.array([1, 1, 1, 1])
    px, py = np.array([0, 1, 0, 1]), np.array([0, 0, 1, 1])
    NX, NY = mi * mx * 2, mj * mx * 2
    J, I = np.mgrid[0:NY, 0:NX].astype(np.float64)
    grids = {"h": np.full((NY, NX), 1.5), "hu": 2.0 * I, "hv": np.zeros((NY, NX)),
             "b": 3.0 + 0.5 * I - 0.25 * J}
    fields = [np.stack([grids[k][y * mx:(y + 1) * mx, x * mx:(x + 1) * mx]
                        for x, y in zip(px, py)]) for k in ("h", "hu", "hv", "b")]
    scale = [0.5, 2.0, 1.0, 0.25]
    f = cnn.features(L, px, py, *fields, mi, mj, mx, scale)
    assert np.all(f[:, 1:17, 1:17, 0] == 3.0)
    assert np.all((f[..., 0] == 3.0) | (f[..., 0] == 0.0))
    # the mean of a linear field over a rectangle of cells is its value at the
    # centre of the rectangle; patch 0 (lower left) has its left and bottom
    # bands outside the domain, its right band 16 cells deep and f = 2
    p = 0
    def centre(lo, hi):
        return 0.5 * (lo + hi - 1)
    bmean = 3.0 + 0.5 * 15.5 - 0.25 * 15.5
    for Y in (1, 5, 16, 17):
        for X in (1, 7, 16, 17):
            i_lo, i_hi = (mx, mx + 16) if X == 17 else (2 * (X - 1), 2 * X)
            j_lo, j_hi = (mx, mx + 16) if Y == 17 else (2 * (Y - 1), 2 * Y)
            ic, jc = centre(i_lo, i_hi), centre(j_lo, j_hi)
            assert np.isclose(f[p, Y, X, 1], 2.0 * ic / 2.0, atol=1e-12)
            assert np.isclose(f[p, Y, X, 3], (3.0 + 0.5 * ic - 0.25 * jc - bmean) / 0.25,
                              atol=1e-12)
    # the left ring of patch 0 lies outside the domain; the bottom-right corner
    # pixel too (below the domain)
    assert np.all(f[p, :, 0, :4] == 0) and np.all(f[p, 0, :, :4] == 0)
    # the left ring of patch 1 averages the 16 rightmost columns of patch 0
    ic = centre(mx - 16, mx)
    assert np.isclose(f[1, 4, 0, 1], ic, atol=1e-12)
    assert np.all(f[..., 4] == 0.25) and np.all(f[..., 5:] == 0)


def test_features_composite_of_a_refined_neighbour():
    # two level-0 patches side by side, the right one refined into 4 level-1
    # leaves: the right ring of patch 0 averages fine cells (mean of children)
    mx, mi, mj = 16, 2, 1
    L = np.array([0, 1, 1, 1, 1])
    px, py = np.array([0, 2, 3, 2, 3]), np.array([0, 0, 0, 1, 1])
    rng = np.random.default_rng(5)
    fields = [rng.random((5, mx, mx)) for _ in range(4)]
    f = cnn.features(L, px, py, *fields, mi, mj, mx, [1, 1, 1, 1])
    # level-0 cell (16 + i, j) is the mean of the 2 x 2 fine cells (2 i .. , 2 j ..)
    # of leaf (2, 0) (j < 8) or (2, 1) (j >= 8); the band is 8 cells deep
    for Y in (1, 8, 9, 16):
        j = Y - 1
        leaf = 1 if j < 8 else 3
        jj = 2 * (j % 8)
        ref = fields[0][leaf, jj:jj + 2, 0:16].mean()
        assert np.isclose(f[0, Y, 17, 0], ref, rtol=1e-12)
    # and the left ring of leaf (2, 0) reads the coarse patch by injection
    # (its band is 8 level-1 cells = 4 level-0 cells deep)
    for Y in (1, 2, 16):
        jc = (Y - 1) // 2
        ref = fields[0][0, jc, 12:16].mean()
        assert np.isclose(f[1, Y, 0, 0], ref, rtol=1e-12)


def test_adam_first_step_is_a_signed_learning_rate():
    g = np.array([1e-2, -3.0, 5e2, -1e-4])
    p0 = np.array([1.0, 2.0, 3.0, 4.0])
    p1, m, v = cnn.adam_step(p0, g, np.zeros(4), np.zeros(4), 1, lr=1e-3)
    # after one step the bias-corrected moments are g and g^2, so the update
    # is -lr g / (|g| + eps)
    assert np.allclose(p1 - p0, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-9, atol=0)
    assert np.allclose(p1 - p0, -1e-3 * np.sign(g), rtol=2e-4)
