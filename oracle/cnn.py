"""FP64 CPU oracle of the learned refinement predictor -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module.  It shares no code with the CUDA library.

The network (an extension beyond the paper, whose refinement criteria are
those of Sec. 4.1): on an 18 x 18 pixel view of a patch (16 x 16 block means
of the interior plus a one-pixel ring of means over the bands of cells, half
a patch deep, beyond its edges),

    a1 = relu(conv3x3_valid(x0; W1) + b1)            16 x 16 x 16
    a2 = relu(conv3x3_same(a1; W2) + b2)             zero padding
    a3 = relu(conv3x3_same(a2; W3) + b3)
    v  = mean over the 256 pixels of a3              16
    z  = wh . v + bh                                 logit
    loss = mean_n w_n * (softplus(z_n) - y_n z_n),   w_n = pos_weight if y_n = 1

with conv(x; W)[y, x, co] = sum_{dy, dx, ci} W[co, tap * 16 + ci] *
x[y + dy, x + dx, ci] over dy, dx in {-1, 0, 1}, tap = (dy + 1) * 3 + (dx + 1)
(cross-correlation, dy the row offset).  Everything is FP64.  With
``rounding=True`` the values that the GPU stores in BF16 (weights, features,
activations and the back-propagated activation gradients) are rounded to
BF16 (round to nearest even) at the same points, so the GPU's results differ
from these only by its FP32 accumulation order.  The backward pass is the
plain adjoint (scatter) of each convolution, not the flipped-kernel
convolution the GPU uses.
"""
from __future__ import annotations

import numpy as np

NCH, KK = 16, 144
NPARAM = 3 * (NCH * KK + NCH) + NCH + 1
TAPS = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def bf16_round(x):
    """Round to the nearest BF16 value (ties to even), via FP32."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_bits_to_float(bits):
    return (np.asarray(bits, np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def float_to_bf16_bits(x):
    f = bf16_round(x).astype(np.float32)
    return (f.view(np.uint32) >> 16).astype(np.uint16)


def unpack(prm):
    """Split the flat parameter vector into (W[3] (16, 144), b[3] (16,), wh, bh)."""
    prm = np.asarray(prm, dtype=np.float64)
    assert prm.shape == (NPARAM,)
    W, b = [], []
    off = 0
    for _ in range(3):
        W.append(prm[off:off + NCH * KK].reshape(NCH, KK))
        off += NCH * KK
        b.append(prm[off:off + NCH])
        off += NCH
    wh = prm[off:off + NCH]
    bh = prm[off + NCH]
    return W, b, wh, bh


def pack(W, b, wh, bh):
    parts = []
    for l in range(3):
        parts += [np.asarray(W[l]).reshape(-1), np.asarray(b[l])]
    parts += [np.asarray(wh), np.atleast_1d(bh)]
    return np.concatenate(parts)


def init_params(rng):
    """He-normal conv weights, zero biases, small head (the caller's choice of
    initialisation; any seeded vector works)."""
    W = [rng.normal(0.0, np.sqrt(2.0 / KK), (NCH, KK)) for _ in range(3)]
    b = [np.zeros(NCH) for _ in range(3)]
    wh = rng.normal(0.0, 0.25, NCH)
    return pack(W, b, wh, 0.0)


def conv3x3(xp, W):
    """Valid 3 x 3 cross-correlation of a padded grid xp [n, H+2, W+2, 16]
    with W [16 co, 144]: returns [n, H, W, 16]."""
    n, H2, W2, _ = xp.shape
    H, Wd = H2 - 2, W2 - 2
    out = np.zeros((n, H, Wd, NCH))
    for tap, (dy, dx) in enumerate(TAPS):
        blk = W[:, tap * NCH:(tap + 1) * NCH]          # [co, ci]
        win = xp[:, 1 + dy:1 + dy + H, 1 + dx:1 + dx + Wd, :]
        out += win @ blk.T
    return out


def conv3x3_adjoint(dy_, W):
    """Adjoint of conv3x3 with respect to its padded input: scatters
    dY [n, H, W, 16] back onto [n, H+2, W+2, 16]."""
    n, H, Wd, _ = dy_.shape
    dxp = np.zeros((n, H + 2, Wd + 2, NCH))
    for tap, (dy, dx) in enumerate(TAPS):
        blk = W[:, tap * NCH:(tap + 1) * NCH]
        dxp[:, 1 + dy:1 + dy + H, 1 + dx:1 + dx + Wd, :] += dy_ @ blk
    return dxp


def conv3x3_wgrad(dy_, xp):
    """Gradient of sum(dY * conv3x3(xp; W)) with respect to W: [16, 144]."""
    n, H, Wd, _ = dy_.shape
    g = np.zeros((NCH, KK))
    for tap, (dy, dx) in enumerate(TAPS):
        win = xp[:, 1 + dy:1 + dy + H, 1 + dx:1 + dx + Wd, :]
        g[:, tap * NCH:(tap + 1) * NCH] = np.einsum("nyxo,nyxi->oi", dy_, win)
    return g


def _pad(a):
    return np.pad(a, ((0, 0), (1, 1), (1, 1), (0, 0)))


def forward(x0, prm, rounding=True):
    """x0: [n, 324, 16] (or [n, 18, 18, 16]) feature values.  Returns a dict
    with the activations a1, a2, a3 [n, 16, 16, 16], the pooled v [n, 16] and
    the logits z [n]."""
    W, b, wh, bh = unpack(prm)
    r = bf16_round if rounding else (lambda t: t)
    x = np.asarray(x0, dtype=np.float64).reshape(-1, 18, 18, NCH)
    if rounding:
        x = bf16_round(x)
    Wq = [r(w) for w in W]
    a1 = r(np.maximum(conv3x3(x, Wq[0]) + b[0], 0.0))
    a2 = r(np.maximum(conv3x3(_pad(a1), Wq[1]) + b[1], 0.0))
    a3 = r(np.maximum(conv3x3(_pad(a2), Wq[2]) + b[2], 0.0))
    v = a3.reshape(len(x), -1, NCH).mean(axis=1)
    z = v @ wh + bh
    return dict(x=x, Wq=Wq, a1=a1, a2=a2, a3=a3, v=v, z=z)


def loss_and_grad(x0, y, prm, pos_weight=1.0, rounding=True):
    """Mean weighted cross-entropy and its gradient with respect to prm."""
    W, b, wh, bh = unpack(prm)
    r = bf16_round if rounding else (lambda t: t)
    f = forward(x0, prm, rounding)
    y = np.asarray(y, dtype=np.float64)
    n = len(y)
    z = f["z"]
    w = np.where(y > 0.5, pos_weight, 1.0)
    loss = float(np.sum(w * (np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z))))) / n)
    dz = w * (1.0 / (1.0 + np.exp(-z)) - y) / n
    g_wh = f["v"].T @ dz
    g_bh = dz.sum()
    # through the mean pool and the relu of layer 3
    d3 = dz[:, None, None, None] * wh[None, None, None, :] / 256.0
    d3 = r(np.where(f["a3"] > 0, np.broadcast_to(d3, f["a3"].shape), 0.0))
    gW3 = conv3x3_wgrad(d3, _pad(f["a2"]))
    gb3 = d3.sum(axis=(0, 1, 2))
    d2 = conv3x3_adjoint(d3, f["Wq"][2])[:, 1:-1, 1:-1, :]
    d2 = r(np.where(f["a2"] > 0, d2, 0.0))
    gW2 = conv3x3_wgrad(d2, _pad(f["a1"]))
    gb2 = d2.sum(axis=(0, 1, 2))
    d1 = conv3x3_adjoint(d2, f["Wq"][1])[:, 1:-1, 1:-1, :]
    d1 = r(np.where(f["a1"] > 0, d1, 0.0))
    gW1 = conv3x3_wgrad(d1, f["x"])
    gb1 = d1.sum(axis=(0, 1, 2))
    grad = pack([gW1, gW2, gW3], [gb1, gb2, gb3], g_wh, g_bh)
    return loss, grad, f


def adam_step(prm, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015, Algorithm 1) at step t >= 1."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return prm - lr * mh / (np.sqrt(vh) + eps), m, v


def composite_fine(levels, pxs, pys, fields, mi, mj, mx):
    """Each field of a forest (fields [nf][npatch][mx][mx]) on the grid of its
    finest leaf level, every leaf's cell value filling the fine cells it
    covers; a cell of level L is then the mean of its fine block."""
    Lf = int(max(levels))
    out = np.zeros((len(fields), mj * mx << Lf, mi * mx << Lf))
    for k, (L, px, py) in enumerate(zip(levels, pxs, pys)):
        r = 1 << (Lf - int(L))
        x0, y0 = px * mx * r, py * mx * r
        for f, a in enumerate(fields):
            out[f, y0:y0 + mx * r, x0:x0 + mx * r] = np.kron(a[k], np.ones((r, r)))
    return out, Lf


def features(levels, pxs, pys, h, hu, hv, b, mi, mj, mx, scale):
    """Network input of every patch of a forest, [n, 18, 18, 16] before
    rounding.  Pixel (Y, X) of the inner 16 x 16 averages the f x f interior
    cells (f = mx / 16) starting at ((Y - 1) f, (X - 1) f); a ring pixel
    averages the band of same-level cells beyond the patch edge beside it,
    mx / 2 cells deep, over the composite of the forest, leaving out cells
    outside the domain (no cell inside: h, hu, hv and the relative bed are
    0).  Channel 3 is the bed minus the mean interior bed; channel 4 is
    level / 4."""
    fine, Lf = composite_fine(levels, pxs, pys, [h, hu, hv, b], mi, mj, mx)
    n = len(levels)
    f, W = mx // 16, mx // 2
    out = np.zeros((n, 18, 18, NCH))

    def span(k):
        if k == 0:
            return -W, 0
        if k == 17:
            return mx, mx + W
        return (k - 1) * f, k * f

    for p in range(n):
        L = int(levels[p])
        r = 1 << (Lf - L)
        NX, NY = mi * mx << L, mj * mx << L
        I0, J0 = pxs[p] * mx, pys[p] * mx
        bmean = np.mean(b[p])
        for Y in range(18):
            j0, j1 = span(Y)
            J_lo, J_hi = max(J0 + j0, 0), min(J0 + j1, NY)
            for X in range(18):
                i0, i1 = span(X)
                I_lo, I_hi = max(I0 + i0, 0), min(I0 + i1, NX)
                if I_lo >= I_hi or J_lo >= J_hi:
                    continue
                blk = fine[:, J_lo * r:J_hi * r, I_lo * r:I_hi * r]
                m = blk.reshape(4, -1).mean(axis=1)
                out[p, Y, X, :4] = (m - np.array([0, 0, 0, bmean])) / np.asarray(scale, float)
        out[p, :, :, 4] = 0.25 * L
    return out
