"""Pins of the proposer's FP64 oracle (oracle/mlp.py) that do not use the oracle against itself:

* central finite differences of the loss reproduce the analytic gradient (every layer, both
  loss terms, masked positions);
* planted mistakes in the backward pass (wrong ReLU derivative, dropped mask, transposed
  weight) are caught by the same difference check;
* a network with zero weights outputs its last bias, whose gradient has a closed form;
* the Adam step matches its first-step closed form (update = -lr * sign(g) up to eps);
* the features of a box of the unit disk lie on the unit circle in the box frame, with
  curvature feature = rho, and the targets count skeleton nodes per position.
"""

import math

import numpy as np
import pytest

from oracle import mlp as M


def _batch(seed, B=6):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(B, M.WIDTH)) * 0.5
    yr = rng.uniform(0.2, 0.8, size=(B, 2))
    ys = rng.uniform(0.0, 1.0, size=(B, 64))
    mask = (rng.uniform(size=(B, 64)) < 0.7).astype(float)
    return x, yr, ys, mask


def _params(seed):
    rng = np.random.default_rng(seed)
    p = M.init_params(seed).astype(np.float64)
    # non-zero biases so every ReLU region is exercised
    off = 0
    for o, i in M.LAYER_SHAPES:
        off += o * i
        p[off:off + o] = rng.normal(size=o) * 0.1
        off += o
    return p


def _fd_check(loss_grad, p, x, yr, ys, mask, idx, h=1e-6):
    _, g = loss_grad(p, x, yr, ys, mask)
    floor = 1e-3 * np.abs(g).max()
    worst = 0.0
    for k in idx:
        e = np.zeros_like(p)
        e[k] = h
        lp, _ = M.loss_and_grad(p + e, x, yr, ys, mask)
        lm, _ = M.loss_and_grad(p - e, x, yr, ys, mask)
        fd = (lp - lm) / (2 * h)
        worst = max(worst, abs(fd - g[k]) / max(floor, abs(fd)))
    return worst


def _sample_indices(seed, n=60):
    rng = np.random.default_rng(seed)
    idx = []
    off = 0
    for li, (o, i) in enumerate(M.LAYER_SHAPES):
        rows = range(o) if li < 2 else range(M.N_OUT_USED)
        rr = rng.choice(list(rows), size=n // 6)
        cc = rng.integers(0, i, size=n // 6)
        idx += [off + r * i + c for r, c in zip(rr, cc)]
        off += o * i
        idx += list(off + rng.choice(list(rows), size=n // 6))
        off += o
    return idx


def test_gradient_matches_finite_differences():
    p = _params(1)
    x, yr, ys, mask = _batch(2)
    worst = _fd_check(M.loss_and_grad, p, x, yr, ys, mask, _sample_indices(3))
    assert worst < 1e-5


def _broken(kind):
    def lg(p16, x, y_rank, y_skel, mask):
        B = x.shape[0]
        o, (x0, z1, h1, z2, h2) = M.forward(p16, x)
        r = o[:, 0:2] - y_rank
        ps = 1 / (1 + np.exp(-o[:, 2:66]))
        do = np.zeros_like(o)
        do[:, 0:2] = 2.0 * r / B
        mk = np.ones_like(mask) if kind == "mask" else mask
        do[:, 2:66] = M.LAM / (64.0 * B) * mk * (ps - y_skel)
        (W1, b1), (W2, b2), (W3, b3) = M.unpack(p16)
        gW3 = do.T @ h2
        dh2 = do @ W3
        dz2 = dh2 * ((z2 >= -0.05) if kind == "relu" else (z2 > 0))
        gW2 = dz2.T @ h1
        dh1 = dz2 @ (W2.T if kind == "transpose" else W2)
        dz1 = dh1 * (z1 > 0)
        gW1 = dz1.T @ x0
        g = np.concatenate([gW1.ravel(), dz1.sum(0), gW2.ravel(), dz2.sum(0), gW3.ravel(), do.sum(0)])
        return 0.0, g
    return lg


@pytest.mark.parametrize("kind", ["relu", "mask", "transpose"])
def test_planted_backward_mistakes_are_caught(kind):
    p = _params(4)
    x, yr, ys, mask = _batch(5)
    assert _fd_check(_broken(kind), p, x, yr, ys, mask, _sample_indices(6, 120)) > 1e-3


def test_bias_only_network_closed_form():
    p = np.zeros(M.N_PARAMS)
    rng = np.random.default_rng(7)
    b3 = rng.normal(size=M.WIDTH) * 0.3
    p[-M.WIDTH:] = b3
    x, yr, ys, mask = _batch(8, B=5)
    loss, g = M.loss_and_grad(p, x, yr, ys, mask)
    B = x.shape[0]
    sig = 1 / (1 + np.exp(-b3[2:66]))
    exp_b3 = np.zeros(M.WIDTH)
    exp_b3[0:2] = 2.0 * (b3[0:2] - yr).sum(0) / B
    exp_b3[2:66] = M.LAM / (64.0 * B) * (mask * (sig - ys)).sum(0)
    assert np.allclose(g[-M.WIDTH:], exp_b3, rtol=1e-12, atol=1e-15)
    assert np.all(g[:-M.WIDTH] == 0.0)
    bce = -(ys * np.log(sig) + (1 - ys) * np.log(1 - sig))
    exp_loss = ((b3[0:2] - yr) ** 2).sum() / B + M.LAM / (64.0 * B) * (mask * bce).sum()
    assert abs(loss - exp_loss) < 1e-12


def test_adam_first_step_is_signed_lr():
    rng = np.random.default_rng(9)
    g = rng.normal(size=50)
    w = rng.normal(size=50)
    w1, m, v = M.adam_step(w, np.zeros(50), np.zeros(50), g, step=1, lr=1e-3)
    assert np.allclose(w1 - w, -1e-3 * np.sign(g), atol=1e-9)


def test_fp16_rounding_is_ieee_half():
    assert M.fp16(np.array([1.0 + 2 ** -11]))[0] == 1.0          # ties to even
    assert M.fp16(np.array([1.0 + 3 * 2 ** -11]))[0] == 1.0 + 2 ** -9
    assert M.fp16(np.array([65504.0]))[0] == 65504.0


def test_disk_box_features_and_targets():
    n = 256
    th = 2 * np.pi * np.arange(n) / n
    x, y, kap = np.cos(th), np.sin(th), np.ones(n)
    b, e = 64, 96
    cx, cy = x[b:e].mean(), y[b:e].mean()
    rho = np.hypot(x[b:e] - cx, y[b:e] - cy).max()
    f = M.box_features(x, y, kap, b, e, cx, cy, rho, 10.0, 20.0, 1e-10, 2, 32, 32, 50, 64)
    px = f[0:96:3] * rho + cx
    py = f[1:96:3] * rho + cy
    assert np.allclose(px ** 2 + py ** 2, 1.0, atol=1e-12)
    assert np.allclose(f[2:96:3], rho)
    assert abs(f[96] - 2 * rho * 10 / 32) < 1e-15 and abs(f[98] - 1.0) < 1e-15
    assert abs(f[100] - math.log2(33) / 8) < 1e-15 and np.all(f[104:] == 0)
    # every position holds one node; skeleton = even positions of the flux half
    act = [np.arange(b, e), np.arange(b, e)]
    skel = [np.arange(b, e, 2), np.array([b + 3])]
    yr, t, mask = M.box_targets(b, e, act, skel)
    assert abs(yr[0] - math.log2(17) / 8) < 1e-15 and abs(yr[1] - 1 / 8) < 1e-15
    assert np.all(mask == 1)
    assert np.all(t[0:32:2] == 1) and np.all(t[1:32:2] == 0)
    assert t[32 + 3] == 1 and t[32:].sum() == 1
