"""FP64 oracle of the learned rank / skeleton proposer (test infrastructure only).

The proposer is not part of the paper's method: it is the learned addition of the
project's brief (a small MLP that, from a box's geometry and the tolerance, proposes
the box's column-ID ranks and where its skeleton lies; every proposal is checked
against the ID tolerance and otherwise replaced by the plain ID of Sec. 4.1).  This
module states, in plain numpy FP64, what the GPU path computes:

* ``box_features``: the 128 input features of one box;
* ``box_targets``: the training targets the plain ID yields for that box;
* ``forward`` / ``loss_and_grad`` / ``adam_step``: the network, its loss, gradients
  and optimiser step, with the weights rounded to FP16 before use (the network keeps
  FP32 master weights and evaluates with their FP16 copy; gradients are taken with
  respect to the FP16 values).

Network: x (128) -> ReLU(W1 x + b1) (128) -> ReLU(W2 h1 + b2) (128) -> W3 h2 + b3 (128, of
which outputs 0..65 are used).  Output 0 / 1: log2(1 + rank) / 8 of the flux / trace
half; outputs 2..33 / 34..65: skeleton logits of the flux / trace half at 32 positions
along the box.  Parameters are packed [W1 (row-major 128 x 128), b1, W2, b2, W3, b3].

Loss over a batch of B boxes:
    L = (1/B) sum_b sum_h (o_bh - y_bh)^2
        + (lam / (64 B)) sum_b sum_(h,j) mask_bhj * BCE(sigmoid(o_b,2+32h+j), t_bhj),
BCE(p, t) = -(t log p + (1 - t) log(1 - p)), lam = 0.1.

Pins (tests/test_oracle_mlp.py): central finite differences of the loss reproduce the
gradients; the bias-only network has a closed-form gradient; planted mistakes in the
backward pass fail the difference check; features of a disk box are the circle's.
"""

from __future__ import annotations

import math

import numpy as np

WIDTH = 128
N_OUT_USED = 66
N_POS = 32
LAM = 0.1
LAYER_SHAPES = [(WIDTH, WIDTH), (WIDTH, WIDTH), (WIDTH, WIDTH)]
N_PARAMS = sum(o * i + o for o, i in LAYER_SHAPES)


def unpack(p: np.ndarray):
    """[(W, b)] views of the packed parameter vector."""
    out, off = [], 0
    for o, i in LAYER_SHAPES:
        W = p[off:off + o * i].reshape(o, i)
        off += o * i
        b = p[off:off + o]
        off += o
        out.append((W, b))
    return out


def fp16(p: np.ndarray) -> np.ndarray:
    """Round to IEEE half precision (round to nearest even) and back to float64."""
    return np.asarray(p, dtype=np.float64).astype(np.float16).astype(np.float64)


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights, zero biases (float32 master values)."""
    rng = np.random.default_rng(seed)
    parts = []
    for li, (o, i) in enumerate(LAYER_SHAPES):
        bound = math.sqrt(6.0 / i) * (0.25 if li == 2 else 1.0)
        W = rng.uniform(-bound, bound, size=(o, i))
        if li == 2:
            W[N_OUT_USED:, :] = 0.0
        parts += [W.ravel(), np.zeros(o)]
    return np.concatenate(parts).astype(np.float32)


def forward(p16: np.ndarray, x: np.ndarray):
    """Outputs (B x 128) and the hidden activations, all in float64."""
    (W1, b1), (W2, b2), (W3, b3) = unpack(p16)
    z1 = x @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    o = h2 @ W3.T + b3
    return o, (x, z1, h1, z2, h2)


def _sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def loss_and_grad(p16: np.ndarray, x, y_rank, y_skel, mask):
    """Loss and its gradient with respect to the (FP16-valued) parameters.

    x: B x 128, y_rank: B x 2, y_skel / mask: B x 64.
    """
    B = x.shape[0]
    o, (x0, z1, h1, z2, h2) = forward(p16, x)
    r = o[:, 0:2] - y_rank
    s = o[:, 2:N_OUT_USED]
    ps = _sigmoid(s)
    eps = 1e-300
    bce = -(y_skel * np.log(np.maximum(ps, eps)) + (1.0 - y_skel) * np.log(np.maximum(1.0 - ps, eps)))
    loss = np.sum(r * r) / B + LAM / (64.0 * B) * np.sum(mask * bce)
    do = np.zeros_like(o)
    do[:, 0:2] = 2.0 * r / B
    do[:, 2:N_OUT_USED] = LAM / (64.0 * B) * mask * (ps - y_skel)
    (W1, b1), (W2, b2), (W3, b3) = unpack(p16)
    gW3 = do.T @ h2
    gb3 = do.sum(axis=0)
    dh2 = do @ W3
    dz2 = dh2 * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (z1 > 0)
    gW1 = dz1.T @ x0
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return float(loss), g


def adam_step(master, m, v, g, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) of the master weights; returns new (master, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return master - lr * mh / (np.sqrt(vh) + eps), m, v


# ------------------------------------------------------------------ features and targets

def box_features(x, y, kappa, begin: int, end: int, cx: float, cy: float, rho: float, k0: float, k1: float,
                 tol: float, height: int, n_act0: int, n_act1: int, m_near: int, nproxy: int) -> np.ndarray:
    """The 128 features of a box whose nodes are [begin, end) of the curve arrays.

    For j = 0..31 the node q_j = begin + ((2j + 1) L) // 64 (L = end - begin) gives
    ((x - cx)/rho, (y - cy)/rho, kappa rho); then 2 rho k0 / 32, 2 rho k1 / 32,
    -log10(tol) / 10, height / 8, log2(1 + n_act0) / 8, log2(1 + n_act1) / 8,
    log2(1 + m_near) / 8, nproxy / 256, and zeros.  rho = 0 is read as 1.
    """
    L = end - begin
    r = rho if rho > 0 else 1.0
    f = np.zeros(WIDTH)
    for j in range(N_POS):
        q = begin + ((2 * j + 1) * L) // 64
        f[3 * j] = (x[q] - cx) / r
        f[3 * j + 1] = (y[q] - cy) / r
        f[3 * j + 2] = kappa[q] * r
    f[96] = 2.0 * rho * k0 / 32.0
    f[97] = 2.0 * rho * k1 / 32.0
    f[98] = -math.log10(tol) / 10.0 if tol > 0 else 3.2
    f[99] = height / 8.0
    f[100] = math.log2(1 + n_act0) / 8.0
    f[101] = math.log2(1 + n_act1) / 8.0
    f[102] = math.log2(1 + m_near) / 8.0
    f[103] = nproxy / 256.0
    return f


def box_targets(begin: int, end: int, act, skel):
    """Targets from a plain ID: act[h] active node indices of half h, skel[h] its skeleton.

    y_rank[h] = log2(1 + |skel[h]|) / 8; an active node q sits at position
    ((q - begin) * 32) // L; t[h][j] is the fraction of the active nodes at position j
    that are skeleton nodes, mask[h][j] = 1 where position j holds an active node.
    """
    L = end - begin
    yr = np.zeros(2)
    t = np.zeros(64)
    mask = np.zeros(64)
    for h in range(2):
        yr[h] = math.log2(1 + len(skel[h])) / 8.0
        cnt = np.zeros(N_POS)
        hit = np.zeros(N_POS)
        sk = set(int(q) for q in skel[h])
        for q in act[h]:
            j = ((int(q) - begin) * N_POS) // L
            cnt[j] += 1
            hit[j] += 1 if int(q) in sk else 0
        for j in range(N_POS):
            if cnt[j] > 0:
                t[32 * h + j] = hit[j] / cnt[j]
                mask[32 * h + j] = 1.0
    return yr, t, mask


def rank_from_output(o: float) -> float:
    """Inverse of the rank target: 2^(8 o) - 1."""
    return 2.0 ** (8.0 * o) - 1.0
