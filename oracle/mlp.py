"""Oracle: the learned initial-guess model, FP64 numpy forward / backward.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper has no learned component; the model is the one the benchmark
configuration asks for: a 3-layer MLP of width 128 mapping per-amplitude
features to T2.  To keep the guess covariant under spinor phase changes it
predicts a complex multiplier of the first-order amplitude:

    x   = (|t_MP2| / 0.05, -D_ij^ab / 10, |<ij||ab>| / max|<ij||ab>|)
    h1  = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  y = W3 h2 + b3
    t2  = (1 + y_0 + i y_1) t_MP2

Loss over a batch of n elements: L = (1/n) sum |t2_pred - t2_target|^2 / 0.05^2.
Parameters are flattened in the order W1 (128x3), b1, W2 (128x128), b2,
W3 (2x128), b3.  Parity: tests/test_oracle_mlp.py checks the gradient against
central finite differences of this loss (a check by the definition of a
derivative, independent of the backward pass below).
"""
from __future__ import annotations

import numpy as np

NF, W, NO = 3, 128, 2
SHAPES = [(W, NF), (W,), (W, W), (W,), (NO, W), (NO,)]
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES)


def unflatten(p):
    out, k = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(np.asarray(p[k:k + n], dtype=np.float64).reshape(s))
        k += n
    return out


def features(tmp2_abs, D, v_abs, v_max):
    return np.stack([tmp2_abs / 0.05, -D / 10.0, v_abs / v_max], axis=-1)


def forward(p, x):
    W1, b1, W2, b2, W3, b3 = unflatten(p)
    z1 = x @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3.T + b3
    return y, (x, z1, h1, z2, h2)


def loss(p, x, tmp2, target):
    """tmp2, target: complex arrays (n,)."""
    y, _ = forward(p, x)
    pred = (1.0 + y[:, 0] + 1j * y[:, 1]) * tmp2
    return float(np.mean(np.abs(pred - target) ** 2) / 0.05 ** 2)


def loss_grad(p, x, tmp2, target):
    """Loss and its gradient (flattened like the parameters), by the chain rule."""
    W1, b1, W2, b2, W3, b3 = unflatten(p)
    y, (x, z1, h1, z2, h2) = forward(p, x)
    n = x.shape[0]
    m = 1.0 + y[:, 0] + 1j * y[:, 1]
    r = m * tmp2 - target
    L = float(np.mean(np.abs(r) ** 2) / 0.05 ** 2)
    # dL/dy0 = 2 Re(conj(r) tmp2) / (n 0.05^2), dL/dy1 = 2 Re(conj(r) i tmp2) / (n 0.05^2)
    c = 2.0 / (n * 0.05 ** 2)
    gy = np.stack([c * np.real(np.conj(r) * tmp2), c * np.real(np.conj(r) * 1j * tmp2)], axis=-1)
    gW3 = gy.T @ h2
    gb3 = gy.sum(0)
    gh2 = gy @ W3
    gz2 = gh2 * (z2 > 0)
    gW2 = gz2.T @ h1
    gb2 = gz2.sum(0)
    gh1 = gz2 @ W2
    gz1 = gh1 * (z1 > 0)
    gW1 = gz1.T @ x
    gb1 = gz1.sum(0)
    g = np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return L, g


def init_params(seed):
    """He-initialised hidden layers, zero output layer (the untrained model is the MP2 guess)."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((W, NF)) * np.sqrt(2.0 / NF)
    W2 = rng.standard_normal((W, W)) * np.sqrt(2.0 / W)
    return np.concatenate([W1.ravel(), np.zeros(W), W2.ravel(), np.zeros(W), np.zeros(NO * W), np.zeros(NO)])
