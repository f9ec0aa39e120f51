"""Pins of the FP64 MLP reference: central finite differences of the loss
match the hand-written backward pass, and the loss matches the
cross-entropy written out directly for a tiny case."""
import math

import numpy as np

from oracle import mlp


def test_backward_matches_finite_differences():
    nf, H = 5, 7
    rng = np.random.default_rng(0)
    theta = rng.normal(0, 0.5, mlp.num_params(nf, H))
    X = rng.normal(0, 1, (40, nf))
    y = (rng.uniform(size=40) < 0.4).astype(float)
    L, g = mlp.loss_grad(theta, X, y, nf, H)
    h = 1e-6
    for i in rng.choice(theta.size, 40, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss(tp, X, y, nf, H) - mlp.loss(tm, X, y, nf, H)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd)


def test_loss_tiny_case_by_hand():
    nf, H = 1, 1
    # W1=1, b1=0, W2=1, b2=0, W3=2, b3=-1 ; x=3 -> z = 2*3 - 1 = 5
    theta = np.array([1.0, 0.0, 1.0, 0.0, 2.0, -1.0])
    z, _ = mlp.forward(theta, [[3.0]], nf, H)
    assert abs(z[0] - 5.0) < 1e-15
    want = -math.log(1 / (1 + math.exp(-5.0)))        # y = 1
    assert abs(mlp.loss(theta, [[3.0]], [1.0], nf, H) - want) < 1e-12
