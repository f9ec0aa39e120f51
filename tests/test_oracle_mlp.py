"""Pins of the FP64 MLP reference: central finite differences of the loss
match the hand-written backward pass, the loss matches the
cross-entropy written out directly for a tiny case, and the Adam step
(Kingma and Ba 2015, Algorithm 1) matches its first two steps computed by
hand."""
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


def test_adam_first_step_by_hand():
    """Step 1 from zero moments: m_hat = g, v_hat = g^2, so every parameter
    moves by lr * g / (|g| + eps): about lr against the sign of g, 0 where
    g = 0. A dropped bias correction would give 0.1 g / (sqrt(0.001) |g|)."""
    lr, eps = 0.01, 1e-8
    g = np.array([3.0, -0.5, 0.0, 2e-9])
    theta = np.array([1.0, 2.0, 3.0, 4.0])
    t1, m1, v1 = mlp.adam_step(theta, np.zeros(4), np.zeros(4), g, 1, lr)
    want = theta - lr * g / (np.abs(g) + eps)
    assert np.max(np.abs(t1 - want)) < 1e-15
    assert np.allclose(m1, 0.1 * g, rtol=1e-15, atol=0)
    assert np.allclose(v1, 0.001 * g * g, rtol=1e-15, atol=0)
    # the last parameter's gradient is below eps: its step is lr g / (g + eps) = lr / 6
    assert abs((theta[3] - t1[3]) - lr * 2e-9 / 1.2e-8) < 1e-15


def test_adam_second_step_by_hand():
    """Step 2 with gradients g1 then g2, written out:
    m2 = 0.09 g1 + 0.1 g2, v2 = 0.000999 g1^2 + 0.001 g2^2,
    theta2 = theta1 - lr (m2 / 0.19) / (sqrt(v2 / 0.001999) + eps)."""
    lr, eps = 0.05, 1e-8
    g1, g2 = np.array([1.0, -2.0]), np.array([3.0, 0.5])
    theta0 = np.array([0.25, -0.75])
    t1, m1, v1 = mlp.adam_step(theta0, np.zeros(2), np.zeros(2), g1, 1, lr)
    t2, m2, v2 = mlp.adam_step(t1, m1, v1, g2, 2, lr)
    m2h = (0.09 * g1 + 0.1 * g2) / 0.19
    v2h = (0.000999 * g1 ** 2 + 0.001 * g2 ** 2) / 0.001999
    want = theta0 - lr * g1 / (np.abs(g1) + eps) - lr * m2h / (np.sqrt(v2h) + eps)
    assert np.max(np.abs(t2 - want)) < 1e-14


def test_adam_training_lowers_loss():
    """A few hundred Adam steps on a separable problem lower the loss of the
    FP64 network well below log 2 (the loss at z = 0)."""
    nf, H = 3, 8
    rng = np.random.default_rng(1)
    X = rng.normal(0, 1, (200, nf))
    y = (X[:, 0] - 0.5 * X[:, 1] > 0).astype(float)
    theta0 = rng.normal(0, 0.3, mlp.num_params(nf, H))
    theta, losses = mlp.train(theta0, X, y, nf, H, 0.02, 300)
    assert mlp.loss(theta, X, y, nf, H) < 0.3 < losses[0]
