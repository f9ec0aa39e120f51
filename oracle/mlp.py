"""FP64 reference of the proposal MLP (test infrastructure only).

nfeat -> H -> H -> 1 logit with ReLU, loss = mean binary cross-entropy with
logits. Parameter vector layout: W1[H][nfeat], b1[H], W2[H][H], b2[H],
W3[H], b3. numpy matrix products serve as the primitive; the backward pass
is the chain rule written out layer by layer. Pinned by central finite
differences in tests/test_oracle_mlp.py.

The optimiser step is Adam as published (Kingma and Ba, "Adam: A Method for
Stochastic Optimization", ICLR 2015, Algorithm 1), in FP64: exponential
moving averages of the gradient and of its square, each divided by its
bias correction, and a step of lr times their ratio. Pinned by hand-computed
first and second steps in tests/test_oracle_mlp.py.
"""
import numpy as np


def unpack(theta, nf, H):
    theta = np.asarray(theta, dtype=np.float64)
    o = 0
    W1 = theta[o:o + H * nf].reshape(H, nf); o += H * nf
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + H * H].reshape(H, H); o += H * H
    b2 = theta[o:o + H]; o += H
    W3 = theta[o:o + H]; o += H
    b3 = theta[o]; o += 1
    assert o == theta.size
    return W1, b1, W2, b2, W3, b3


def num_params(nf, H):
    return H * nf + H + H * H + H + H + 1


def forward(theta, X, nf, H):
    W1, b1, W2, b2, W3, b3 = unpack(theta, nf, H)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0.0)
    z = a2 @ W3 + b3
    return z, (X, z1, a1, z2, a2)


def loss(theta, X, y, nf, H):
    z, _ = forward(theta, X, nf, H)
    y = np.asarray(y, dtype=np.float64)
    # softplus(z) - y z, written stably
    return float(np.mean(np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z)))))


def loss_grad(theta, X, y, nf, H):
    W1, b1, W2, b2, W3, b3 = unpack(theta, nf, H)
    z, (X, z1, a1, z2, a2) = forward(theta, X, nf, H)
    y = np.asarray(y, dtype=np.float64)
    m = X.shape[0]
    L = float(np.mean(np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z)))))
    dz = (1.0 / (1.0 + np.exp(-z)) - y) / m          # dL/dz
    gW3 = a2.T @ dz
    gb3 = dz.sum()
    da2 = np.outer(dz, W3)
    dz2 = da2 * (z2 > 0)
    gW2 = dz2.T @ a1
    gb2 = dz2.sum(axis=0)
    da1 = dz2 @ W2
    dz1 = da1 * (z1 > 0)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])
    return L, g


def adam_step(theta, m, v, g, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t >= 1 (Kingma and Ba 2015, Algorithm 1).
    Returns the new (theta, m, v); the inputs are not modified."""
    theta = np.asarray(theta, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return theta - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def train(theta, X, y, nf, H, lr, steps):
    """`steps` Adam steps of the mean BCE loss on (X, y) from theta, moments
    starting at zero. Returns (theta, losses), losses[t] at the start of
    step t + 1."""
    theta = np.asarray(theta, dtype=np.float64).copy()
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    losses = []
    for t in range(1, steps + 1):
        L, g = loss_grad(theta, X, y, nf, H)
        losses.append(L)
        theta, m, v = adam_step(theta, m, v, g, t, lr)
    return theta, losses
