"""Proposal MLP kernels against the FP64 reference (oracle/mlp.py):
gradients of the GPU's fused forward/backward kernel, BF16 vs FP32
inference, and an Adam training run that lowers the loss."""
import ctypes as C

import numpy as np
import pytest

from oracle import mlp as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    from paper_2304_14969_gb300 import build, qsim
    build.build()
    qsim.lib()
    return qsim


def make(Q, nf, H, seed):
    h = C.c_void_p()
    Q.qsim_mlp_create(nf, H, seed, C.byref(h))
    cnt = C.c_int64()
    Q.qsim_mlp_num_params(h, C.byref(cnt))
    assert cnt.value == M.num_params(nf, H)
    return h, cnt.value


def fptr(a):
    return a.ctypes.data_as(C.c_void_p)


def test_gradients_match_reference(Q):
    nf, H = 12, 64
    h, npar = make(Q, nf, H, 1)
    rng = np.random.default_rng(2)
    X = rng.normal(0, 1, (300, nf)).astype(np.float32)
    y = (rng.uniform(size=300) < 0.3).astype(np.float32)
    theta = np.zeros(npar, dtype=np.float32)
    Q.qsim_mlp_get_params(h, fptr(theta))
    g = np.zeros(npar, dtype=np.float32)
    loss = C.c_float()
    Q.qsim_mlp_loss_grad(h, fptr(X), fptr(y), 300, C.byref(loss), fptr(g))
    L, gref = M.loss_grad(theta.astype(np.float64), X.astype(np.float64), y.astype(np.float64), nf, H)
    assert abs(loss.value - L) <= 1e-5 * max(1.0, abs(L))
    scale = np.max(np.abs(gref))
    assert np.max(np.abs(g - gref)) <= 1e-3 * scale
    Q.qsim_mlp_destroy(h)


def test_bf16_inference_close_to_fp32(Q):
    nf, H = 12, 64
    h, npar = make(Q, nf, H, 3)
    rng = np.random.default_rng(4)
    X = rng.normal(0, 1, (257, nf)).astype(np.float32)
    out32 = np.zeros(257, dtype=np.float32)
    out16 = np.zeros(257, dtype=np.float32)
    Q.qsim_mlp_infer(h, fptr(X), 257, 0, fptr(out32))
    Q.qsim_mlp_infer(h, fptr(X), 257, 1, fptr(out16))
    theta = np.zeros(npar, dtype=np.float32)
    Q.qsim_mlp_get_params(h, fptr(theta))
    zref, _ = M.forward(theta.astype(np.float64), X.astype(np.float64), nf, H)
    assert np.max(np.abs(out32 - zref)) <= 1e-4 * max(1.0, np.max(np.abs(zref)))
    # BF16 weights: 8 significant bits, FP32 accumulation
    assert np.max(np.abs(out16 - zref)) <= 3e-2 * max(1.0, np.max(np.abs(zref)))
    Q.qsim_mlp_destroy(h)


def test_training_lowers_loss(Q):
    nf, H = 12, 64
    h, npar = make(Q, nf, H, 5)
    rng = np.random.default_rng(6)
    X = rng.normal(0, 1, (2000, nf)).astype(np.float32)
    y = (X[:, 0] + 0.5 * X[:, 3] > 0.2).astype(np.float32)
    loss = C.c_float()
    first = None
    for it in range(200):
        Q.qsim_mlp_train_step(h, fptr(X), fptr(y), 2000, C.c_float(3e-3), C.byref(loss))
        if first is None:
            first = loss.value
    assert loss.value < 0.5 * first
    Q.qsim_mlp_destroy(h)
