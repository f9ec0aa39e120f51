"""The oracle's all-core build (the same oracle.c compiled with -fopenmp)
against its one-thread build, which the pins in test_oracle_pins.py check.

Element-wise loops (gate application, probabilities, projection) split their
iterations across threads without changing any arithmetic, so their results
are bit-identical. Sums are split into per-thread compensated partials and
merged, so they agree to within the compensated sums' error (a few ulp of
the sum of magnitudes)."""
import numpy as np
import pytest

import oracle
from paper_2304_14969_gb300 import workloads as W


@pytest.fixture
def both():
    def call(fn, *a):
        oracle.use_all_cores(False)
        r1 = fn(*a)
        oracle.use_all_cores(True)
        try:
            r2 = fn(*a)
        finally:
            oracle.use_all_cores(False)
        return r1, r2
    return call


def test_all_core_build_uses_several_threads():
    oracle.use_all_cores(True)
    try:
        nt = oracle.threads()
    finally:
        oracle.use_all_cores(False)
    assert oracle.threads() == 1
    assert nt >= 1


@pytest.mark.parametrize("which", ["qft", "grid", "random", "paper"])
def test_gate_application_bit_identical(both, which):
    if which == "qft":
        n, g = 14, W.qft_circuit(14)
    elif which == "grid":
        n, g = 12, W.grid_rcs_circuit(3, 4, 6, seed=1)
    elif which == "random":
        n, g = 13, W.random_1q_circuit(13, 120, 3)
    else:
        n, g = 12, W.paper_random_circuit(3, 4, 5, seed=2)
    x = W.gaussian_state(n, 4)
    a, b = both(oracle.apply_circuit, x, g)
    assert np.array_equal(a.view(np.float64), b.view(np.float64))


def test_block_and_probs_bit_identical(both):
    n = 13
    x = W.gaussian_state(n, 5)
    U = W.random_unitary(5, 6)
    a, b = both(oracle.apply_kq, x, [12, 0, 7, 3, 9], U)
    assert np.array_equal(a.view(np.float64), b.view(np.float64))
    pa, pb = both(oracle.probs, a)
    assert np.array_equal(pa, pb)


def test_sums_agree(both):
    n = 16
    x = W.gaussian_state(n, 7)
    y = W.gaussian_state(n, 8)
    tol = 8 * np.finfo(float).eps
    a, b = both(oracle.norm2, x)
    assert abs(a - b) <= tol * a
    a, b = both(oracle.inner, x, y)
    assert abs(a - b) <= tol * np.sum(np.abs(x) * np.abs(y))
    for q in (0, 7, 15):
        a, b = both(oracle.prob1, x, q)
        assert abs(a - b) <= tol
        ra, rb = both(oracle.bloch, x, q)
        assert np.max(np.abs(ra - rb)) <= tol
    a, b = both(oracle.dft_sample, x, 12345)
    assert abs(a - b) <= tol * np.sum(np.abs(x)) / np.sqrt(x.size)


@pytest.mark.parametrize("p", [0.1, 0.4])
def test_sdrp_run_same_decisions(both, p):
    n = 12
    g = W.grid_rcs_circuit(3, 4, 6, seed=3)
    (pa, Fa, na, la), (pb, Fb, nb, lb) = both(oracle.sdrp_run, n, g, p, 1e-13)
    assert na == nb
    assert list(la["action"]) == list(lb["action"]) and list(la["qubit"]) == list(lb["qubit"])
    assert np.max(np.abs(la["eps"] - lb["eps"])) <= 1e-13
    assert abs(Fa - Fb) <= 1e-13
    assert abs(abs(np.vdot(pa, pb)) ** 2 - 1) <= 1e-12
