"""Pins of the FP64 CPU oracle against facts outside it: closed forms of
the paper, numpy library routines (FFT, SVD, kron-built dense matrices),
brute force on tiny inputs, identities and hand-derived textbook values.

A plausible mistake in the oracle (a dropped term, a wrong sign, a swapped
qubit index, a transposed matrix) fails at least one of these."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2304_14969_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

I2 = np.eye(2)
X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]])
Z = np.diag([1.0, -1.0]).astype(complex)
H = np.array([[1, 1], [1, -1]], dtype=complex) / math.sqrt(2)


# ------------------------------------------------------------------ QFT

def test_qft_textbook_golden():
    """Eq. (dft) values derived by hand (tests/golden/qft_textbook.txt)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "qft_textbook.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) >= 16
    for n, x, j, re, im in rows:
        n, x, j = int(n), int(x), int(j)
        y = oracle.apply_circuit(W.basis_state(n, x), W.qft_circuit(n))
        assert abs(y[j] - complex(float(re), float(im))) < 1e-15


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11])
def test_qft_basis_closed_form(n):
    """QFT|x> = 2^{-n/2} sum_k exp(2 pi i x k / 2^n) |k>."""
    N = 1 << n
    for seed in range(3):
        x = W.basis_index(n, seed)
        y = oracle.apply_circuit(W.basis_state(n, x), W.qft_circuit(n))
        k = np.arange(N)
        ref = np.exp(2j * np.pi * ((x * k) % N) / N) / math.sqrt(N)
        assert np.max(np.abs(y - ref)) < 1e-13 * max(1, n)


@pytest.mark.parametrize("n", [2, 4, 7, 10, 13])
def test_qft_gaussian_matches_numpy_fft(n):
    """The DFT of Eq. (dft) with w = exp(+2 pi i/N) is numpy's ifft * sqrt(N)."""
    x = W.gaussian_state(n, 7 + n)
    y = oracle.apply_circuit(x, W.qft_circuit(n))
    ref = np.fft.ifft(x) * math.sqrt(1 << n)
    assert np.max(np.abs(y - ref)) < 1e-13


def test_qft_zero_and_ghz_closed_forms():
    n = 9
    N = 1 << n
    y0 = oracle.apply_circuit(W.basis_state(n, 0), W.qft_circuit(n))
    assert np.max(np.abs(y0 - 1 / math.sqrt(N))) < 1e-14
    yg = oracle.apply_circuit(W.ghz_state(n), W.qft_circuit(n))
    k = np.arange(N)
    ref = (1 + np.exp(2j * np.pi * (((N - 1) * k) % N) / N)) / math.sqrt(2 * N)
    assert np.max(np.abs(yg - ref)) < 1e-14


def test_dft_sample_matches_numpy():
    n = 12
    x = W.gaussian_state(n, 3)
    ref = np.fft.ifft(x) * math.sqrt(1 << n)
    for j in [0, 1, 5, 1000, (1 << n) - 1]:
        assert abs(oracle.dft_sample(x, j) - ref[j]) < 1e-14


def test_qft_gate_count():
    for n, want in [(16, 144), (27, 391), (30, 480), (33, 577)]:
        assert len(W.qft_circuit(n)) == want


# ------------------------------------------------------- gate matrices

def test_gate_matrix_identities():
    m = lambda name, *p: oracle.gate_matrix(W.Gate(name, (0,) if name not in W.TWO_QUBIT else (0, 1), p))
    W_ = (X + Y) / math.sqrt(2)
    assert np.allclose(m("h"), H, atol=1e-15)
    assert np.allclose(m("sqrtx") @ m("sqrtx"), X, atol=1e-15)
    assert np.allclose(m("sqrty") @ m("sqrty"), Y, atol=1e-15)
    assert np.allclose(m("sqrtw") @ m("sqrtw"), W_, atol=1e-15)
    assert np.allclose(m("s") @ m("s"), Z, atol=1e-15)
    assert np.allclose(m("t") @ m("t"), m("s"), atol=1e-15)
    # Sec. III.C U(theta, phi, lambda): textbook special cases
    assert np.allclose(m("u3", math.pi, 0, math.pi), X, atol=1e-15)
    assert np.allclose(m("u3", math.pi / 2, 0, math.pi), H, atol=1e-15)
    assert np.allclose(m("u3", 0, 0, 0.3), m("phase", 0.3), atol=1e-15)
    assert np.allclose(m("u3", math.pi, math.pi / 2, math.pi / 2), Y, atol=1e-15)
    assert np.allclose(m("rz", 0.4), np.exp(-0.2j) * m("phase", 0.4), atol=1e-15)
    # two-qubit kinds on |00>,|01>,|10>,|11> with q0 = low bit
    cp = m("cp", 0.7)
    assert np.allclose(cp, np.diag([1, 1, 1, np.exp(0.7j)]), atol=1e-15)
    sw = m("swap")
    assert np.allclose(sw @ np.array([0, 1, 0, 0]), [0, 0, 1, 0])
    f = m("fsim", math.pi / 2, math.pi / 6)
    assert np.allclose(f @ np.array([0, 1, 0, 0]), [0, 0, -1j, 0], atol=1e-15)
    assert np.allclose(f @ np.array([0, 0, 0, 1]), [0, 0, 0, np.exp(-1j * math.pi / 6)], atol=1e-15)
    assert np.allclose(m("fsim", 0, 0), np.eye(4), atol=1e-15)
    for name in ("h", "x", "y", "z", "s", "t", "sqrtx", "sqrty", "sqrtw"):
        u = m(name)
        assert np.allclose(u.conj().T @ u, I2, atol=1e-15), name
    for u in (m("u3", 1.1, 2.2, 0.3), m("fsim", 0.4, 1.9), cp):
        assert np.allclose(u.conj().T @ u, np.eye(u.shape[0]), atol=1e-15)


# ------------------------------------------------------ dense and loops

def _kron_full(n, g):
    """Dense matrix of one gate from numpy kron products (test-side
    construction, independent of the oracle's element-wise builder)."""
    u = oracle.gate_matrix(W.Gate(g.name, g.qubits, g.params, (), (), g.matrix))
    N = 1 << n
    if len(g.qubits) == 1 and not g.controls:
        ops = [I2] * n
        ops[g.qubits[0]] = u
        M = np.array([[1.0 + 0j]])
        for q in range(n - 1, -1, -1):
            M = np.kron(M, ops[q])
        return M
    # general: permute so the acted-on qubits sit at the bottom, then embed
    M = np.zeros((N, N), dtype=complex)
    act = list(g.qubits)
    for c in range(N):
        for r in range(N):
            if any(((r >> q) & 1) != ((c >> q) & 1) for q in range(n) if q not in act):
                continue
            if g.controls and any(((c >> cq) & 1) != cv for cq, cv in zip(g.controls, g.cvals)):
                M[r, c] = 1.0 if r == c else 0.0
                continue
            lr = sum(((r >> q) & 1) << b for b, q in enumerate(act))
            lc = sum(((c >> q) & 1) << b for b, q in enumerate(act))
            M[r, c] = u[lr, lc]
    return M


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (3, 2), (4, 3), (5, 4)])
def test_dense_matches_kron_and_loops(n, seed):
    gates = W.random_1q_circuit(n, 14, seed)
    D = oracle.dense_circuit(n, gates)
    K = np.eye(1 << n, dtype=complex)
    for g in gates:
        K = _kron_full(n, g) @ K
    assert np.max(np.abs(D - K)) < 1e-13
    # the loop path agrees with the dense product on every basis state
    for x in range(1 << n):
        y = oracle.apply_circuit(W.basis_state(n, x), gates)
        assert np.max(np.abs(y - D[:, x])) < 1e-13


def test_single_qubit_kron_order():
    """Little-endian: X on qubit 0 maps index 0 to index 1; on qubit 2 to 4."""
    for q, want in [(0, 1), (2, 4)]:
        y = oracle.apply_circuit(W.basis_state(3, 0), [W.Gate("x", (q,))])
        assert abs(y[want] - 1) < 1e-15


def test_controls_and_anticontrols():
    # CX with control 1 (value 1) on target 0: |10> (index 2) -> |11> (index 3)
    y = oracle.apply_circuit(W.basis_state(2, 2), [W.Gate("x", (0,), (), (1,), (1,))])
    assert abs(y[3] - 1) < 1e-15
    # AX: fires on control value 0: |00> -> |01>
    y = oracle.apply_circuit(W.basis_state(2, 0), [W.Gate("x", (0,), (), (1,), (0,))])
    assert abs(y[1] - 1) < 1e-15
    y = oracle.apply_circuit(W.basis_state(2, 2), [W.Gate("x", (0,), (), (1,), (0,))])
    assert abs(y[2] - 1) < 1e-15


@pytest.mark.parametrize("n", [6, 9])
def test_circuit_times_inverse_is_identity_and_norm(n):
    x = W.gaussian_state(n, 11)
    g = W.random_1q_circuit(n, 60, 5)
    y = oracle.apply_circuit(x, g)
    assert abs(oracle.norm2(y) - 1) < 1e-13
    z = oracle.apply_circuit(y, W.inverse_circuit(g))
    assert np.max(np.abs(z - x)) < 1e-13
    q = W.qft_circuit(n)
    z = oracle.apply_circuit(oracle.apply_circuit(x, q), W.inverse_circuit(q))
    assert np.max(np.abs(z - x)) < 1e-13


def test_apply_kq_matches_sequential_and_dense():
    n = 7
    x = W.gaussian_state(n, 2)
    # kron of two one-qubit gates applied as a k=2 block == sequential
    a, b = W.random_unitary(1, 1), W.random_unitary(1, 2)
    blk = np.kron(b, a)  # row bit 0 <- qubits[0]
    y1 = oracle.apply_kq(x, [5, 2], blk)
    y2 = oracle.apply_circuit(x, [W.Gate("mat1", (5,), matrix=a), W.Gate("mat1", (2,), matrix=b)])
    assert np.max(np.abs(y1 - y2)) < 1e-14
    # k=2 block on (q0, q1) equals the mat2 gate on the same qubits
    U = W.random_unitary(2, 9)
    assert np.max(np.abs(oracle.apply_kq(x, [3, 6], U)
                         - oracle.apply_circuit(x, [W.Gate("mat2", (3, 6), matrix=U)]))) < 1e-14
    # k=3 block: check against numpy tensordot on the reshaped state
    U3 = W.random_unitary(3, 4)
    qs = [1, 6, 4]
    y = oracle.apply_kq(x, qs, U3)
    T = x.reshape([2] * n)          # axis a <-> qubit n-1-a
    axes = [n - 1 - q for q in reversed(qs)]  # U row index bits: qs[2] qs[1] qs[0]
    Ut = U3.reshape([2] * 6)
    R = np.tensordot(Ut, T, axes=([3, 4, 5], axes))
    R = np.moveaxis(R, [0, 1, 2], axes)
    assert np.max(np.abs(y - R.reshape(-1))) < 1e-14


# ---------------------------------------------------------- reductions

def test_reductions_brute_force():
    n = 10
    a, b = W.gaussian_state(n, 1), W.gaussian_state(n, 2)
    a2 = a * 1.7
    assert abs(oracle.norm2(a2) - np.sum(np.abs(a2) ** 2)) < 1e-13
    assert np.max(np.abs(oracle.probs(a) - np.abs(a) ** 2)) < 1e-17
    for q in (0, 4, 9):
        mask = (np.arange(1 << n) >> q) & 1 == 1
        assert abs(oracle.prob1(a, q) - np.sum(np.abs(a[mask]) ** 2)) < 1e-14
    assert abs(oracle.inner(a, b) - np.vdot(a, b)) < 1e-14
    assert abs(oracle.fidelity(a, a) - 1) < 1e-13


def _schmidt(psi, n, q):
    """Largest Schmidt branch of qubit q vs the rest from numpy's SVD."""
    T = np.moveaxis(psi.reshape([2] * n), n - 1 - q, 0).reshape(2, -1)
    U, s, Vh = np.linalg.svd(T, full_matrices=False)
    return U[:, 0], s, Vh[0]


def test_bloch_textbook_golden():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "sdrp_textbook.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) >= 5
    for name, q, eps, fid, *amps in rows:
        psi = np.array([float(v) for v in amps], dtype=np.complex128)
        r = oracle.bloch(psi, int(q))
        e = (1 - np.linalg.norm(r)) / 2
        assert abs(e - float(eps)) < 1e-14, name
        out = oracle.sdrp_project(psi, int(q), r)
        assert abs(oracle.fidelity(out, psi) - float(fid)) < 1e-14, name


@pytest.mark.parametrize("alpha", [0.1, 0.5, 1.0, 1.3])
def test_bloch_cos_sin_state(alpha):
    psi = np.zeros(4, dtype=np.complex128)
    psi[0], psi[3] = math.cos(alpha), math.sin(alpha)
    for q in (0, 1):
        r = oracle.bloch(psi, q)
        e = (1 - np.linalg.norm(r)) / 2
        assert abs(e - min(math.cos(alpha) ** 2, math.sin(alpha) ** 2)) < 1e-14


def test_bloch_product_state_is_pure_and_matches_factor():
    n = 6
    rest = W.gaussian_state(n - 1, 3)
    f = W.random_unitary(1, 8)[:, 0]
    for q in (0, 3, 5):
        # insert the one-qubit factor f at qubit q
        T = np.tensordot(f, rest.reshape([2] * (n - 1)), axes=0)  # axis0 = factor
        T = np.moveaxis(T, 0, n - 1 - q)
        psi = np.ascontiguousarray(T.reshape(-1))
        r = oracle.bloch(psi, q)
        s = np.conj(f[0]) * f[1]
        want = [2 * s.real, 2 * s.imag, abs(f[0]) ** 2 - abs(f[1]) ** 2]
        assert np.max(np.abs(r - want)) < 1e-14
        assert abs(np.linalg.norm(r) - 1) < 1e-14


@pytest.mark.parametrize("q", [0, 2, 6])
def test_projection_matches_svd_branch(q):
    """Eq. (sdrp): the projected state is the dominant Schmidt term, and
    eps = (1 - |r|)/2 is the smaller squared Schmidt coefficient; the
    fidelity to the input is 1 - eps (Sec. III.B)."""
    n = 7
    # weakly entangled state: a product state plus a small random part
    prod = np.kron(W.gaussian_state(n - 1, 1), np.array([1.0, 0.0]))
    psi = prod + 0.3 * W.gaussian_state(n, 2)
    psi /= np.linalg.norm(psi)
    psi = np.ascontiguousarray(psi.astype(np.complex128))
    r = oracle.bloch(psi, q)
    eps = (1 - np.linalg.norm(r)) / 2
    u, s, v = _schmidt(psi, n, q)
    assert abs(eps - s[1] ** 2) < 1e-13
    out = oracle.sdrp_project(psi, q, r)
    T = np.tensordot(u, v, axes=0)
    ref = np.moveaxis(T.reshape([2] + [2] * (n - 1)), 0, n - 1 - q).reshape(-1)
    assert abs(abs(np.vdot(ref, out)) - 1) < 1e-13
    assert abs(oracle.norm2(out) - 1) < 1e-13
    assert abs(oracle.fidelity(out, psi) - (1 - eps)) < 1e-13
    assert abs(np.linalg.norm(oracle.bloch(out, q)) - 1) < 1e-12


# ---------------------------------------------------------------- SDRP run

def test_sdrp_p0_is_exact():
    rows, cols = 3, 4
    g = W.grid_rcs_circuit(rows, cols, 4, seed=3)
    n = rows * cols
    psi, F, nr, log = oracle.sdrp_run(n, g, p=0.0, tau=1e-13)
    exact = oracle.apply_circuit(W.basis_state(n, 0), g)
    assert F == 1.0 and nr == 0
    assert abs(oracle.fidelity(psi, exact) - 1) < 1e-12


def test_sdrp_p0_separates_exactly_without_rounding():
    """QFT of |0...0> at p = 0: every controlled phase meets a control in |0>,
    so the checks find eps exactly 0; with p = 0 nothing rounds (exact
    simulation), each such check is an exact separation (action 2), and the
    result is the closed form of Eq. (dft) for x = 0."""
    n = 8
    psi, F, nr, log = oracle.sdrp_run(n, W.qft_circuit(n), p=0.0, tau=1e-13)
    assert F == 1.0 and nr == 0
    assert len(log) > 0 and set(int(a) for a in log["action"]) <= {0, 2} and (log["action"] == 2).any()
    assert abs(oracle.fidelity(psi, np.full(1 << n, 2.0 ** (-n / 2), dtype=np.complex128)) - 1) < 1e-12


def test_sdrp_single_projection_fidelity_is_exact():
    """With exactly one rounding, F = 1 - eps equals F_exact (Sec. III.B)."""
    n = 5
    g = [W.Gate("u3", (q,), (0.2 + 0.1 * q, 0.3, 0.1)) for q in range(n)]
    g += [W.Gate("x", (1,), (), (0,), (1,))]
    g += [W.Gate("u3", (q,), (1.1, 0.4 * q, 0.2)) for q in range(n)]
    g += [W.Gate("u3", (q,), (0.7, 0.1, 0.4 * q)) for q in range(n)]
    psi, F, nr, log = oracle.sdrp_run(n, g, p=0.2, tau=1e-13)
    assert nr == 1
    exact = oracle.apply_circuit(W.basis_state(n, 0), g)
    assert abs(F - oracle.fidelity(psi, exact)) < 1e-12
    rounded = log[log["action"] == 1]
    assert abs(F - (1 - rounded["eps"][0])) < 1e-15


def test_sdrp_p1_gives_product_state():
    rows, cols = 2, 4
    n = rows * cols
    g = W.grid_rcs_circuit(rows, cols, 3, seed=1)
    psi, F, nr, log = oracle.sdrp_run(n, g, p=1.0, tau=1e-13)
    assert nr > 0 and 0 < F < 1
    for q in range(n):
        assert abs(np.linalg.norm(oracle.bloch(psi, q)) - 1) < 1e-10
    assert abs(oracle.norm2(psi) - 1) < 1e-12


def test_sdrp_threshold_inclusive_and_log_consistent():
    rows, cols = 3, 3
    n = 9
    g = W.paper_random_circuit(rows, cols, 3, seed=4)
    psi, F, nr, log = oracle.sdrp_run(n, g, p=0.3, tau=1e-13)
    assert nr == int(np.sum(log["action"] == 1))
    assert np.all(log["eps"][log["action"] == 1] <= 0.15)
    assert np.all(log["eps"][log["action"] == 0] > 0.15)
    prod = np.prod(1 - log["eps"][log["action"] == 1])
    assert abs(F - prod) < 1e-14
    # replaying the same decisions through the forced schedule is identical
    force = np.stack([log["gate"], log["qubit"]], axis=1)
    psi2, F2, nr2, log2 = oracle.sdrp_run(n, g, p=0.3, tau=1e-13, force=force)
    assert F2 == F and np.array_equal(log2["action"], log["action"])
    assert np.max(np.abs(psi2 - psi)) == 0


def test_sdrp_forced_actions():
    """Replaying another run's decisions (the near-tie reading of Sec. III.A
    checks): forcing the natural decisions is bit-identical to the natural
    run; forcing a single rounding where eps > p/2 gives F = 1 - eps and a
    state at exactly that fidelity to the exact one (Sec. III.B, the
    per-projection fidelity); forcing a keep leaves the exact state."""
    n = 9
    g = W.paper_random_circuit(3, 3, 3, seed=4)
    psi, F, nr, log = oracle.sdrp_run(n, g, p=0.3, tau=1e-13)
    force = np.stack([log["gate"], log["qubit"]], axis=1)
    psi2, F2, nr2, log2 = oracle.sdrp_run(n, g, p=0.3, tau=1e-13, force=force, force_actions=log["action"])
    assert F2 == F and nr2 == nr and np.max(np.abs(psi2 - psi)) == 0
    exact = oracle.apply_circuit(W.basis_state(n, 0), g)
    # one forced check that would not round at p = 0.3
    j = int(np.flatnonzero((log["action"] == 0) & (log["eps"] > 0.2))[0])
    one = force[j:j + 1]
    psi3, F3, nr3, log3 = oracle.sdrp_run(n, g, p=0.3, tau=1e-13, force=one, force_actions=[1])
    assert nr3 == 1 and log3["action"][0] == 1
    eps = log3["eps"][0]
    assert abs(F3 - (1 - eps)) < 1e-15
    assert abs(oracle.fidelity(psi3, exact) - (1 - eps)) < 1e-12
    # one forced keep of a check that would round
    k = int(np.flatnonzero(log["action"] == 1)[0])
    psi4, F4, nr4, _ = oracle.sdrp_run(n, g, p=0.3, tau=1e-13, force=force[k:k + 1], force_actions=[0])
    assert F4 == 1.0 and nr4 == 0
    assert np.max(np.abs(psi4 - exact)) == 0


def _cx(c, t, v=1):
    return W.Gate("x", (t,), (), (c,), (v,))


def test_unobservable_definition_on_basis_input():
    """Sec. II.B: a transformation is unobservable when |<psi0|C'^dag C|psi0>|^2
    = 1. On a basis input every control is a Z eigenstate: CX with control
    |1> acts as a local X, with control |0> (or an anti-control in |1>) as
    nothing, a CP with either qubit in |0> as nothing and with one in |1> as
    a phase on the other. Every gate is reduced, nothing merges, no check
    runs, and the state equals the gate-by-gate result exactly."""
    n = 6
    g = [W.Gate("x", (0,)), W.Gate("x", (3,)),
         _cx(0, 1), _cx(1, 2), _cx(4, 5), _cx(0, 4, 0), _cx(2, 5, 0),
         W.Gate("cp", (0, 3), (0.7,)), W.Gate("cp", (4, 1), (0.3,)), W.Gate("cp", (5, 2), (1.1,)),
         W.Gate("x", (5,), (), (0, 3), (1, 1))]
    st = {}
    psi, F, nr, log = oracle.sdrp_run(n, g, p=0.5, tau=1e-13, unobservable=True, stats=st)
    assert len(log) == 0 and F == 1.0 and nr == 0
    assert st["unobservable"] == 9
    ex = oracle.apply_circuit(W.basis_state(n, 0), g)
    assert np.max(np.abs(psi - ex)) == 0
    # without the rule every one of those gates merges and checks
    _, _, _, log0 = oracle.sdrp_run(n, g, p=0.5, tau=1e-13)
    assert len(log0) > 0


def test_unobservable_qft_of_zero_state():
    """QFT of |0...0> (Sec. II.E): every controlled phase meets a qubit still
    in |0>, so the rule removes all n(n-1)/2 of them; no subsystem is ever
    composed and the result is the closed form of Eq. (dft) for x = 0."""
    n = 10
    g = W.qft_circuit(n)
    st = {}
    psi, F, nr, log = oracle.sdrp_run(n, g, p=0.0, tau=1e-13, unobservable=True, stats=st)
    assert st["unobservable"] == n * (n - 1) // 2 and len(log) == 0 and F == 1.0
    assert np.max(np.abs(psi - 2.0 ** (-n / 2))) < 1e-14


def test_unobservable_partial_and_near_eigenstate():
    """A two-control X with one control in |1> drops that control and merges
    only the target with the other control (checks run on those two alone);
    a control within tau of |0> (U3 with theta = 1e-8: P(1) = sin^2(5e-9),
    below tau = 1e-13) is projected onto |0> first: the state then has
    fidelity 1 - P(1) with the exact one, and F is unchanged."""
    n = 4
    g = [W.Gate("x", (1,)), W.Gate("h", (2,)), W.Gate("x", (0,), (), (1, 2), (1, 1))]
    psi, F, nr, log = oracle.sdrp_run(n, g, p=0.0, tau=1e-13, unobservable=True)
    assert sorted(set(int(q) for q in log["qubit"])) == [0, 2]
    assert np.max(np.abs(psi - oracle.apply_circuit(W.basis_state(n, 0), g))) == 0
    th = 1e-8
    g = [W.Gate("u3", (0,), (th, 0.0, 0.0)), W.Gate("h", (1,)), _cx(0, 1)]
    st = {}
    psi, F, nr, log = oracle.sdrp_run(2, g, p=0.0, tau=1e-13, unobservable=True, stats=st)
    ex = oracle.apply_circuit(W.basis_state(2, 0), g)
    assert st["unobservable"] == 1 and F == 1.0 and len(log) == 0
    assert abs(oracle.fidelity(psi, ex) - (1 - np.sin(th / 2) ** 2)) < 1e-15
    assert abs(psi[1]) < 1e-300 and abs(psi[3]) < 1e-300   # qubit 0 exactly |0>


def test_rho2_against_partial_trace():
    """The pair's reduced density matrix against numpy's partial trace of
    |psi><psi| (reshape and einsum), a pair in either bit order."""
    n = 7
    psi = W.gaussian_state(n, 41)
    for qa, qb in ((1, 4), (5, 0), (6, 2)):
        T = psi.reshape([2] * n)            # axis k = qubit n - 1 - k
        ax = [n - 1 - qa, n - 1 - qb]
        rest = [k for k in range(n) if k not in ax]
        M = np.transpose(T, ax[::-1] + rest).reshape(4, -1)   # row index = b_qa + 2 b_qb
        want = M @ M.conj().T
        got = oracle.rho2(psi, qa, qb)
        assert np.max(np.abs(got - want / np.trace(want).real)) < 1e-14


def test_herm4_eig_against_numpy():
    rng = np.random.default_rng(5)
    for _ in range(20):
        A = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
        H = A + A.conj().T
        w, V = oracle.herm4_eig(H)
        wn = np.linalg.eigvalsh(H)
        assert np.max(np.abs(w - wn)) < 1e-12 * np.max(np.abs(wn))
        for e in range(4):
            v = V[:, e]
            assert abs(np.vdot(v, v).real - 1) < 1e-12
            assert np.max(np.abs(H @ v - w[e] * v)) < 1e-11 * np.max(np.abs(wn))


def test_pair_projection_fidelity_and_purity():
    """Sec. III.B's per-projection fidelity for the pair: projecting onto the
    top eigenvector of rho_pair keeps fidelity lambda_max = 1 - eps with the
    input, leaves the pair pure (rho_pair of rank one) and the norm 1."""
    n = 8
    psi = W.gaussian_state(n, 43)
    w, V = oracle.herm4_eig(oracle.rho2(psi, 2, 6))
    out = oracle.sdrp_project2(psi, 2, 6, V[:, 3])
    assert abs(oracle.fidelity(out, psi) - w[3]) < 1e-13
    assert abs(oracle.norm2(out) - 1) < 1e-13
    w2, _ = oracle.herm4_eig(oracle.rho2(out, 2, 6))
    assert abs(w2[3] - 1) < 1e-12 and np.max(np.abs(w2[:3])) < 1e-12


def test_pair_check_separates_a_bell_pair():
    """Two Bell pairs (0, 1) and (2, 3), joined into one subsystem by a
    gate that entangles nothing new (CP of angle 0 on qubits 1, 2), then a
    CZ on (0, 1): each single qubit has eps = 1/2, so no one-qubit check
    acts, yet the pair (0, 1) is separable from the rest, eps_pair = 0, and
    the pair check splits it off exactly (only reachable with two-qubit
    subsystems)."""
    n = 4
    g = [W.Gate("h", (0,)), W.Gate("x", (1,), (), (0,), (1,)), W.Gate("h", (2,)), W.Gate("x", (3,), (), (2,), (1,)),
         W.Gate("cp", (1, 2), (0.0,)), W.Gate("cp", (0, 1), (np.pi,))]
    psi, F, nr, log = oracle.sdrp_run(n, g, p=0.0, tau=1e-13, pairs=True)
    pair = [e for e in log if e["pad"] > 0]
    last = [e for e in pair if int(e["gate"]) == 5]
    assert len(last) == 1
    e = last[0]
    assert e["action"] == 2 and e["eps"] < 1e-13 and (int(e["qubit"]), int(e["pad"]) - 1) == (0, 1)
    # the pair (1, 2) after gate 4 is not separable: two halves of different Bell pairs
    e4 = [e for e in pair if int(e["gate"]) == 4][0]
    assert e4["action"] == 0 and abs(e4["eps"] - 0.75) < 1e-12
    assert abs(oracle.fidelity(psi, oracle.apply_circuit(W.basis_state(n, 0), g)) - 1) < 1e-12
    # every one-qubit check kept (eps = 1/2)
    assert all(abs(e["eps"] - 0.5) < 1e-12 and e["action"] == 0 for e in log if e["pad"] == 0)


def pair_weak_circuit(delta=0.2):
    """Bell pairs (0, 1) and (2, 3), a weak controlled rotation U3(delta) from
    qubit 1 to qubit 2, then a CZ on (0, 1): every single qubit stays close to
    maximally mixed, while the pair (0, 1) is only weakly entangled with
    (2, 3)."""
    return [W.Gate("h", (0,)), W.Gate("x", (1,), (), (0,), (1,)), W.Gate("h", (2,)), W.Gate("x", (3,), (), (2,), (1,)),
            W.Gate("u3", (2,), (delta, 0.0, 0.0), (1,), (1,)), W.Gate("cp", (0, 1), (np.pi,))]


def test_pair_rounding_model():
    """Exactly one rounding, of the pair (0, 1) at the CZ: F = 1 - eps_pair
    equals the exact fidelity (Sec. III.B); eps_pair equals the smaller
    Schmidt weight of the (0, 1) | (2, 3) cut computed by numpy's SVD; pairs
    off reproduces the plain run bit for bit."""
    n = 4
    g = pair_weak_circuit()
    exact = oracle.apply_circuit(W.basis_state(n, 0), g)
    psi, F, nr, log = oracle.sdrp_run(n, g, p=0.1, tau=1e-13, pairs=True)
    rounded = [e for e in log if e["action"] == 1]
    assert len(rounded) == 1 and rounded[0]["pad"] == 2 and int(rounded[0]["qubit"]) == 0
    M = exact.reshape(4, 4).T          # rows: index bits 0-1 (pair), columns: bits 2-3
    sv = np.linalg.svd(M, compute_uv=False) ** 2
    assert abs(rounded[0]["eps"] - (1 - sv[0])) < 1e-13
    assert abs(F - (1 - rounded[0]["eps"])) < 1e-15
    assert abs(F - oracle.fidelity(psi, exact)) < 1e-12
    base = oracle.sdrp_run(n, g, p=0.1, tau=1e-13)
    off = oracle.sdrp_run(n, g, p=0.1, tau=1e-13, pairs=False)
    assert np.max(np.abs(base[0] - off[0])) == 0 and len(base[3]) == len(off[3])


def test_p_grid_count():
    """Appendix A: 8 width x depth sets x 100 circuits x 41 values of p on
    [0, 1] in steps of 0.025 = 32,800 observations."""
    grid = np.round(np.arange(0, 1.0 + 1e-9, 0.025), 3)
    assert len(grid) == 41 and 8 * 100 * len(grid) == 32800


def test_grid_couplers_counts():
    counts = [len(W.grid_couplers(5, 6, p)) for p in "ABCD"]
    assert counts == [15, 10, 12, 12]
    g = W.grid_rcs_circuit(5, 6, 10, seed=0)
    assert len(g) == 300 + 15 + 10 + 12 + 12 + 15 + 10 + 12 + 12 + 15 + 10
    # no immediate repeat of a one-qubit gate on a qubit
    last = {}
    for x in g:
        if x.name.startswith("sqrt"):
            assert last.get(x.qubits[0]) != x.name
            last[x.qubits[0]] = x.name
