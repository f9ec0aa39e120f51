"""Tensor-core dense blocks (tcgen05, 3xTF32 and BF16x3 splits with FP32
accumulation on complex64 kets, BF16X6 on complex128 kets) against the FP64
oracle's k-qubit block application. Tolerance: state infidelity <= 1e-6
(complex64), <= 1e-12 (complex128)."""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2304_14969_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    from paper_2304_14969_gb300 import build, qsim
    build.build()
    qsim.lib()
    return qsim


def infid(a, b):
    a = a.astype(np.complex128)
    b = b.astype(np.complex128)
    return 1 - abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real)


def apply(Q, n, qs, U, prec, x, dtype=0):
    st = Q.State(n, dtype)
    st.upload(x)
    k = len(qs)
    qa = (C.c_int * k)(*qs)
    u = np.ascontiguousarray(np.asarray(U, dtype=np.complex128).ravel().view(np.float64))
    Q.qsim_apply_fused(st.h, k, qa, u.ctypes.data_as(C.c_void_p), prec)
    y = st.download()
    st.close()
    return y


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("n,qs", [(6, [0, 1, 2, 3, 4, 5]), (8, [2, 7, 0, 5, 3, 6]), (12, [11, 3, 8, 5, 9, 1]),
                                  (16, [4, 15, 9]), (18, [0]), (20, [19, 18, 17, 16, 2, 10]),
                                  # n >= 13 (BF16x3: TMA-fed pipelined kernel): low block, two to four
                                  # boxes per tile, block on the top qubits
                                  (13, [0, 1, 2, 3, 4, 5]), (14, [8, 10, 12, 3, 1, 13]),
                                  (22, [7, 9, 11, 13, 15, 17]), (21, [20, 14, 9, 7, 3, 11]),
                                  (19, [18, 17, 16, 15, 14, 13])])
def test_tc_block_vs_oracle(Q, prec, n, qs):
    x = W.gaussian_state(n, n)
    U = W.random_unitary(len(qs), 7 + n)
    ref = oracle.apply_kq(x, qs, U)
    y = apply(Q, n, qs, U, prec, x)
    assert infid(y, ref) <= 1e-6
    assert np.max(np.abs(y - ref)) <= 2e-5 * np.max(np.abs(ref)) + 1e-7


@pytest.mark.parametrize("n,dt,prec", [(10, 1, 2), (14, 1, 2), (14, 1, 1), (12, 1, 3), (14, 0, 3)])
def test_tc_block_rejects_unsupported_pairings(Q, n, dt, prec):
    """complex128 kets take only BF16X6 (n >= 13); complex64 kets not BF16X6."""
    st = Q.State(n, dt)
    qa = (C.c_int * 2)(0, 1)
    u = np.ascontiguousarray(np.eye(4, dtype=np.complex128).ravel().view(np.float64))
    with pytest.raises(Q.QsimError) as e:
        Q.qsim_apply_fused(st.h, 2, qa, u.ctypes.data_as(C.c_void_p), prec)
    assert e.value.status == 6
    st.close()


# complex128 blocks (BF16X6): low blocks (rotated reads), blocks whose
# quarter-tile bits are group bits, block bits or one of each, padded blocks,
# two to four boxes per quarter tile
C128_CASES = [(13, [0, 1, 2, 3, 4, 5]), (14, [0, 1, 2, 3, 4, 12]), (14, [8, 10, 12, 3, 1, 13]),
              (22, [7, 9, 11, 13, 15, 17]), (21, [20, 14, 9, 7, 3, 11]), (19, [18, 17, 16, 15, 14, 13]),
              (16, [4, 15, 9]), (18, [0]), (17, [2, 0, 1]), (20, [5, 6, 7, 8, 9, 10])]


@pytest.mark.parametrize("n,qs", C128_CASES)
def test_tc_bf16x6_block_vs_oracle(Q, n, qs):
    """One complex128 block on the tensor cores (three BF16 slices per
    operand, six products, FP32 accumulation) against the FP64 oracle:
    infidelity <= 1e-12, every amplitude within 1e-6 of the largest."""
    x = W.gaussian_state(n, n + 1)
    U = W.random_unitary(len(qs), 11 + n)
    ref = oracle.apply_kq(x, qs, U)
    y = apply(Q, n, qs, U, 3, x, dtype=1)
    assert y.dtype == np.complex128
    assert infid(y, ref) <= 1e-12
    assert np.max(np.abs(y - ref)) <= 1e-6 * np.max(np.abs(ref))


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("which", ["grid", "random", "qft"])
def test_tc_plan_vs_oracle(Q, prec, which):
    """Whole circuits fused into <= 6-qubit blocks on the tensor cores."""
    if which == "grid":
        n, g, x = 20, W.grid_rcs_circuit(4, 5, 8, seed=2), W.basis_state(20, 0)
    elif which == "random":
        n = 14
        g, x = W.random_1q_circuit(n, 200, 5), W.gaussian_state(n, 5)
    else:
        n = 16
        g, x = W.qft_circuit(n), W.gaussian_state(n, 6)
    ref = oracle.apply_circuit(x, g)
    st = Q.State(n, 0)
    st.upload(x)
    st.run(Q.Circuit(n, g), mode=1, prec=prec, relabel=1)
    y = st.download()
    st.close()
    assert infid(y, ref) <= 1e-6


@pytest.mark.parametrize("which", ["grid", "random", "qft"])
def test_tc_bf16x6_plan_vs_oracle(Q, which):
    """Whole circuits on complex128 kets fused into BF16X6 tensor-core blocks
    (deferred controlled phases applied in FP32 by the converters):
    infidelity against the FP64 oracle <= 1e-12."""
    if which == "grid":
        n, g, x = 20, W.grid_rcs_circuit(4, 5, 8, seed=2), W.gaussian_state(20, 2)
    elif which == "random":
        n = 14
        g, x = W.random_1q_circuit(n, 200, 5), W.gaussian_state(n, 5)
    else:
        n = 16
        g, x = W.qft_circuit(n), W.gaussian_state(n, 6)
    ref = oracle.apply_circuit(x, g)
    st = Q.State(n, 1)
    st.upload(x)
    st.run(Q.Circuit(n, g), mode=1, prec=3, relabel=1)
    y = st.download()
    st.close()
    assert infid(y, ref) <= 1e-12


def test_tc_bf16x6_qft27_basis_closed_form(Q):
    """27-qubit QFT on a complex128 ket (2 GiB) through BF16X6 tensor-core
    blocks, from a basis state |x>: every output against the closed form
    y_k = 2^(-n/2) exp(2 pi i x k / 2^n) of Eq. (dft), infidelity <= 1e-12;
    and the fused norm of the last block's write-back."""
    n = 27
    N = 1 << n
    x = 0x5A3C1F7 % N
    st = Q.State(n, 1)
    Q.qsim_set_basis(st.h, x)
    plan = Q.Plan(Q.Circuit(n, W.qft_circuit(n)), dtype=1, prec=3, state=st)
    nf = plan.execute_norm(st)
    assert abs(nf - 1.0) <= 1e-6
    y = st.download()
    st.close()
    ks = np.arange(N, dtype=np.int64)
    ref = np.exp(2j * np.pi * ((x * ks) % N).astype(np.float64) / N) / np.sqrt(N)
    assert infid(y, ref) <= 1e-12
    assert np.max(np.abs(y - ref)) <= 1e-6 / np.sqrt(N)


@pytest.mark.parametrize("prec", [1, 2])
def test_tc_qft27_full_size_sampled(Q, prec):
    """27-qubit QFT on tensor-core blocks (controlled phases deferred into
    per-group pre-diagonals): sampled outputs against Eq. (dft) evaluated
    one by one; relative squared error <= 1e-6."""
    n = 27
    x = W.gaussian_state(n, 0)
    st = Q.State(n, 0)
    st.upload(x)
    st.run(Q.Circuit(n, W.qft_circuit(n)), mode=1, prec=prec, relabel=1)
    y = st.download()
    st.close()
    num = den = 0.0
    for j in [0, 3, 77777, (1 << n) - 5]:
        r = oracle.dft_sample(x, j)
        num += abs(y[j] - r) ** 2
        den += abs(r) ** 2
    assert num / den <= 1e-6


@pytest.mark.parametrize("max_block", [0, 7])
def test_tc_qft30_basis_closed_form(Q, max_block):
    """30-qubit QFT (8 GiB complex64 ket) on tensor-core blocks, BF16x3, 6- and
    7-qubit blocks, from a basis state |x>: Eq. (dft) gives every output in
    closed form, y_k = 2^(-n/2) exp(2 pi i x k / 2^n). Checked on the whole
    state (infidelity <= 1e-6, the closed form computed chunk by chunk), on
    4096 sampled outputs (relative squared error <= 1e-6) and on the FP64
    norm."""
    n = 30
    N = 1 << n
    x = 0x2A5F3B1D % N
    st = Q.State(n, 0)
    Q.qsim_set_basis(st.h, x)
    st.run(Q.Circuit(n, W.qft_circuit(n)), mode=1, prec=2, relabel=1, max_block=max_block)
    assert abs(st.norm() - 1.0) < 1e-5
    y = st.download()
    st.close()
    rng = np.random.default_rng(30)
    ks = np.concatenate([[0, 1, N - 1], rng.integers(0, N, 4093)])
    ref = np.exp(2j * np.pi * ((x * ks) % N).astype(np.float64) / N) / np.sqrt(N)
    got = y[ks].astype(np.complex128)
    assert np.sum(np.abs(got - ref) ** 2) / np.sum(np.abs(ref) ** 2) <= 1e-6
    ip, ny = 0j, 0.0
    for a in range(0, N, 1 << 24):
        k = np.arange(a, a + (1 << 24), dtype=np.int64)
        rr = np.exp(2j * np.pi * ((x * k) % N).astype(np.float64) / N) / np.sqrt(N)
        yy = y[a:a + (1 << 24)].astype(np.complex128)
        ip += np.vdot(yy, rr)
        ny += float(np.vdot(yy, yy).real)
    assert 1.0 - abs(ip) ** 2 / ny <= 1e-6


@pytest.mark.parametrize("which", ["qft16", "grid20", "simt_qft16"])
def test_plan_execute_norm(Q, which):
    """qsim_plan_execute_norm: the norm taken by the last tensor-core block's
    write-back equals a separate FP64 norm of the result (same ket, FP32 runs
    summed in FP64, different order); plans that do not end with a
    tensor-core block fall back to the separate reduction."""
    if which.endswith("qft16"):
        n, g = 16, W.qft_circuit(16)
    else:
        n, g = 20, W.grid_rcs_circuit(4, 5, 8, seed=4)
    x = W.gaussian_state(n, 9)
    st = Q.State(n, 0)
    st.upload(x)
    plan = Q.Plan(Q.Circuit(n, g), dtype=0, state=st, **({} if which.startswith("simt") else {"prec": 2}))
    nf = plan.execute_norm(st)
    ns = st.norm()
    assert abs(nf - ns) <= 1e-6 * ns
    assert abs(nf - 1.0) <= 1e-5
    ref = oracle.apply_circuit(x, g)
    assert infid(st.download(), ref) <= 1e-6
    st.close()
