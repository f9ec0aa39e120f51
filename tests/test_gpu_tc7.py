"""7-qubit tensor-core blocks (the Table I fused block at k = 7 on complex64
kets with the BF16x3 split, n >= 14) against the FP64 oracle.

The kernel keeps Re U and Im U of the 128 x 128 block (hi and lo BF16 parts)
in shared memory and forms the real and imaginary outputs from the signed
parts of the amplitudes (one product negated through the instruction
descriptor), so a sign or part mix-up shows as a large error here. Cases
cover a block on the lowest qubits (vector stores, rotated shared-memory
reads), on the highest (groups on the low qubits), scattered blocks whose
tiles take two to four boxes per eighth, one tile per CTA and several.
Tolerance as for the 6-qubit blocks: infidelity <= 1e-6, every amplitude
within 2e-5 of the largest."""
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


def apply7(Q, n, qs, U, x):
    st = Q.State(n, Q.QSIM_C64)
    st.upload(x)
    qa = (C.c_int * 7)(*qs)
    u = np.ascontiguousarray(np.asarray(U, dtype=np.complex128).ravel().view(np.float64))
    Q.qsim_apply_fused(st.h, 7, qa, u.ctypes.data_as(C.c_void_p), Q.QSIM_PREC_BF16X3)
    y = st.download()
    st.close()
    return y


CASES = [(14, [0, 1, 2, 3, 4, 5, 6]), (14, [7, 8, 9, 10, 11, 12, 13]), (15, [13, 2, 9, 0, 5, 14, 7]),
         (16, [0, 1, 5, 9, 12, 14, 15]), (18, [1, 3, 5, 7, 9, 11, 13]), (20, [19, 18, 17, 16, 2, 10, 0]),
         (21, [20, 14, 9, 7, 3, 11, 1]), (22, [7, 9, 11, 13, 15, 17, 19]), (24, [3, 8, 12, 17, 20, 22, 23])]


@pytest.mark.parametrize("n,qs", CASES)
def test_tc7_block_vs_oracle(Q, n, qs):
    x = W.gaussian_state(n, 3 * n)
    U = W.random_unitary(7, 5 + n)
    ref = oracle.apply_kq(x, qs, U)
    y = apply7(Q, n, qs, U, x)
    assert infid(y, ref) <= 1e-6
    assert np.max(np.abs(y - ref)) <= 2e-5 * np.max(np.abs(ref)) + 1e-7


def test_tc7_block_of_one_real_and_one_imaginary_matrix(Q):
    """U = i V with V real (Re U = 0) and U = V: the two halves of the
    complex product, each on its own, against the oracle."""
    n, qs = 16, [2, 4, 6, 8, 10, 12, 14]
    x = W.gaussian_state(n, 1)
    V = np.linalg.qr(np.random.default_rng(4).standard_normal((128, 128)))[0]
    for U in (V.astype(np.complex128), 1j * V):
        ref = oracle.apply_kq(x, qs, U)
        y = apply7(Q, n, qs, U, x)
        assert infid(y, ref) <= 1e-6
        assert np.max(np.abs(y - ref)) <= 2e-5 * np.max(np.abs(ref)) + 1e-7


@pytest.mark.parametrize("n", [10, 13])
def test_tc7_rejects_small_kets(Q, n):
    st = Q.State(n, Q.QSIM_C64)
    qa = (C.c_int * 7)(*range(7))
    u = np.ascontiguousarray(np.eye(128, dtype=np.complex128).ravel().view(np.float64))
    with pytest.raises(Q.QsimError) as e:
        Q.qsim_apply_fused(st.h, 7, qa, u.ctypes.data_as(C.c_void_p), Q.QSIM_PREC_BF16X3)
    assert e.value.status == 6
    st.close()


PLANS = {
    "grid20": lambda: (20, W.grid_rcs_circuit(4, 5, 8, seed=2), W.basis_state(20, 0)),
    "paper20": lambda: (20, W.paper_random_circuit(4, 5, 7, seed=3), W.gaussian_state(20, 4)),
    "random14": lambda: (14, W.random_1q_circuit(14, 200, 5), W.gaussian_state(14, 5)),
    "qft16": lambda: (16, W.qft_circuit(16), W.gaussian_state(16, 6)),
    "qft21": lambda: (21, W.qft_circuit(21), W.gaussian_state(21, 7)),
}


@pytest.mark.parametrize("name", sorted(PLANS))
def test_tc7_plan_vs_oracle(Q, name):
    """Whole circuits fused into <= 7-qubit blocks (max_block = 7), deferred
    controlled phases included: infidelity <= 1e-6 against the oracle. The
    fused norm of the last block equals the FP64 norm of the ket it wrote (to
    its FP32 runs' rounding), and stays within 1e-4 of the input's: the
    BF16x3 blocks are unitary to about 2^-17 each, and the random circuit
    takes 22 of them."""
    n, g, x = PLANS[name]()
    ref = oracle.apply_circuit(x, g)
    st = Q.State(n, Q.QSIM_C64)
    st.upload(x)
    p = Q.Plan(Q.Circuit(n, g), dtype=Q.QSIM_C64, prec=Q.QSIM_PREC_BF16X3, state=st, max_block=7)
    p6 = Q.Plan(Q.Circuit(n, g), dtype=Q.QSIM_C64, prec=Q.QSIM_PREC_BF16X3, state=st)
    assert p.info()["passes"] <= p6.info()["passes"]
    nf = p.execute_norm(st)
    y = st.download()
    st.close()
    assert infid(y, ref) <= 1e-6
    y64 = y.astype(np.complex128)
    assert abs(nf - np.vdot(y64, y64).real) <= 1e-6
    assert abs(nf - np.vdot(x, x).real) <= 1e-4 * np.vdot(x, x).real


@pytest.mark.parametrize("dt,prec", [(0, 1), (1, 3), (1, 2)])
def test_tc7_rejects_other_pairings(Q, dt, prec):
    """7-qubit tensor-core blocks exist for complex64 kets with BF16x3 only:
    3xTF32 on complex64 and every complex128 precision are refused on the
    host, before any launch."""
    st = Q.State(16, dt)
    qa = (C.c_int * 7)(*range(7))
    u = np.ascontiguousarray(np.eye(128, dtype=np.complex128).ravel().view(np.float64))
    with pytest.raises(Q.QsimError) as e:
        Q.qsim_apply_fused(st.h, 7, qa, u.ctypes.data_as(C.c_void_p), prec)
    assert e.value.status == 6
    st.close()
