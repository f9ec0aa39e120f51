"""Full-size parity of the benchmark's own sequence: the 391-gate QFT on a
27-qubit complex64 ket (1 GiB) on BF16x3 tensor-core blocks, run exactly as
bench.py runs it. The ket lives in a torch-owned device buffer wrapped by the
library; a first plan starts from the identity qubit map and leaves the ket
bit-reversed (the QFT's swaps are relabels, Table I); a second plan starts
from that map; each runs through qsim_plan_execute_norm (the FP64 norm taken
by the last block's write-back).

Checks (Sec. II.E, Eq. (dft); the complex64 bound is infidelity <= 1e-6):
- basis input |x>: every one of the 2^27 outputs of the first plan against
  the closed form y_k = 2^(-n/2) exp(2 pi i x k / 2^n); the second plan
  applies the QFT again and QFT^2 |x> = |-x mod 2^n> (the DFT applied twice
  reverses the index), checked on every output;
- Gaussian input: the whole output state against the FP64 oracle's gate-by-
  gate QFT (all-core build), then the second plan's output against the
  exact identity QFT^2 x = x[-j mod 2^n];
- probabilities of the result in logical index order: qsim_probs equals
  |amplitude|^2 of the downloaded ket up to FP64 rounding, and against the
  oracle's probabilities the total variation distance is at most
  sqrt(1 - F) (it is bounded by the trace distance of the two pure states),
  with the most likely outcome the same;
- the fused norms within 4e-6 per block applied of 1: a BF16x3 block is
  unitary only to about 2^-17 per element of U and of the amplitudes, and
  the drift accumulates over the blocks (both plans: 8 blocks of 7 qubits,
  10 of 6)."""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2304_14969_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N_QUBITS = 27


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


def bench_state(Q, n):
    """A ket in a torch-owned device buffer wrapped by the library, on its own
    stream (as bench.py sets it up)."""
    import torch
    stream = torch.cuda.Stream()
    dev = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    st = Q.State(n, Q.QSIM_C64, stream=stream.cuda_stream, dev_ptr=dev.data_ptr())
    return st, dev, stream


def closed_form(x, n):
    N = 1 << n
    ks = np.arange(N, dtype=np.int64)
    return np.exp(2j * np.pi * ((x * ks) % N).astype(np.float64) / N) / np.sqrt(N)


# block sizes of the benchmark's tensor-core plans: 6-qubit blocks (five
# passes of k_tc_pipe) and 7-qubit blocks (four passes of k_tc_pipe7)
BLOCKS = {0: 5, 7: 4}
NORM_PER_BLOCK = 4e-6


@pytest.mark.parametrize("max_block", sorted(BLOCKS))
def test_qft27_bench_sequence_basis_closed_form(Q, max_block):
    n = N_QUBITS
    N = 1 << n
    x = W.basis_index(n, 27)
    st, dev, _ = bench_state(Q, n)
    Q.qsim_set_basis(st.h, x)
    circ = Q.Circuit(n, W.qft_circuit(n))
    p0 = Q.Plan(circ, dtype=Q.QSIM_C64, prec=Q.QSIM_PREC_BF16X3, state=st, max_block=max_block)
    assert p0.info()["passes"] == BLOCKS[max_block]
    nf = p0.execute_norm(st)
    assert abs(nf - 1.0) <= NORM_PER_BLOCK * BLOCKS[max_block]
    y = st.download()
    ref = closed_form(x, n)
    assert infid(y, ref) <= 1e-6
    assert np.max(np.abs(y - ref)) <= 1e-3 / np.sqrt(N)
    del ref
    # the second plan of the bench, from the bit-reversed map the first left
    p1 = Q.Plan(circ, dtype=Q.QSIM_C64, prec=Q.QSIM_PREC_BF16X3, state=st, max_block=max_block)
    nf = p1.execute_norm(st)
    assert abs(nf - 1.0) <= NORM_PER_BLOCK * 2 * BLOCKS[max_block]
    assert list(st.qubit_map()) == list(range(n))
    y = st.download()
    j = (N - x) % N
    assert abs(abs(y[j]) - 1.0) <= 1e-5
    y[j] = 0
    assert np.max(np.abs(y)) <= 1e-5
    st.close()
    del dev


_REF = {}


def oracle_qft27(x, g):
    """The oracle's QFT of the Gaussian input and its probabilities (all-core
    build), computed once for both block sizes."""
    if "ref" not in _REF:
        oracle.use_all_cores(True)
        try:
            _REF["ref"] = oracle.apply_circuit(x, g)
            _REF["pref"] = oracle.probs(_REF["ref"])
        finally:
            oracle.use_all_cores(False)
    return _REF["ref"], _REF["pref"]


@pytest.mark.parametrize("max_block", sorted(BLOCKS))
def test_qft27_bench_sequence_gaussian_vs_oracle(Q, max_block):
    import torch
    n = N_QUBITS
    N = 1 << n
    g = W.qft_circuit(n)
    x = W.gaussian_state(n, 0)
    st, dev, _ = bench_state(Q, n)
    host_in = torch.from_numpy(x.astype(np.complex64)).pin_memory()
    Q.qsim_upload(st.h, C.c_void_p(host_in.data_ptr()))
    circ = Q.Circuit(n, g)
    p0 = Q.Plan(circ, dtype=Q.QSIM_C64, prec=Q.QSIM_PREC_BF16X3, state=st, max_block=max_block)
    assert p0.info()["passes"] == BLOCKS[max_block]
    nf = p0.execute_norm(st)
    assert abs(nf - 1.0) <= NORM_PER_BLOCK * BLOCKS[max_block]
    y = st.download()
    probs = st.probs()
    ref, pref = oracle_qft27(x, g)
    f = infid(y, ref)
    assert f <= 1e-6, f
    # probabilities in logical index order: the library's FP64 squares of its
    # own amplitudes (to FP64 rounding), then against the oracle's
    y64 = y.astype(np.complex128)
    mine = y64.real ** 2 + y64.imag ** 2
    assert np.max(np.abs(probs - mine) / np.maximum(mine, 1e-300)) <= 4 * np.finfo(np.float64).eps
    tvd = 0.5 * np.sum(np.abs(probs - pref))
    assert tvd <= np.sqrt(f) + 1e-9, (tvd, f)
    top = np.argsort(pref)[-2:]
    if pref[top[1]] - pref[top[0]] > 2 * np.max(np.abs(probs - pref)):
        assert int(np.argmax(probs)) == int(top[1])
    del ref, pref, probs, mine, y64
    # second plan: QFT^2 x = x[-j mod N] exactly
    p1 = Q.Plan(circ, dtype=Q.QSIM_C64, prec=Q.QSIM_PREC_BF16X3, state=st, max_block=max_block)
    nf = p1.execute_norm(st)
    assert abs(nf - 1.0) <= NORM_PER_BLOCK * 2 * BLOCKS[max_block]
    y2 = st.download()
    idx = (-np.arange(N, dtype=np.int64)) % N
    assert infid(y2, x[idx]) <= 2e-6
    st.close()
    del dev
