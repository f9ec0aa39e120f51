"""Batched persistent runner and autotuner against the oracle: a mixed
batch of QFT and grid circuits of uneven size and depth runs in one launch
(captured in a CUDA graph); every circuit's final ket matches the oracle
within the complex64 tolerance."""
import ctypes as C
import os
import tempfile

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


def make_batch(Q, specs, use_graph=1, cache=None, tile=0, path=0):
    circs = [Q.Circuit(s["n"], s["gates"]) for s in specs]
    arr = (C.POINTER(Q.qsim_circuit) * len(circs))(*[C.pointer(c.c) for c in circs])
    o = Q.qsim_batch_opts(use_graph=use_graph, tile_qubits=tile, path=path,
                          tune_cache=cache.encode() if cache else None)
    h = C.c_void_p()
    Q.qsim_batch_create(C.cast(arr, C.c_void_p), len(circs), C.byref(o), C.byref(h))
    return h, circs


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("use_graph", [0, 1])
def test_batch_matches_oracle(Q, use_graph, path):
    """path 1: every circuit as fused SIMT passes in the persistent launch;
    path 2: circuits with n >= 13 as tensor-core blocks (grouped launches per
    block round, concurrent with the SIMT launch for the smaller ones)."""
    specs = W.batch_circuits(12, seed=3, nmin=10, nmax=17, dmin=2, dmax=8)
    h, circs = make_batch(Q, specs, use_graph, path=path)
    info = np.zeros(8, dtype=np.int64)
    Q.qsim_batch_info(h, info.ctypes.data_as(C.c_void_p))
    ntc = sum(s["n"] >= 13 for s in specs)
    assert info[0] == 12 and info[7] == (ntc if path == 2 else 0)
    assert 0 < ntc < 12
    # Gaussian inputs for even circuits, |0...0> for odd ones
    inputs = []
    Q.qsim_batch_reset(h)
    for i, s in enumerate(specs):
        x = W.gaussian_state(s["n"], 100 + i) if i % 2 == 0 else W.basis_state(s["n"], 0)
        inputs.append(x)
        if i % 2 == 0:
            xs = np.ascontiguousarray(x.astype(np.complex64))
            Q.qsim_batch_upload(h, i, xs.ctypes.data_as(C.c_void_p))
    secs = C.c_double()
    lat = np.zeros(12)
    Q.qsim_batch_run(h, C.byref(secs), lat.ctypes.data_as(C.c_void_p))
    assert secs.value > 0 and np.all(lat >= 0)
    for i, s in enumerate(specs):
        out = np.zeros(1 << s["n"], dtype=np.complex64)
        Q.qsim_batch_download(h, i, out.ctypes.data_as(C.c_void_p))
        ref = oracle.apply_circuit(inputs[i], s["gates"])
        assert infid(out, ref) <= 1e-6, (i, s["kind"], s["n"])
    # a second run needs a reset or upload first
    with pytest.raises(Q.QsimError):
        Q.qsim_batch_run(h, None, None)
    Q.qsim_batch_reset(h)
    Q.qsim_batch_run(h, None, None)
    Q.qsim_batch_destroy(h)


def test_autotune_and_cache(Q):
    g = W.qft_circuit(16)
    c = Q.Circuit(16, g)
    best = Q.qsim_run_opts()
    secs = C.c_double()
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.jsonl")
        Q.qsim_autotune(c.ptr(), 0, path.encode(), C.byref(best), C.byref(secs))
        assert secs.value > 0
        # the fastest candidate: a SIMT tile width, or the tensor-core plan
        assert (10 <= best.tile_qubits <= 14 and best.prec == 0) or (best.tile_qubits == 0 and best.prec == 2)
        lines = open(path).read().strip().splitlines()
        assert len(lines) >= 5 and sum('"path": "tc"' in x for x in lines) == 1
        specs = [{"n": 16, "gates": g, "kind": "qft"}]
        h, circs = make_batch(Q, specs, cache=path)
        Q.qsim_batch_run(h, None, None)
        out = np.zeros(1 << 16, dtype=np.complex64)
        Q.qsim_batch_download(h, 0, out.ctypes.data_as(C.c_void_p))
        assert np.allclose(out, 2 ** -8, atol=1e-6)
        Q.qsim_batch_destroy(h)
