"""Batched persistent runner and autotuner against the oracle: a mixed
batch of QFT and grid circuits of uneven size and depth runs in one launch
(captured in a CUDA graph); every circuit's final ket matches the oracle
within the complex64 tolerance. The batch configuration's own distribution
(n ~ U{10..24}, depth ~ U{4..20}, QFT / grid 50/50) runs at 64 circuits on
the autotuned path mix and on tensor-core blocks for every n >= 13."""
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


_REFS = {}


def _reference(spec, x_seed):
    """Oracle result of one batch circuit on its Gaussian input (all-core
    build; identical circuits on identical inputs are computed once)."""
    key = (spec["kind"], spec["n"], spec["depth"] if spec["kind"] == "grid" else 0,
           spec["seed"] if spec["kind"] == "grid" else 0, x_seed)
    if key not in _REFS:
        x = W.gaussian_state(spec["n"], x_seed)
        oracle.use_all_cores(True)
        try:
            _REFS[key] = (x, oracle.apply_circuit(x, spec["gates"]))
        finally:
            oracle.use_all_cores(False)
    return _REFS[key]


@pytest.mark.parametrize("path", [0, 2])
def test_batch_config_distribution(Q, path):
    """64 circuits drawn from the batch configuration's distribution, one
    launch from a CUDA graph. path 0: per qubit count the autotuner's choice
    (tensor-core plan or SIMT tile width), from a tune cache written here by
    qsim_autotune on one grid circuit of each of four qubit counts (the other
    counts take the default SIMT plan); path 2: tensor-core blocks for every
    n >= 13. Every ket against the oracle, infidelity <= 1e-6. A QFT input is
    seeded by its size, so equal circuits on equal inputs share one oracle
    run."""
    specs = W.batch_circuits(64, seed=7)
    cache = None
    with tempfile.TemporaryDirectory() as d:
        if path == 0:
            cache = os.path.join(d, "tune.jsonl")
            done = set()
            for sp in specs:
                if sp["kind"] != "grid" or sp["n"] in done or sp["n"] not in (12, 16, 20, 24):
                    continue
                best = Q.qsim_run_opts()
                sec = C.c_double()
                Q.qsim_autotune(Q.Circuit(sp["n"], sp["gates"]).ptr(), 0, cache.encode(), C.byref(best),
                                C.byref(sec))
                done.add(sp["n"])
            assert len(done) >= 3
        h, circs = make_batch(Q, specs, 1, cache=cache, path=path)
    info = np.zeros(8, dtype=np.int64)
    Q.qsim_batch_info(h, info.ctypes.data_as(C.c_void_p))
    assert info[0] == 64
    ntc = sum(s["n"] >= 13 for s in specs)
    if path == 2:
        assert info[7] == ntc
    Q.qsim_batch_reset(h)
    seeds = []
    for i, s in enumerate(specs):
        xs = s["n"] if s["kind"] == "qft" else 1000 + i
        seeds.append(xs)
        x, _ = _reference(s, xs)
        xc = np.ascontiguousarray(x.astype(np.complex64))
        Q.qsim_batch_upload(h, i, xc.ctypes.data_as(C.c_void_p))
    secs = C.c_double()
    lat = np.zeros(64)
    Q.qsim_batch_run(h, C.byref(secs), lat.ctypes.data_as(C.c_void_p))
    assert secs.value > 0 and np.all(lat >= 0)
    worst = 0.0
    for i, s in enumerate(specs):
        out = np.zeros(1 << s["n"], dtype=np.complex64)
        Q.qsim_batch_download(h, i, out.ctypes.data_as(C.c_void_p))
        _, ref = _reference(s, seeds[i])
        f = infid(out, ref)
        worst = max(worst, f)
        assert f <= 1e-6, (i, s["kind"], s["n"], s["depth"], f)
    Q.qsim_batch_destroy(h)
