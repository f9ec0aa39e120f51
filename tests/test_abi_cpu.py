"""CPU checks of the C-ABI library: it builds, loads, exports every entry
point declared in include/qsim.h, rejects bad arguments on the host, and
its planner produces the expected pass structure (the planner is host
code; plans reach the device only at their first execution)."""
import ctypes as C
import os
import re
import shutil

import numpy as np
import pytest

from paper_2304_14969_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qsim.h")

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists(
    os.path.join(ROOT, "paper_2304_14969_gb300", "libqsim.so")), reason="needs nvcc or a built libqsim.so")


@pytest.fixture(scope="module")
def Q():
    from paper_2304_14969_gb300 import build, qsim
    build.build()
    qsim.lib()
    return qsim


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qsim_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(Q):
    names = declared_functions()
    assert len(names) >= 40
    L = Q.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(Q.EXPORTED)
    assert "sm_103a" in Q.qsim_version()


def test_struct_sizes_match_header(Q):
    assert C.sizeof(Q.qsim_gate) == 80
    assert C.sizeof(Q.qsim_run_opts) == 48


def test_host_validation_before_any_launch(Q):
    h = C.c_void_p()
    with pytest.raises(Q.QsimError) as e:
        Q.qsim_create(0, Q.QSIM_C64, None, C.byref(h))
    assert e.value.status == 1
    with pytest.raises(Q.QsimError):
        Q.qsim_create(40, Q.QSIM_C64, None, C.byref(h))
    with pytest.raises(Q.QsimError):
        Q.qsim_create(4, 7, None, C.byref(h))
    with pytest.raises(Q.QsimError):
        Q.qsim_wrap(4, Q.QSIM_C64, C.c_void_p(8), None, C.byref(h))   # misaligned


def test_circuit_validation(Q):
    bad = [
        [W.Gate("h", (5,))],                              # qubit out of range
        [W.Gate("cp", (1, 1), (0.3,))],                   # duplicate
        [W.Gate("x", (0,), (), (0,), (1,))],              # control == target
        [W.Gate("x", (0,), (), (1, 1), (1, 1))],          # duplicate control
    ]
    for gates in bad:
        c = Q.Circuit(3, gates)
        h = C.c_void_p()
        with pytest.raises(Q.QsimError) as e:
            Q.qsim_plan_create(c.ptr(), Q.QSIM_C64, None, C.byref(h))
        assert e.value.status == 1


def plan_info(Q, n, gates, dt=0, tile=0):
    c = Q.Circuit(n, gates)
    p = Q.Plan(c, dtype=dt, tile=tile)
    return p.info()


def test_qft27_plans_three_passes(Q):
    """QFT: every controlled phase is deferred to the next H on its control,
    swaps are relabels, so 27 qubits need ceil((27-13)/8) + 1 = 3 passes."""
    info = plan_info(Q, 27, W.qft_circuit(27))
    assert info["passes"] == 3
    assert info["dense"] == 27
    assert info["swaps_relabelled"] == 13
    assert info["per_gate_steps"] == 0
    for n, want in [(16, 2), (20, 2), (21, 2), (30, 4), (33, 4)]:
        assert plan_info(Q, n, W.qft_circuit(n))["passes"] == want, n


def test_grid_plan_covers_all_gates(Q):
    g = W.grid_rcs_circuit(5, 6, 10, seed=0)
    info = plan_info(Q, 30, g)
    assert info["dense"] == len(g)
    assert info["per_gate_steps"] == 0
    assert 1 <= info["passes"] <= 40


def test_multi_controlled_gate_becomes_per_gate_step(Q):
    g = [W.Gate("h", (q,)) for q in range(10)] + [W.Gate("x", (2,), (), (0, 1), (1, 1))]
    g += [W.Gate("rz", (3,), (0.3,))]
    info = plan_info(Q, 10, g)
    assert info["per_gate_steps"] >= 2


def test_library_has_no_unresolved_internal_symbols(Q):
    """Every internal (qs::) function the library calls is defined in it."""
    import subprocess
    lib = os.path.join(ROOT, "paper_2304_14969_gb300", "libqsim.so")
    out = subprocess.run(["nm", "-D", "--undefined-only", lib], capture_output=True, text=True).stdout
    assert "_ZN2qs" not in out, [l for l in out.splitlines() if "_ZN2qs" in l]
