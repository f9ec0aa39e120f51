"""Thin ctypes binding of libqsim.so (include/qsim.h), same names as the C ABI.

Only argument marshalling happens here: every step of the simulation runs
in the library's CUDA kernels. Loading fails loudly when libqsim.so is
missing or cannot be loaded; there is no fallback.

Besides the raw ``qsim_*`` functions (which return a status and raise
``QsimError`` on any status other than QSIM_OK), the module offers
``Circuit`` (packs a list of ``workloads.Gate`` into qsim_gate records) and
small helpers that return numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqsim.so")

QSIM_C64, QSIM_C128 = 0, 1
QSIM_PREC_NATIVE, QSIM_PREC_3XTF32, QSIM_PREC_BF16X3, QSIM_PREC_BF16X6 = 0, 1, 2, 3
QSIM_MODE_PER_GATE, QSIM_MODE_FUSED = 0, 1
QSIM_SCHED_EXHAUSTIVE, QSIM_SCHED_MLP, QSIM_SCHED_FORCED = 0, 1, 2
STATUS = {0: "QSIM_OK", 1: "QSIM_E_INVAL", 2: "QSIM_E_NOMEM", 3: "QSIM_E_CUDA", 4: "QSIM_E_TIMEOUT",
          5: "QSIM_E_BUDGET", 6: "QSIM_E_UNSUPPORTED"}
KIND = {"h": 0, "x": 1, "y": 2, "z": 3, "s": 4, "t": 5, "sqrtx": 6, "sqrty": 7, "sqrtw": 8,
        "u3": 9, "phase": 10, "rz": 11, "mat1": 12, "cp": 16, "swap": 17, "fsim": 18, "mat2": 19}
MAX_CONTROLS = 4


class QsimError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class qsim_gate(C.Structure):
    _fields_ = [("kind", C.c_int32), ("q0", C.c_int32), ("q1", C.c_int32), ("ncontrols", C.c_int32),
                ("controls", C.c_int32 * MAX_CONTROLS), ("control_values", C.c_uint32),
                ("reserved", C.c_int32), ("params", C.c_double * 4), ("matrix_offset", C.c_int64)]


class qsim_circuit(C.Structure):
    _fields_ = [("n", C.c_int32), ("ngates", C.c_int32), ("gates", C.POINTER(qsim_gate)),
                ("matrices", C.POINTER(C.c_double)), ("nmatrix_doubles", C.c_int64)]


class qsim_run_opts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("prec", C.c_int32), ("tile_qubits", C.c_int32),
                ("low_qubits", C.c_int32), ("max_block", C.c_int32), ("relabel_swaps", C.c_int32),
                ("reserved", C.c_int32 * 6)]


class qsim_decision(C.Structure):
    _fields_ = [("gate", C.c_int32), ("qubit", C.c_int32), ("action", C.c_int32), ("reserved", C.c_int32),
                ("eps", C.c_double), ("r", C.c_double * 3)]


class qsim_approx_opts(C.Structure):
    _fields_ = [("budget_bytes", C.c_double), ("tau", C.c_double), ("dtype", C.c_int32),
                ("schedule", C.c_int32), ("top_m", C.c_int32), ("fallback_every", C.c_int32),
                ("exhaustive_from", C.c_int32), ("mlp", C.c_void_p), ("force", C.POINTER(C.c_int32)), ("nforce", C.c_int32),
                ("log_cap", C.c_int32), ("log", C.POINTER(qsim_decision)), ("state_out", C.c_void_p),
                ("trace_features", C.POINTER(C.c_float)), ("trace_labels", C.POINTER(C.c_int32)),
                ("trace_cap", C.c_int64), ("stream", C.c_void_p), ("unobservable", C.c_int32),
                ("pairs", C.c_int32)]


class qsim_approx_result(C.Structure):
    _fields_ = [("fidelity_model", C.c_double), ("seconds", C.c_double), ("n_rounds", C.c_int64),
                ("n_exact", C.c_int64), ("n_checks", C.c_int64), ("n_bloch_passes", C.c_int64),
                ("peak_bytes", C.c_int64), ("n_log", C.c_int64), ("n_trace", C.c_int64),
                ("max_subsystem_qubits", C.c_int32), ("budget_gate", C.c_int32), ("n_unobservable", C.c_int64)]


class qsim_batch_opts(C.Structure):
    _fields_ = [("tile_qubits", C.c_int32), ("low_qubits", C.c_int32), ("ctas", C.c_int32),
                ("use_graph", C.c_int32), ("path", C.c_int32), ("tune_cache", C.c_char_p), ("stream", C.c_void_p)]


_lib = None
P = C.c_void_p


def _sig(L):
    i32, u64, f64, f32 = C.c_int, C.c_uint64, C.c_double, C.c_float
    S = C.c_int
    pp = C.POINTER(C.c_void_p)
    table = {
        "qsim_create": [i32, i32, P, pp],
        "qsim_wrap": [i32, i32, P, P, pp],
        "qsim_destroy": [P],
        "qsim_set_basis": [P, u64],
        "qsim_upload": [P, P],
        "qsim_download": [P, P],
        "qsim_device_ptr": [P, pp],
        "qsim_qubit_map": [P, P],
        "qsim_materialize": [P],
        "qsim_synchronize": [P],
        "qsim_download_async": [P, P],
        "qsim_plan_execute_norm": [P, P, P],
        "qsim_selftest_wait_timeout": [P, C.c_int64],
        "qsim_apply_gate": [P, P, i32, P, i32, u64],
        "qsim_apply_cphase": [P, i32, i32, f64],
        "qsim_apply_2q": [P, P, i32, i32],
        "qsim_apply_swap": [P, i32, i32, i32],
        "qsim_apply_fused": [P, i32, P, P, i32],
        "qsim_run_circuit": [P, P, P],
        "qsim_plan_create": [P, i32, P, pp],
        "qsim_plan_create_for_state": [P, P, P, pp],
        "qsim_plan_destroy": [P],
        "qsim_plan_info": [P, P],
        "qsim_plan_execute": [P, P],
        "qsim_norm": [P, P],
        "qsim_renormalize": [P],
        "qsim_measure_prob": [P, i32, P],
        "qsim_probs": [P, P],
        "qsim_inner_product": [P, P, P],
        "qsim_inner_product_noalloc": [P, P, i32, i32, P, P],
        "qsim_bloch": [P, i32, P],
        "qsim_bloch_all": [P, P],
        "qsim_approx_run": [P, f64, P, P],
        "qsim_batch_create": [P, i32, P, pp],
        "qsim_batch_destroy": [P],
        "qsim_batch_upload": [P, i32, P],
        "qsim_batch_reset": [P],
        "qsim_batch_run": [P, P, P],
        "qsim_batch_download": [P, i32, P],
        "qsim_batch_info": [P, P],
        "qsim_autotune": [P, i32, C.c_char_p, P, P],
        "qsim_mlp_create": [i32, i32, u64, pp],
        "qsim_mlp_destroy": [P],
        "qsim_mlp_num_params": [P, P],
        "qsim_mlp_get_params": [P, P],
        "qsim_mlp_set_params": [P, P],
        "qsim_mlp_infer": [P, P, i32, i32, P],
        "qsim_mlp_loss_grad": [P, P, P, i32, P, P],
        "qsim_mlp_train_step": [P, P, P, i32, f32, P],
    }
    for name, args in table.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = S
    L.qsim_last_error.restype = C.c_char_p
    L.qsim_last_error.argtypes = []
    L.qsim_version.restype = C.c_char_p
    L.qsim_version.argtypes = []
    return table


EXPORTED = None


def lib():
    """Loads libqsim.so (raises if it is missing: no CPU fallback exists)."""
    global _lib, EXPORTED
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2304_14969_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        EXPORTED = sorted(_sig(L)) + ["qsim_last_error", "qsim_version"]
        _lib = L
    return _lib


def _check(st):
    if st != 0:
        raise QsimError(st, lib().qsim_last_error().decode())
    return st


def _wrap(name):
    def f(*args):
        return _check(getattr(lib(), name)(*args))
    f.__name__ = name
    return f


for _n in ["qsim_create", "qsim_wrap", "qsim_destroy", "qsim_set_basis", "qsim_upload", "qsim_download",
           "qsim_device_ptr", "qsim_qubit_map", "qsim_materialize", "qsim_synchronize", "qsim_selftest_wait_timeout", "qsim_plan_execute_norm",
           "qsim_download_async",
           "qsim_apply_gate",
           "qsim_apply_cphase", "qsim_apply_2q", "qsim_apply_swap", "qsim_apply_fused", "qsim_run_circuit",
           "qsim_plan_create", "qsim_plan_create_for_state", "qsim_plan_destroy", "qsim_plan_info", "qsim_plan_execute", "qsim_norm",
           "qsim_renormalize", "qsim_measure_prob", "qsim_probs", "qsim_inner_product",
           "qsim_inner_product_noalloc", "qsim_bloch",
           "qsim_bloch_all", "qsim_approx_run", "qsim_batch_create", "qsim_batch_destroy", "qsim_batch_upload",
           "qsim_batch_reset", "qsim_batch_run", "qsim_batch_download", "qsim_batch_info", "qsim_autotune",
           "qsim_mlp_create", "qsim_mlp_destroy", "qsim_mlp_num_params", "qsim_mlp_get_params",
           "qsim_mlp_set_params", "qsim_mlp_infer", "qsim_mlp_loss_grad", "qsim_mlp_train_step"]:
    globals()[_n] = _wrap(_n)


def qsim_last_error() -> str:
    return lib().qsim_last_error().decode()


def qsim_version() -> str:
    return lib().qsim_version().decode()


# ------------------------------------------------------------ helpers

def _arr(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(C.c_void_p)


class Circuit:
    """qsim_circuit built from a list of workloads.Gate (keeps buffers alive)."""

    def __init__(self, n: int, gates):
        self.n = n
        self.gates = list(gates)
        self._g = (qsim_gate * max(1, len(self.gates)))()
        pool = []
        for k, g in enumerate(self.gates):
            r = self._g[k]
            r.kind = KIND[g.name]
            r.q0 = g.qubits[0]
            r.q1 = g.qubits[1] if len(g.qubits) > 1 else 0
            if len(g.controls) > MAX_CONTROLS:
                raise ValueError("too many controls")
            r.ncontrols = len(g.controls)
            cv = 0
            for j, (c, v) in enumerate(zip(g.controls, g.cvals)):
                r.controls[j] = c
                cv |= (int(v) & 1) << j
            r.control_values = cv
            for j, p in enumerate(g.params):
                r.params[j] = float(p)
            if g.matrix is not None:
                r.matrix_offset = len(pool)
                pool.extend(np.asarray(g.matrix, dtype=np.complex128).ravel().view(np.float64).tolist())
            else:
                r.matrix_offset = -1
        self._pool = np.ascontiguousarray(pool if pool else [0.0], dtype=np.float64)
        self.c = qsim_circuit(n, len(self.gates), self._g,
                              self._pool.ctypes.data_as(C.POINTER(C.c_double)), len(pool))

    def ptr(self):
        return C.byref(self.c)


class State:
    """Owning handle of a qsim_state (library-allocated ket)."""

    def __init__(self, n: int, dtype: int = QSIM_C64, stream=None, dev_ptr=None):
        self.n, self.dtype = n, dtype
        h = C.c_void_p()
        if dev_ptr is None:
            qsim_create(n, dtype, stream, C.byref(h))
        else:
            qsim_wrap(n, dtype, C.c_void_p(dev_ptr), stream, C.byref(h))
        self.h = h

    def close(self):
        if self.h:
            qsim_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def np_dtype(self):
        return np.complex64 if self.dtype == QSIM_C64 else np.complex128

    def upload(self, psi):
        a, p = _arr(psi, self.np_dtype)
        assert a.size == 1 << self.n
        qsim_upload(self.h, p)

    def download(self):
        out = np.empty(1 << self.n, dtype=self.np_dtype)
        qsim_download(self.h, out.ctypes.data_as(C.c_void_p))
        return out

    def run(self, circ: Circuit, mode=QSIM_MODE_PER_GATE, relabel=0, prec=QSIM_PREC_NATIVE, tile=0, max_block=0):
        o = qsim_run_opts(mode=mode, prec=prec, tile_qubits=tile, max_block=max_block, relabel_swaps=relabel)
        qsim_run_circuit(self.h, circ.ptr(), C.byref(o))

    def norm(self):
        x = C.c_double()
        qsim_norm(self.h, C.byref(x))
        return x.value

    def prob1(self, q):
        x = C.c_double()
        qsim_measure_prob(self.h, q, C.byref(x))
        return x.value

    def probs(self):
        out = np.empty(1 << self.n, dtype=np.float64)
        qsim_probs(self.h, out.ctypes.data_as(C.c_void_p))
        return out

    def bloch(self, q):
        r = (C.c_double * 3)()
        qsim_bloch(self.h, q, r)
        return np.array(r[:])

    def bloch_all(self):
        r = np.zeros(3 * self.n)
        qsim_bloch_all(self.h, r.ctypes.data_as(C.c_void_p))
        return r.reshape(self.n, 3)

    def inner(self, other: "State"):
        r = (C.c_double * 2)()
        qsim_inner_product(self.h, other.h, r)
        return complex(r[0], r[1])

    def qubit_map(self):
        m = np.zeros(self.n, dtype=np.int32)
        qsim_qubit_map(self.h, m.ctypes.data_as(C.c_void_p))
        return m


class Plan:
    """Fused plan; with `state` it starts from that state's current qubit map."""

    def __init__(self, circ: Circuit, dtype=QSIM_C64, prec=QSIM_PREC_NATIVE, tile=0, state=None, max_block=0):
        self.circ = circ
        o = qsim_run_opts(mode=QSIM_MODE_FUSED, prec=prec, tile_qubits=tile, max_block=max_block, relabel_swaps=1)
        h = C.c_void_p()
        if state is None:
            qsim_plan_create(circ.ptr(), dtype, C.byref(o), C.byref(h))
        else:
            qsim_plan_create_for_state(circ.ptr(), state.h, C.byref(o), C.byref(h))
        self.h = h

    def info(self):
        a = np.zeros(8, dtype=np.int64)
        qsim_plan_info(self.h, a.ctypes.data_as(C.c_void_p))
        keys = ["passes", "gates", "dense", "swaps_relabelled", "tile_qubits", "low_qubits", "per_gate_steps",
                "transposes"]
        return dict(zip(keys, a.tolist()))

    def execute(self, st: State):
        qsim_plan_execute(st.h, self.h)

    def execute_norm(self, st: State) -> float:
        """Executes the plan and returns the FP64 sum of |psi_i|^2 of the result."""
        x = C.c_double()
        qsim_plan_execute_norm(st.h, self.h, C.byref(x))
        return x.value

    def close(self):
        if self.h:
            qsim_plan_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def u2(m) -> np.ndarray:
    """2x2 complex -> 8 doubles (re/im interleaved, row-major)."""
    return np.ascontiguousarray(np.asarray(m, dtype=np.complex128).ravel().view(np.float64))


def approx_run(n, gates, p, dtype=QSIM_C64, tau=0.0, budget=0.0, schedule=QSIM_SCHED_EXHAUSTIVE, mlp=None,
               top_m=4, fallback_every=0, exhaustive_from=0, want_state=False, trace_cap=0, log_cap=0,
               unobservable=0, pairs=0):
    """qsim_approx_run on a list of workloads.Gate; returns (result, state or
    None, (features, labels) or None, decisions list)."""
    circ = Circuit(n, gates)
    o = qsim_approx_opts()
    o.dtype = dtype
    o.tau = tau
    o.budget_bytes = budget
    o.schedule = schedule
    o.top_m = top_m
    o.fallback_every = fallback_every
    o.exhaustive_from = exhaustive_from
    o.unobservable = int(unobservable)
    o.pairs = int(pairs)
    if mlp is not None:
        o.mlp = mlp
    state = None
    if want_state:
        state = np.zeros(1 << n, dtype=np.complex64 if dtype == QSIM_C64 else np.complex128)
        o.state_out = state.ctypes.data_as(C.c_void_p)
    feats = labels = None
    if trace_cap:
        feats = np.zeros((trace_cap, 12), dtype=np.float32)
        labels = np.zeros(trace_cap, dtype=np.int32)
        o.trace_features = feats.ctypes.data_as(C.POINTER(C.c_float))
        o.trace_labels = labels.ctypes.data_as(C.POINTER(C.c_int32))
        o.trace_cap = trace_cap
    log = None
    if log_cap:
        log = (qsim_decision * log_cap)()
        o.log = log
        o.log_cap = log_cap
    r = qsim_approx_result()
    qsim_approx_run(circ.ptr(), float(p), C.byref(o), C.byref(r))
    tr = None
    if trace_cap:
        k = min(r.n_trace, trace_cap)
        tr = (feats[:k].copy(), labels[:k].copy())
    dec = []
    if log_cap:
        dec = [(log[i].gate, log[i].qubit, log[i].action, log[i].eps) for i in range(min(r.n_log, log_cap))]
    return r, state, tr, dec
