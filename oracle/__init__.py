"""Plain FP64 CPU oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It shares no code with the GPU library
(``paper_2304_14969_gb300``) and never imports it; both sides read circuits
from the seeded generators in ``paper_2304_14969_gb300.workloads``, which hold
no arithmetic of the method.

The arithmetic lives in ``oracle.c`` (single-threaded C, ``double complex``),
compiled here with gcc into ``oracle/_build/liboracle.so``. This module only
marshals numpy arrays into it. The same file compiled with ``-fopenmp``
(``liboracle_mt.so``, the only difference being its ``omp`` pragmas) runs the
index loops on all host cores; ``use_all_cores(True)`` routes the calls below
to it (large parity cases and the all-core CPU baseline). The one-thread build
stays the default and is the one the pins check; the all-core build is checked
against it. Paper sections followed (arXiv 2304.14969):
Sec. II (gate-by-gate Schroedinger evolution), Eq. (dft) (QFT definition),
Sec. III.A (SDRP check and projection), Eq. (fid_model) and Eq. (fid_exact).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_OUT_MT = os.path.join(_HERE, "_build", "liboracle_mt.so")
_lock = threading.Lock()
_libs = {}
_all_cores = False

# The oracle's own gate numbering (mirrors the enum in oracle.c).
KIND = {
    "h": 1, "x": 2, "y": 3, "z": 4, "s": 5, "t": 6,
    "sqrtx": 7, "sqrty": 8, "sqrtw": 9, "u3": 10, "phase": 11, "rz": 12, "mat1": 13,
    "cp": 32, "swap": 33, "fsim": 34, "mat2": 35,
}
MAXCTRL = 6

GATE_DTYPE = np.dtype([
    ("kind", np.int32), ("q", np.int32, 2), ("nctrl", np.int32),
    ("ctrl", np.int32, MAXCTRL), ("cval", np.int32, MAXCTRL),
    ("prm", np.float64, 4), ("mat", np.float64, 32),
], align=True)

DECISION_DTYPE = np.dtype([
    ("gate", np.int32), ("qubit", np.int32), ("action", np.int32), ("pad", np.int32),
    ("eps", np.float64), ("r", np.float64, 3),
], align=True)


def _compile(out: str, extra, force: bool) -> str:
    with _lock:
        if (not force and os.path.exists(out)
                and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
            return out
        os.makedirs(os.path.dirname(out), exist_ok=True)
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared",
                               "-fno-fast-math", *extra, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
        return out


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (no fast-math: the compensated sums need
    IEEE semantics), one-thread and all-core builds. Returns the path of the
    one-thread library."""
    _compile(_OUT_MT, ["-fopenmp"], force)
    return _compile(_OUT, [], force)


def use_all_cores(flag: bool = True) -> None:
    """Routes the calls of this module to the all-core build (True) or the
    one-thread build (False, the default)."""
    global _all_cores
    _all_cores = bool(flag)


def threads() -> int:
    """Threads the selected build runs its index loops on."""
    return int(lib().orc_threads())


def _load(path):
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i32, f64, u64 = ctypes.c_int, ctypes.c_double, ctypes.c_uint64
    L.orc_threads.restype = i32
    L.orc_gate_matrix.argtypes = [P, P]
    L.orc_apply_circuit.argtypes = [P, i32, P, i32]
    L.orc_apply_kq.argtypes = [P, i32, i32, P, P]
    L.orc_dense_circuit.argtypes = [i32, P, i32, P]
    L.orc_norm2.argtypes = [P, i32]
    L.orc_norm2.restype = f64
    L.orc_probs.argtypes = [P, i32, P]
    L.orc_prob1.argtypes = [P, i32, i32]
    L.orc_prob1.restype = f64
    L.orc_inner.argtypes = [P, P, i32, P]
    L.orc_bloch.argtypes = [P, i32, i32, P]
    L.orc_dft_sample.argtypes = [P, i32, u64, P]
    L.orc_sdrp_project.argtypes = [P, i32, i32, P]
    L.orc_sdrp_run.argtypes = [P, i32, P, i32, f64, f64, P, i32, P, i32, i32, P, P, P, P, i32]
    L.orc_rho2.argtypes = [P, i32, i32, i32, P]
    L.orc_herm4_eig.argtypes = [P, P, P]
    L.orc_sdrp_project2.argtypes = [P, i32, i32, i32, P]
    L.orc_sdrp_run.restype = i32
    return L


def lib():
    key = "mt" if _all_cores else "st"
    if key not in _libs:
        path = build()
        _libs[key] = _load(_OUT_MT if _all_cores else path)
    return _libs[key]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _nq(psi: np.ndarray) -> int:
    n = int(psi.size).bit_length() - 1
    if psi.dtype != np.complex128 or (1 << n) != psi.size or not psi.flags.c_contiguous:
        raise ValueError("oracle states are contiguous complex128 arrays of length 2^n")
    return n


def gates_to_records(gates) -> np.ndarray:
    """Converts generator gates (objects with name, qubits, params, controls,
    cvals, matrix) into the oracle's gate records."""
    rec = np.zeros(len(gates), dtype=GATE_DTYPE)
    for k, g in enumerate(gates):
        r = rec[k]
        r["kind"] = KIND[g.name]
        r["q"][: len(g.qubits)] = g.qubits
        if len(g.controls) > MAXCTRL:
            raise ValueError("too many controls")
        r["nctrl"] = len(g.controls)
        r["ctrl"][: len(g.controls)] = g.controls
        r["cval"][: len(g.controls)] = g.cvals
        r["prm"][: len(g.params)] = g.params
        if g.matrix is not None:
            m = np.asarray(g.matrix, dtype=np.complex128).ravel()
            r["mat"][: 2 * m.size] = m.view(np.float64)
    return rec


def gate_matrix(g) -> np.ndarray:
    rec = gates_to_records([g])
    out = np.zeros(16, dtype=np.complex128)
    d = lib().orc_gate_matrix(_ptr(rec), _ptr(out))
    if d == 0:
        raise ValueError(f"unknown gate {g.name}")
    return out[: d * d].reshape(d, d).copy()


def apply_circuit(psi: np.ndarray, gates) -> np.ndarray:
    """Returns C|psi> computed gate by gate (Sec. II)."""
    n = _nq(psi)
    out = psi.copy()
    rec = gates_to_records(gates)
    if lib().orc_apply_circuit(_ptr(out), n, _ptr(rec), len(rec)):
        raise ValueError("unknown gate kind")
    return out


def apply_kq(psi: np.ndarray, qubits, u: np.ndarray) -> np.ndarray:
    n = _nq(psi)
    out = psi.copy()
    q = np.ascontiguousarray(qubits, dtype=np.int32)
    U = np.ascontiguousarray(u, dtype=np.complex128)
    assert U.shape == (1 << len(q), 1 << len(q))
    lib().orc_apply_kq(_ptr(out), n, len(q), _ptr(q), _ptr(U))
    return out


def dense_circuit(n: int, gates) -> np.ndarray:
    """2^n x 2^n matrix of the circuit from element-wise dense gate
    matrices (n <= 10)."""
    rec = gates_to_records(gates)
    M = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    if lib().orc_dense_circuit(n, _ptr(rec), len(rec), _ptr(M)):
        raise ValueError("dense check supports n <= 10 and known kinds")
    return M


def norm2(psi):
    return lib().orc_norm2(_ptr(psi), _nq(psi))


def probs(psi):
    out = np.empty(psi.size, dtype=np.float64)
    lib().orc_probs(_ptr(psi), _nq(psi), _ptr(out))
    return out


def prob1(psi, q):
    return lib().orc_prob1(_ptr(psi), _nq(psi), q)


def inner(a, b):
    """<a|b> as a Python complex."""
    out = np.zeros(2)
    n = _nq(a)
    assert _nq(b) == n
    lib().orc_inner(_ptr(a), _ptr(b), n, _ptr(out))
    return complex(out[0], out[1])


def fidelity(a, b):
    """Eq. (fid_exact): |<a|b>|^2 for normalised a, b."""
    return abs(inner(a, b)) ** 2


def bloch(psi, q):
    out = np.zeros(3)
    lib().orc_bloch(_ptr(psi), _nq(psi), q, _ptr(out))
    return out


def dft_sample(x, j):
    """Eq. (dft) evaluated at output index j from the definition."""
    out = np.zeros(2)
    lib().orc_dft_sample(_ptr(x), _nq(x), int(j), _ptr(out))
    return complex(out[0], out[1])


def sdrp_project(psi, q, r):
    out = psi.copy()
    rr = np.ascontiguousarray(r, dtype=np.float64)
    lib().orc_sdrp_project(_ptr(out), _nq(out), q, _ptr(rr))
    return out


def sdrp_run(n: int, gates, p: float, tau: float, force=None, psi0=None, force_actions=None,
             unobservable=False, stats=None, pairs=False):
    """Runs the circuit from |0...0> (or psi0, a product state) with SDRP
    rounding on the full state vector. Returns (psi, F, nround, log) where
    log is a structured array of decisions (gate, qubit, action, eps, r).
    force: (gate, qubit) checks to run instead of the exhaustive schedule;
    force_actions (with force): the decision of each forced check (0 keep,
    1 round, 2 separate exactly, -1 decide by eps). unobservable: Sec.
    II.B's elimination of Z-eigenstate controls (stats["unobservable"]
    receives the number of gates removed or reduced, when stats is a dict).
    pairs: the two-qubit-subsystem check after each gate coupling two
    qubits (log entries with pad = 1 + the pair's second qubit)."""
    psi = np.zeros(1 << n, dtype=np.complex128) if psi0 is None else psi0.astype(np.complex128).copy()
    if psi0 is None:
        psi[0] = 1.0
    rec = gates_to_records(gates)
    cap = max(16, 64 * len(gates) + 16)
    log = np.zeros(cap, dtype=DECISION_DTYPE)
    F = ctypes.c_double(0.0)
    nr = ctypes.c_int(0)
    if force is not None:
        f = np.ascontiguousarray(np.asarray(force, dtype=np.int32).reshape(-1, 2))
        fptr, nf = _ptr(f), f.shape[0]
    else:
        f, fptr, nf = None, None, 0
    aptr = None
    if force_actions is not None:
        if f is None:
            raise ValueError("force_actions needs force")
        acts = np.ascontiguousarray(np.asarray(force_actions, dtype=np.int32).reshape(-1))
        if acts.size != nf:
            raise ValueError("one action per forced check")
        aptr = _ptr(acts)
    nu = ctypes.c_int(0)
    nlog = lib().orc_sdrp_run(_ptr(psi), n, _ptr(rec), len(rec), float(p), float(tau),
                              fptr, nf, aptr, int(bool(unobservable)), int(bool(pairs)), ctypes.byref(F),
                              ctypes.byref(nr),
                              ctypes.byref(nu), _ptr(log), cap)
    if stats is not None:
        stats["unobservable"] = nu.value
    if nlog < 0:
        raise ValueError("unknown gate kind")
    return psi, F.value, nr.value, log[: min(nlog, cap)].copy()


def rho2(psi, qa, qb):
    """Normalised reduced density matrix of the pair (qa: bit 0, qb: bit 1)."""
    out = np.zeros(16, dtype=np.complex128)
    lib().orc_rho2(_ptr(psi), _nq(psi), qa, qb, _ptr(out))
    return out.reshape(4, 4)


def herm4_eig(H):
    """(eigenvalues ascending, eigenvectors as columns) of a Hermitian 4 x 4."""
    Hc = np.ascontiguousarray(H, dtype=np.complex128)
    w = np.zeros(4)
    v = np.zeros(16, dtype=np.complex128)
    lib().orc_herm4_eig(_ptr(Hc), _ptr(w), _ptr(v))
    return w, v.reshape(4, 4)


def sdrp_project2(psi, qa, qb, phi):
    out = psi.copy()
    ph = np.ascontiguousarray(phi, dtype=np.complex128)
    lib().orc_sdrp_project2(_ptr(out), _nq(out), qa, qb, _ptr(ph))
    return out
