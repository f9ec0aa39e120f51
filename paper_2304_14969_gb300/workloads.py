"""Seeded synthetic inputs: circuits and initial states.

This module is the one piece shared by the GPU path and the CPU oracle. It
describes circuits as lists of named gates with qubits and parameters and
draws seeded random inputs; it builds no gate matrix and applies nothing,
so it holds none of the simulation arithmetic. Each side turns the names
into matrices with its own code.

Workloads (arXiv 2304.14969):
  - QFT circuits (Sec. II.E, Eq. qft/dft): H plus controlled phases
    CP(2 pi / 2^m) plus the final qubit-reversal swaps, little-endian qubits.
  - Grid random circuits: per layer one gate from {sqrt(X), sqrt(Y),
    sqrt(W)} on every qubit (no immediate repeat on a qubit), then
    fSim(pi/2, pi/6) on the nearest-neighbour couplers of one of four
    patterns A, B, C, D used in turn (Sec. III.C names the Sycamore-style
    coupler patterns; the gate set is the Sycamore one).
  - The paper's own random family (Sec. III.C): U(theta, phi, lambda) on
    every qubit, then random C/A-Pauli couplers on pattern ABCDCDAB.
  - Initial states: basis |x>, iid complex Gaussian normalised in FP64,
    |0...0>, and GHZ (Eq. ghz).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

ONE_QUBIT = ("h", "x", "y", "z", "s", "t", "sqrtx", "sqrty", "sqrtw", "u3", "phase", "rz", "mat1")
TWO_QUBIT = ("cp", "swap", "fsim", "mat2")


@dataclass(frozen=True)
class Gate:
    """A named gate. qubits[0] is the target of a one-qubit gate; for a
    two-qubit gate qubits[0] is bit 0 and qubits[1] bit 1 of the 4x4
    matrix's row index. A one-qubit gate acts only where bit controls[j]
    equals cvals[j] for all j (cval 1 = "C" control, 0 = "A" control)."""
    name: str
    qubits: tuple
    params: tuple = ()
    controls: tuple = ()
    cvals: tuple = ()
    matrix: Optional[np.ndarray] = field(default=None, compare=False)

    def __post_init__(self):
        if self.name not in ONE_QUBIT + TWO_QUBIT:
            raise ValueError(f"unknown gate {self.name}")
        want = 1 if self.name in ONE_QUBIT else 2
        if len(self.qubits) != want:
            raise ValueError(f"{self.name} takes {want} qubit(s)")
        if len(self.controls) != len(self.cvals):
            raise ValueError("controls and cvals differ in length")
        if self.controls and want == 2:
            raise ValueError("controls apply to one-qubit gates only")

    @property
    def is_two_qubit(self) -> bool:
        return self.name in TWO_QUBIT or len(self.controls) > 0


# ------------------------------------------------------------------ QFT

def qft_circuit(n: int, swaps: bool = True) -> list:
    """QFT on n little-endian qubits: for t = n-1 .. 0, H(t) then
    CP(2 pi / 2^(t-c+1)) with control c, target t, for c = t-1 .. 0; then
    SWAP(q, n-1-q) for q < n/2. Gate count n(n+1)/2 + floor(n/2)."""
    g = []
    for t in range(n - 1, -1, -1):
        g.append(Gate("h", (t,)))
        for c in range(t - 1, -1, -1):
            g.append(Gate("cp", (c, t), (2.0 * math.pi / float(1 << (t - c + 1)),)))
    if swaps:
        for q in range(n // 2):
            g.append(Gate("swap", (q, n - 1 - q)))
    return g


def inverse_circuit(gates: Sequence[Gate]) -> list:
    """Gate list of the inverse circuit made of named gates: self-inverse
    gates as they are; phases, U3 and fSim with negated angles; explicit
    matrices conjugate-transposed; a gate G of finite order m (sqrt(P) has
    order 4, S order 4, T order 8) as G repeated m - 1 times."""
    inv = []
    for g in reversed(list(gates)):
        if g.name in ("h", "x", "y", "z", "swap"):
            inv.append(g)
        elif g.name in ("cp", "phase", "rz"):
            inv.append(Gate(g.name, g.qubits, (-g.params[0],), g.controls, g.cvals))
        elif g.name in ("mat1", "mat2"):
            inv.append(Gate(g.name, g.qubits, (), g.controls, g.cvals,
                            matrix=np.conj(np.asarray(g.matrix)).T.copy()))
        elif g.name == "u3":
            th, ph, la = g.params
            inv.append(Gate("u3", g.qubits, (-th, -la, -ph), g.controls, g.cvals))
        elif g.name == "fsim":
            inv.append(Gate("fsim", g.qubits, (-g.params[0], -g.params[1])))
        elif g.name in ("sqrtx", "sqrty", "sqrtw", "s", "t"):
            inv.extend([g] * (7 if g.name == "t" else 3))
        else:
            raise ValueError(f"no named inverse for {g.name}")
    return inv


# ------------------------------------------------------------ grid RCS

def grid_couplers(rows: int, cols: int, pattern: str) -> list:
    """Nearest-neighbour pairs of one pattern on a rows x cols grid, qubit
    id = r * cols + c. A: horizontal pairs starting at an even column;
    B: horizontal, odd column; C: vertical pairs starting at an even row;
    D: vertical, odd row. A grid whose last row is partial (n < rows*cols)
    drops couplers touching missing qubits at the caller."""
    out = []
    if pattern in "AB":
        par = 0 if pattern == "A" else 1
        for r in range(rows):
            for c in range(par, cols - 1, 2):
                out.append((r * cols + c, r * cols + c + 1))
    elif pattern in "CD":
        par = 0 if pattern == "C" else 1
        for r in range(par, rows - 1, 2):
            for c in range(cols):
                out.append((r * cols + c, (r + 1) * cols + c))
    else:
        raise ValueError(pattern)
    return out


def grid_rcs_circuit(rows: int, cols: int, layers: int, seed: int,
                     patterns: str = "ABCD", n: Optional[int] = None,
                     fsim_theta: float = math.pi / 2, fsim_phi: float = math.pi / 6) -> list:
    """Sycamore-style grid random circuit. Each layer: one of sqrt(X),
    sqrt(Y), sqrt(W) on every qubit (uniform over 3 in the first layer,
    afterwards uniform over the 2 that differ from the qubit's previous
    gate), then fSim(theta, phi) on every coupler of pattern
    patterns[layer % len(patterns)]. n < rows*cols keeps qubits 0..n-1."""
    nq = rows * cols if n is None else n
    rng = np.random.default_rng(seed)
    names = ("sqrtx", "sqrty", "sqrtw")
    prev = [-1] * nq
    g = []
    for layer in range(layers):
        for q in range(nq):
            if prev[q] < 0:
                k = int(rng.integers(0, 3))
            else:
                k = [x for x in range(3) if x != prev[q]][int(rng.integers(0, 2))]
            prev[q] = k
            g.append(Gate(names[k], (q,)))
        for a, b in grid_couplers(rows, cols, patterns[layer % len(patterns)]):
            if a < nq and b < nq:
                g.append(Gate("fsim", (a, b), (fsim_theta, fsim_phi)))
    return g


def grid_shape(n: int) -> tuple:
    """Grid for a circuit of n qubits: cols = ceil(sqrt(n)),
    rows = ceil(n / cols)."""
    cols = int(math.ceil(math.sqrt(n)))
    rows = int(math.ceil(n / cols))
    return rows, cols


def paper_random_circuit(rows: int, cols: int, layers: int, seed: int,
                         patterns: str = "ABCDCDAB", n: Optional[int] = None) -> list:
    """The paper's random family (Sec. III.C): U(theta, phi, lambda) on every
    qubit with theta in [0, 4 pi), phi, lambda in [0, 2 pi), then on every
    coupler of the layer's pattern one gate drawn from CX, CY, CZ, AX, AY,
    AZ with a random choice of which end is the control. n < rows * cols
    keeps the first n grid sites (couplers touching the others are dropped)."""
    nq = rows * cols if n is None else n
    rng = np.random.default_rng(seed)
    g = []
    for layer in range(layers):
        for q in range(nq):
            th = float(rng.uniform(0.0, 4.0 * math.pi))
            ph = float(rng.uniform(0.0, 2.0 * math.pi))
            la = float(rng.uniform(0.0, 2.0 * math.pi))
            g.append(Gate("u3", (q,), (th, ph, la)))
        for a, b in grid_couplers(rows, cols, patterns[layer % len(patterns)]):
            if a >= nq or b >= nq:
                continue
            pauli = ("x", "y", "z")[int(rng.integers(0, 3))]
            cval = int(rng.integers(0, 2))
            if int(rng.integers(0, 2)):
                a, b = b, a
            g.append(Gate(pauli, (b,), (), (a,), (cval,)))
    return g


# --------------------------------------------------------------- batch

def batch_circuits(count: int, seed: int, nmin: int = 10, nmax: int = 24,
                   dmin: int = 4, dmax: int = 20) -> list:
    """Mixed batch: per circuit n ~ U{nmin..nmax}, depth ~ U{dmin..dmax},
    type ~ Bernoulli(0.5) between a full QFT (depth unused) and a grid
    circuit of that depth on a ceil(sqrt(n))-column grid. Returns a list of
    dicts with keys n, kind, depth, gates, seed."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        d = int(rng.integers(dmin, dmax + 1))
        kind = "qft" if int(rng.integers(0, 2)) == 0 else "grid"
        cseed = int(rng.integers(0, 2**31 - 1))
        if kind == "qft":
            gates = qft_circuit(n)
        else:
            rows, cols = grid_shape(n)
            gates = grid_rcs_circuit(rows, cols, d, cseed, n=n)
        out.append({"n": n, "kind": kind, "depth": d, "gates": gates, "seed": cseed})
    return out


# -------------------------------------------------------------- states

def basis_index(n: int, seed: int) -> int:
    return int(np.random.default_rng(seed).integers(0, 1 << n))


def basis_state(n: int, x: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[x] = 1.0
    return psi


def gaussian_state(n: int, seed: int) -> np.ndarray:
    """iid N(0,1) real and imaginary parts, divided by the FP64 norm."""
    rng = np.random.default_rng(seed)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi /= np.sqrt(np.sum(np.abs(psi) ** 2))
    return psi.astype(np.complex128)


def ghz_state(n: int) -> np.ndarray:
    """Eq. (ghz): (|0...0> + |1...1>)/sqrt(2)."""
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = psi[-1] = 1.0 / math.sqrt(2.0)
    return psi


def random_unitary(k: int, seed: int) -> np.ndarray:
    """2^k x 2^k unitary from the QR factorisation of a complex Gaussian
    matrix with the phases of R's diagonal divided out."""
    rng = np.random.default_rng(seed)
    d = 1 << k
    z = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return (q * ph).astype(np.complex128)


def random_1q_circuit(n: int, ngates: int, seed: int, with_controls: bool = True) -> list:
    """Random mix of every gate kind on random qubits (for kernel coverage):
    named one-qubit gates, U3, controlled/anti-controlled Paulis, CP,
    SWAP, fSim and explicit random 2x2 / 4x4 unitaries."""
    rng = np.random.default_rng(seed)
    g = []
    names1 = ("h", "x", "y", "z", "s", "t", "sqrtx", "sqrty", "sqrtw")
    for i in range(ngates):
        r = int(rng.integers(0, 9 if n >= 2 else 4))
        q = int(rng.integers(0, n))
        others = [x for x in range(n) if x != q]
        if r == 0:
            g.append(Gate(names1[int(rng.integers(0, len(names1)))], (q,)))
        elif r == 1:
            g.append(Gate("u3", (q,), tuple(float(v) for v in rng.uniform(0, 2 * math.pi, 3))))
        elif r == 2:
            g.append(Gate("phase", (q,), (float(rng.uniform(0, 2 * math.pi)),)))
        elif r == 3:
            g.append(Gate("mat1", (q,), matrix=random_unitary(1, int(rng.integers(0, 2**31)))))
        elif r == 4 and with_controls:
            nc = int(rng.integers(1, min(3, n - 1) + 1))
            cs = tuple(int(x) for x in rng.choice(others, size=nc, replace=False))
            cv = tuple(int(x) for x in rng.integers(0, 2, size=nc))
            g.append(Gate(("x", "y", "z", "h", "sqrtw")[int(rng.integers(0, 5))], (q,), (), cs, cv))
        elif r == 5:
            b = int(rng.choice(others))
            g.append(Gate("cp", (q, b), (float(rng.uniform(0, 2 * math.pi)),)))
        elif r == 6:
            b = int(rng.choice(others))
            g.append(Gate("swap", (q, b)))
        elif r == 7:
            b = int(rng.choice(others))
            g.append(Gate("fsim", (q, b), tuple(float(v) for v in rng.uniform(0, 2 * math.pi, 2))))
        else:
            b = int(rng.choice(others))
            g.append(Gate("mat2", (q, b), matrix=random_unitary(2, int(rng.integers(0, 2**31)))))
    return g


def sparse_control_circuit(n: int, ngates: int, seed: int) -> list:
    """Controlled gates on a ket that stays close to the computational basis
    (a workload for the unobservable optimisation of Sec. II.B): a seeded
    mix of X and T on single qubits, an occasional H or U3, CX / anti-CX,
    two-control X, CZ (a controlled phase of pi) and controlled phases of
    random angle on random qubits. Many controls are then Z eigenstates."""
    rng = np.random.default_rng(seed)
    g = []
    for _ in range(ngates):
        r = float(rng.uniform())
        q = int(rng.integers(0, n))
        others = [x for x in range(n) if x != q]
        if r < 0.20:
            g.append(Gate("x", (q,)))
        elif r < 0.28:
            g.append(Gate("t", (q,)))
        elif r < 0.34:
            g.append(Gate("h", (q,)))
        elif r < 0.38:
            g.append(Gate("u3", (q,), tuple(float(v) for v in rng.uniform(0, 2 * math.pi, 3))))
        elif r < 0.62:
            c = int(rng.choice(others))
            g.append(Gate("x", (q,), (), (c,), (int(rng.integers(0, 2)),)))
        elif r < 0.72 and n >= 3:
            cs = tuple(int(x) for x in rng.choice(others, size=2, replace=False))
            g.append(Gate("x", (q,), (), cs, (1, int(rng.integers(0, 2)))))
        elif r < 0.86:
            g.append(Gate("cp", (q, int(rng.choice(others))), (math.pi,)))
        else:
            g.append(Gate("cp", (q, int(rng.choice(others))), (float(rng.uniform(0, 2 * math.pi)),)))
    return g
