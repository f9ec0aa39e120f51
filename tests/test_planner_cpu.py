"""Host-side check of the tensor-core block planner (no GPU).

The planner groups a circuit into <= 6-qubit dense blocks, defers diagonal
gates (controlled phases, Z/S/T/phase, the diagonal part of fSim) into the
next block that needs them, either folded into the block matrix or, for a
term whose partner qubit stays outside, as a per-group phase read from the
group index, and relabels SWAPs (Table I). tests/tc_plan_emu.cpp applies the
resulting steps on the CPU exactly as the block kernel interprets them; the
result must equal the FP64 oracle's state for the same circuit."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2304_14969_gb300 import qsim as Q
from paper_2304_14969_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2304_14969_gb300", "csrc")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


@pytest.fixture(scope="module")
def emu():
    out = os.path.join(HERE, "_build", "libtcemu.so")
    os.makedirs(os.path.dirname(out), exist_ok=True)
    srcs = [os.path.join(HERE, "tc_plan_emu.cpp"), os.path.join(CSRC, "planner.cpp"), os.path.join(CSRC, "gates.cpp"),
            os.path.join(CSRC, "tc_geom.cpp")]
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
           "-I", os.path.join(CUDA, "include"), "-o", out] + srcs + \
          ["-L", os.path.join(CUDA, "lib64"), "-lcudart", "-Wl,-rpath," + os.path.join(CUDA, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail("building the planner emulator failed:\n" + r.stderr[-3000:])
    lib = C.CDLL(out)
    lib.emu_tc_run.restype = C.c_int
    return lib


@pytest.fixture(scope="module")
def femu():
    """CPU emulation of fused SIMT plans (tests/fused_plan_emu.cpp)."""
    out = os.path.join(HERE, "_build", "libfusedemu.so")
    os.makedirs(os.path.dirname(out), exist_ok=True)
    srcs = [os.path.join(HERE, "fused_plan_emu.cpp"), os.path.join(CSRC, "planner.cpp"), os.path.join(CSRC, "gates.cpp"),
            os.path.join(CSRC, "tc_geom.cpp")]
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
           "-I", os.path.join(CUDA, "include"), "-o", out] + srcs + \
          ["-L", os.path.join(CUDA, "lib64"), "-lcudart", "-Wl,-rpath," + os.path.join(CUDA, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail("building the fused-plan emulator failed:\n" + r.stderr[-3000:])
    lib = C.CDLL(out)
    lib.emu_fused_run.restype = C.c_int
    return lib


def run_fused(lib, n, gates, x, dt, tile=0, start=None):
    c = Q.Circuit(n, gates)
    y = np.ascontiguousarray(x.astype(np.complex128)).copy()
    info = (C.c_int64 * 4)()
    sp = (C.c_int * n)(*start) if start is not None else None
    rc = lib.emu_fused_run(c.ptr(), dt, tile, sp, y.ctypes.data_as(C.c_void_p), info)
    assert rc == 0, rc
    return y, list(info)


def run(lib, n, gates, x, start=None, prec=1, max_block=0):
    c = Q.Circuit(n, gates)
    y = np.ascontiguousarray(x.astype(np.complex128)).copy()
    info = (C.c_int64 * 3)()
    sp = (C.c_int * n)(*start) if start is not None else None
    rc = lib.emu_tc_run(c.ptr(), prec, sp, max_block, y.ctypes.data_as(C.c_void_p), info)
    assert rc == 0, rc
    return y, list(info)


def infid(y, ref):
    return 1 - abs(np.vdot(ref, y)) ** 2 / (np.vdot(ref, ref).real * np.vdot(y, y).real)


CASES = {
    "grid20": lambda: (20, W.grid_rcs_circuit(4, 5, 8, seed=2), W.basis_state(20, 0)),
    "paper16": lambda: (16, W.paper_random_circuit(4, 4, 6, seed=3), W.gaussian_state(16, 3)),
    "random14": lambda: (14, W.random_1q_circuit(14, 200, 5), W.gaussian_state(14, 5)),
    "random10": lambda: (10, W.random_1q_circuit(10, 300, 11), W.gaussian_state(10, 11)),
    "qft16": lambda: (16, W.qft_circuit(16), W.gaussian_state(16, 6)),
    "iqft12": lambda: (12, W.inverse_circuit(W.qft_circuit(12)), W.gaussian_state(12, 2)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_tc_plan_matches_oracle(emu, name):
    n, g, x = CASES[name]()
    ref = oracle.apply_circuit(x, g)
    y, info = run(emu, n, g, x)
    assert info[0] >= 1
    assert infid(y, ref) <= 1e-12
    assert np.max(np.abs(y - ref)) <= 1e-12


FUSED_CASES = {
    "qft14": lambda: (14, W.qft_circuit(14), W.gaussian_state(14, 1)),
    "iqft12": lambda: (12, W.inverse_circuit(W.qft_circuit(12)), W.gaussian_state(12, 2)),
    "grid16": lambda: (16, W.grid_rcs_circuit(4, 4, 8, seed=3), W.gaussian_state(16, 3)),
    "paper15": lambda: (15, W.paper_random_circuit(3, 5, 6, seed=4), W.gaussian_state(15, 4)),
    "random13": lambda: (13, W.random_1q_circuit(13, 250, 7), W.gaussian_state(13, 7)),
    # 2-D circuits whose passes take their high qubits from candidate sets
    "grid20": lambda: (20, W.grid_rcs_circuit(4, 5, 10, seed=1), W.gaussian_state(20, 5)),
    "paper20": lambda: (20, W.paper_random_circuit(4, 5, 9, seed=2), W.gaussian_state(20, 5)),
}


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("name", sorted(FUSED_CASES))
def test_fused_plan_matches_oracle(femu, name, dt):
    """Fused SIMT plans (passes of on-chip tiles, deferred phases, register
    transposes), applied on the CPU with the kernel's semantics for the
    staged constant block, against the oracle: infidelity <= 1e-12 for
    complex128 plans (FP64 coefficients), <= 1e-6 for complex64 ones (FP32
    coefficients)."""
    n, g, x = FUSED_CASES[name]()
    ref = oracle.apply_circuit(x, g)
    y, info = run_fused(femu, n, g, x, dt)
    assert info[0] >= 1
    assert infid(y, ref) <= (1e-12 if dt else 1e-6)


@pytest.mark.parametrize("tile", [9, 10, 11, 12])
def test_fused_plan_tile_sizes_and_start_maps(femu, tile):
    """Smaller tiles (more passes, more deferred phases from outside the
    tile) and a permuted start map."""
    n, g, x = FUSED_CASES["grid16"]()
    ref = oracle.apply_circuit(x, g)
    start = [int(v) for v in np.random.default_rng(tile).permutation(n)]
    for dt in (0, 1):
        y, info = run_fused(femu, n, g, x, dt, tile=tile, start=start)
        assert infid(y, ref) <= (1e-12 if dt else 1e-6)
    n, g, x = FUSED_CASES["qft14"]()
    y, _ = run_fused(femu, n, g, x, 1, tile=tile, start=list(range(n))[::-1])
    assert infid(y, oracle.apply_circuit(x, g)) <= 1e-12


@pytest.mark.parametrize("name", ["qft16", "random14", "grid20"])
def test_tc_plan_from_permuted_map(emu, name):
    """Plans start from a state's current qubit map (bit-reversed after an
    odd number of QFTs with relabelled SWAPs)."""
    n, g, x = CASES[name]()
    ref = oracle.apply_circuit(x, g)
    rng = np.random.default_rng(n)
    for start in (list(range(n))[::-1], [int(v) for v in rng.permutation(n)]):
        y, _ = run(emu, n, g, x, start=start)
        assert infid(y, ref) <= 1e-12


@pytest.mark.parametrize("case", ["grid", "paper"])
def test_tc_plan_candidate_sets_on_grids(emu, case):
    """On 2-D circuits the planner picks each block's qubits among candidate
    sets (interaction-graph clusters), which a first-fit sweep would not: a
    4x5 grid circuit of 8 layers takes at most 12 blocks (first fit: 16) and
    the paper-family 4x5 circuit at most 13; the result still matches the
    oracle from a Gaussian ket and from a permuted start map."""
    n = 20
    g = W.grid_rcs_circuit(4, 5, 8, seed=2) if case == "grid" else W.paper_random_circuit(4, 5, 8, seed=9)
    x = W.gaussian_state(n, 21)
    ref = oracle.apply_circuit(x, g)
    y, info = run(emu, n, g, x)
    assert info[0] <= (12 if case == "grid" else 13)
    assert infid(y, ref) <= 1e-12 and np.max(np.abs(y - ref)) <= 1e-12
    start = [int(v) for v in np.random.default_rng(5).permutation(n)]
    y, _ = run(emu, n, g, x, start=start)
    assert infid(y, ref) <= 1e-12


@pytest.mark.parametrize("name", ["grid20", "paper16", "random14", "qft16"])
def test_tc_plan7_matches_oracle(emu, name):
    """Plans of 7-qubit blocks (max_block = 7, the 7-qubit kernel): the same
    sweep with blocks of up to 7 qubits, padded to 7. Applied as the kernel
    interprets them (deferred phases from the group index, then the
    128 x 128 block), they must give the oracle's state, from the identity
    map and from a permuted one, with no more blocks than 6-qubit plans."""
    n, g, x = CASES[name]()
    ref = oracle.apply_circuit(x, g)
    y, info = run(emu, n, g, x, prec=2, max_block=7)
    _, info6 = run(emu, n, g, x, prec=2)
    assert info[0] <= info6[0]
    assert infid(y, ref) <= 1e-12 and np.max(np.abs(y - ref)) <= 1e-12
    start = [int(v) for v in np.random.default_rng(9).permutation(n)]
    y, _ = run(emu, n, g, x, start=start, prec=2, max_block=7)
    assert infid(y, ref) <= 1e-12 and np.max(np.abs(y - ref)) <= 1e-12


def test_tc_plan7_refused_outside_its_kernel():
    """7-qubit blocks exist for complex64 kets with BF16X3 and n >= 14 only;
    other requests fail at plan creation (no silent fallback to 6)."""
    Q.lib()
    c = Q.Circuit(16, W.qft_circuit(16))
    for dt, prec in [(Q.QSIM_C128, Q.QSIM_PREC_BF16X6), (Q.QSIM_C64, Q.QSIM_PREC_3XTF32)]:
        with pytest.raises(Q.QsimError):
            Q.Plan(c, dtype=dt, prec=prec, max_block=7)
    with pytest.raises(Q.QsimError):
        Q.Plan(Q.Circuit(13, W.qft_circuit(13)), dtype=Q.QSIM_C64, prec=Q.QSIM_PREC_BF16X3, max_block=7)
    assert Q.Plan(c, dtype=Q.QSIM_C64, prec=Q.QSIM_PREC_BF16X3, max_block=7).info()["passes"] == 3


def test_tc_plan_qft_block_count(emu):
    """QFT-16: controlled phases deferred into the Hadamards' blocks; the
    whole transform takes three six-qubit blocks and no per-gate step."""
    n, g, x = CASES["qft16"]()
    _, info = run(emu, n, g, x)
    assert info[0] == 3 and info[1] == 0


@pytest.mark.parametrize("n", [6, 7, 8, 9])
def test_tc_plan_padding_with_partner_qubits(emu, n):
    """Blocks of fewer than six qubits are padded with free qubits; in a small
    QFT the only free ones are often partners of the block's deferred phases,
    which then act inside the block rather than from the group index."""
    g, x = W.qft_circuit(n), W.gaussian_state(n, n)
    ref = oracle.apply_circuit(x, g)
    y, info = run(emu, n, g, x)
    assert infid(y, ref) <= 1e-12
    assert np.max(np.abs(y - ref)) <= 1e-12


def tile_base(tpos, t):
    base = t
    for p in tpos:
        base = ((base >> p) << (p + 1)) | (base & ((1 << p) - 1))
    return base


def block_qubits(rng, seed, n, kb=6):
    if seed % 4 == 0:
        q6 = [int(v) for v in rng.choice(n, kb, replace=False)]
    elif seed % 4 == 1:
        q6 = [int(v) for v in rng.choice(np.arange(0, n, 2), kb, replace=False)]
    elif seed % 4 == 2:
        q6 = [n - 1 - i for i in range(kb)]
    else:
        q6 = [int(v) for v in rng.choice(min(n, kb + 3), kb, replace=False)]
    return sorted(q6)                # tc_build orders block bits by qubit


def geometry(emu, n, qk, kind):
    kb = 7 if kind == 3 else 6
    dims = (C.c_int64 * 40)()
    tpos = (C.c_int * 14)()
    posL, posG = (C.c_int * 128)(), (C.c_int * 128)()
    spL, spG = (C.c_uint64 * 128)(), (C.c_uint64 * 128)()
    rc = emu.emu_tc_geometry(n, (C.c_int * kb)(*qk), kind, dims, tpos, posL, posG, spL, spG)
    return rc, list(dims), list(tpos)[:kb + 7], list(posL)[:1 << kb], list(posG), list(spL)[:1 << kb], list(spG)


@pytest.mark.parametrize("kind", [0, 1, 2, 3])
@pytest.mark.parametrize("seed", range(40))
def test_tc_pipe_tile_geometry(emu, seed, kind):
    """The pipelined tensor-core kernel loads a tile (the block's 6 qubits and
    the 7 lowest others) with up to four 5-D TMA boxes of 8-byte elements.
    Replaying the box semantics (element (i0..i4) of box v sits at sum_d
    (c_d + i_d) * stride_d, c_4 shifted by the box's offset; the boxes land
    one after another in shared memory, dimension 0 fastest) must give every
    amplitude of the tile exactly once, at the in-stage index posL[l] |
    posG[g] the kernel reads, with all coordinates inside the tensor. For
    complex128 (kind 1) and for complex64 with TF32 operands (kind 2) a load
    is a quarter tile: the block's two highest qubits (block bits 4, 5: the
    converter's part) are fixed by the load's index and the in-stage index
    ranks the other 11 tile qubits; for complex128 dimension 0 counts the
    two 8-byte halves of an amplitude. 7-qubit blocks (kind 3): the tile has
    14 qubits and a load is an eighth of it, block bits 4, 5, 6 fixed by the
    load's index (the A chunk l >> 4 the converters write)."""
    wide = kind == 1
    split = kind != 0
    kb = 7 if kind == 3 else 6
    ntq = kb + 7
    rng = np.random.default_rng(seed)
    n = int(rng.integers(ntq, 31))
    q6 = block_qubits(rng, seed, n, kb)
    rc, d, tp, posL, posG, spL, spG = geometry(emu, n, q6, kind)
    assert rc == 0
    assert d[36] == kind and d[38] == kb
    lo, bits, box, gdim, gstr = d[0:5], d[5:10], d[10:15], d[15:20], d[20:24]
    nload, xoff, box_bytes = d[24], d[25:29], d[29]
    rot_bits, vecw, rot_shift, dwide = d[30], d[31], d[32], d[33]
    qpos = d[34:36] + [d[37]]
    es = 16 if wide else 8                  # bytes per amplitude
    hpa = es // 8                           # 8-byte elements per amplitude
    assert dwide == wide and rot_shift == (3 if wide else 4)
    assert sorted(tp) == tp and set(q6) <= set(tp)
    free = [p for p in range(n) if p not in q6][:7]
    assert sorted(set(q6) | set(free)) == tp
    strides = [8] + gstr          # bytes; dimension 0 is contiguous
    for k in range(1, 5):          # dense, non-overlapping dimensions
        assert strides[k] == strides[k - 1] * gdim[k - 1]
        assert strides[k] % 16 == 0 and strides[k] < 2 ** 40
    assert all(1 <= b <= 256 for b in box) and box[0] * 8 % 16 == 0
    assert gdim[0] * 8 == es << bits[0]
    nsel = kb - 4 if split else 0           # block bits that select a load
    nq = 1 << nsel                          # loads per tile
    tile = 1 << ntq                         # amplitudes per tile
    stage_elems = tile * es // 8 // nq      # 8-byte elements per load
    assert box_bytes == 8 * int(np.prod(box)) and box_bytes * nload == stage_elems * 8
    assert stage_elems * 8 <= (16384 if kind in (2, 3) else 32768 if wide else 65536)

    # the load of (g, l): its bits at the load-select qubits, which are block
    # bits 4.., i.e. l >> 4
    def load_of(g, l):
        x = spG[g] | spL[l]
        return sum(((x >> qpos[i]) & 1) << i for i in range(nsel))

    if split:
        assert qpos[:nsel] == q6[4:kb]
        for g in range(0, 128, 9):
            for l in range(0, 1 << kb, 5):
                assert load_of(g, l) == l >> 4
    ntiles = 1 << (n - ntq)
    for t in {0, ntiles - 1, int(rng.integers(0, ntiles))}:
        base = tile_base(tp, t)
        assert all(not (base >> p) & 1 for p in tp)
        for q in range(nq):
            bq = base | sum(((q >> i) & 1) << qpos[i] for i in range(nsel))
            c = [(bq >> lo[k]) & ((1 << bits[k]) - 1) for k in range(5)]
            c[0] *= hpa
            stage = np.full(stage_elems, -1, dtype=np.int64)
            for v in range(nload):
                cc = list(c)
                cc[4] += xoff[v]
                for k in range(5):
                    assert 0 <= cc[k] and cc[k] + box[k] <= gdim[k]
                idx = np.zeros(1, dtype=np.int64)
                for k in range(5):       # box elements, dimension 0 fastest
                    off = (cc[k] + np.arange(box[k], dtype=np.int64)) * (strides[k] // 8)
                    idx = (idx[None, :] + off[:, None]).reshape(-1)
                stage[v * (box_bytes // 8):(v + 1) * (box_bytes // 8)] = idx
            gl = [(g, l) for g in range(128) for l in range(1 << kb) if not split or load_of(g, l) == q]
            assert len(gl) == tile // nq
            want = np.array([base + spL[l] + spG[g] for g, l in gl], dtype=np.int64)
            pos = np.array([posL[l] | posG[g] for g, l in gl])
            assert np.array_equal(np.sort(pos), np.arange(tile // nq))
            for h in range(hpa):         # each 8-byte half of the amplitude
                assert np.array_equal(stage[pos * hpa + h], want * hpa + h)
    # converter reads: lane (group g = 32 quarter + lane) reads block index
    # 16 part + (i ^ rot(lane)) at instruction i; the 2^rot_shift lanes that
    # share a 128-byte shared-memory row must hit distinct slots of it
    row = 1 << rot_shift
    assert rot_bits == sum(q < rot_shift for q in q6)
    # store runs: 2^vecw adjacent amplitudes, at most 32 bytes, aligned
    run = 0
    while run < len(q6) and q6[run] == run:
        run += 1
    assert vecw == (0 if wide else min(run, 2))
    for quarter in range(4):
        for part in range(1 << (kb - 4)):
            for i in range(16):
                for hw in range(32 // row):
                    slots = set()
                    for lane in range(row * hw, row * hw + row):
                        rot = (lane >> (rot_shift - rot_bits)) & ((1 << rot_bits) - 1) if rot_bits else 0
                        g, l = 32 * quarter + lane, 16 * part + (i ^ rot)
                        slots.add((posG[g] | posL[l]) % row)
                    assert len(slots) == row, (q6, quarter, part, i, hw)
    w = 1 << vecw
    for l in range(0, 1 << kb, w):
        assert all(spL[l + i] == spL[l] + i for i in range(w)) and spL[l] % w == 0
    assert all(spG[g] % w == 0 for g in range(128))


@pytest.mark.parametrize("kind", [0, 1, 2, 3])
def test_tc_pipe_geometry_always_covered(emu, kind):
    """Every block the planner can emit has a tile geometry (at most five
    tensor dimensions plus two extra-box qubits): all blocks among qubits
    0..13 (0..14 for 7-qubit blocks) at n = 20, and random blocks at n up to
    36."""
    import itertools
    kb = 7 if kind == 3 else 6
    cases = [(20, list(q)) for q in itertools.combinations(range(kb + 8), kb)]
    rng = np.random.default_rng(7)
    for _ in range(3000):
        n = int(rng.integers(kb + 7, 37))
        cases.append((n, sorted(int(v) for v in rng.choice(n, kb, replace=False))))
    for n, q6 in cases:
        rc = geometry(emu, n, q6, kind)[0]
        assert rc == 0, (n, q6, kind)


@pytest.mark.parametrize("kb", [6, 7])
@pytest.mark.parametrize("seed", range(12))
def test_tc_pipe_phase_tables(emu, seed, kb):
    """Deferred phases in the pipelined kernels: block bit b of the amplitude
    with index x is multiplied by exp(2 pi i T_b(x)), T_b(x) = sum of the
    turns of b's partners whose bit is set in x. The kernel forms it as
    (tile factor from tturn[b][tile-index bits]) x gfac[g][b]; for random
    partner lists and amplitudes that product must equal the direct sum
    (kb = 6 or 7 block bits; the tile is the block and the 7 lowest other
    qubits)."""
    rng = np.random.default_rng(100 + seed)
    ntq = kb + 7
    n = int(rng.integers(ntq, 29))
    q6 = [int(v) for v in rng.choice(n, kb, replace=False)]
    outside = [p for p in range(n) if p not in q6]
    off, pbit, tw = [0], [], []
    for b in range(kb):
        k = int(rng.integers(0, min(12, len(outside)) + 1))
        for p in rng.choice(outside, k, replace=False):
            pbit.append(int(p))
            tw.append(int(rng.integers(0, 2 ** 63)) * 2 + int(rng.integers(0, 2)))
        off.append(len(pbit))
    out = np.zeros(kb * 24 * 8 + 128 * kb * 8, dtype=np.uint8)
    rc = emu.emu_tc_tables(n, kb, (C.c_int * kb)(*q6), (C.c_int32 * (kb + 1))(*off),
                           (C.c_int32 * max(1, len(pbit)))(*pbit), (C.c_uint64 * max(1, len(tw)))(*tw),
                           out.ctypes.data_as(C.c_void_p))
    assert rc == out.size
    tturn = out[:kb * 24 * 8].view(np.uint64).reshape(kb, 24)
    gfac = out[kb * 24 * 8:].view(np.float32).reshape(128, kb, 2)
    free = [p for p in range(n) if p not in q6][:7]
    tile = sorted(q6 + free)
    tbits = [p for p in range(n) if p not in tile]
    for _ in range(20):
        t = int(rng.integers(0, 1 << (n - ntq)))
        gi = int(rng.integers(0, 128))
        x = sum(1 << tbits[i] for i in range(n - ntq) if (t >> i) & 1)
        x |= sum(1 << free[f] for f in range(7) if (gi >> f) & 1)
        for b in range(kb):
            direct = sum(tw[e] for e in range(off[b], off[b + 1]) if (x >> pbit[e]) & 1) % 2 ** 64
            tt = sum(int(tturn[b, i]) for i in range(n - ntq) if (t >> i) & 1) % 2 ** 64
            f = np.exp(2j * np.pi * tt / 2 ** 64) * complex(gfac[gi, b, 0], gfac[gi, b, 1])
            assert abs(f - np.exp(2j * np.pi * direct / 2 ** 64)) < 1e-6


# Passes of fused SIMT plans and blocks of tensor-core plans (plan only, no
# GPU): the per-pass / per-block choice among candidate high-qubit sets gives
# these counts; first-fit tiles give grid20 9 / 11, paper20 6 / 9, grid30
# 17 / 21 passes (complex64 / complex128) and 30 tensor-core blocks on grid30.
# The last column is 7-qubit blocks (max_block = 7).
# A regression that turns the choice off, or plans more passes, fails here.
PASS_COUNTS = {
    "grid20": (lambda: (20, W.grid_rcs_circuit(4, 5, 10, seed=1)), 7, 10, 15, 11),
    "paper20": (lambda: (20, W.paper_random_circuit(4, 5, 9, seed=2)), 6, 7, 15, 11),
    "grid30": (lambda: (30, W.grid_rcs_circuit(5, 6, 10, seed=0)), 14, 17, 22, 20),
    "paper30": (lambda: (30, W.paper_random_circuit(5, 6, 10, seed=0)), 13, 15, 24, 22),
    "qft27": (lambda: (27, W.qft_circuit(27)), 3, 4, 5, 4),
}


@pytest.mark.parametrize("name", sorted(PASS_COUNTS))
def test_plan_pass_counts(name):
    mk, c64, c128, tc, tc7 = PASS_COUNTS[name]
    n, g = mk()
    Q.lib()
    circ = Q.Circuit(n, g)
    assert Q.Plan(circ, dtype=Q.QSIM_C64).info()["passes"] == c64
    assert Q.Plan(circ, dtype=Q.QSIM_C128).info()["passes"] == c128
    assert Q.Plan(circ, dtype=Q.QSIM_C64, prec=Q.QSIM_PREC_BF16X3).info()["passes"] == tc
    assert Q.Plan(circ, dtype=Q.QSIM_C64, prec=Q.QSIM_PREC_BF16X3, max_block=7).info()["passes"] == tc7
