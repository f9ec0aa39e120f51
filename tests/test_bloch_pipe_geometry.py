"""CPU model of the index arithmetic of the pipelined Bloch pass
(k_red_bloch_pipe in csrc/k_reduce.cu; Sec. III.A step 1 needs the Bloch
vectors of every qubit). The formulas below restate the kernel's: where
each thread's 16-byte copies come from and land, where its three 16-amplitude
slices are read, and how the tile base advances. Checked: every copy stays
inside its stage and the ket, the copies of a tile cover the stage exactly
once, each stage position then holds the amplitude the read patterns expect,
the reads of a warp phase hit distinct shared-memory banks, and the
masked-add advance of the tile base equals the bit insertion it replaces.
The passes' plan (which qubits each pass tiles and reports) and the sums the
passes form from their slices are emulated in FP64 against the oracle."""
import random

import numpy as np
import pytest

M64 = (1 << 64) - 1


def tile_expand(w, ins):
    for p in sorted(ins):
        w = ((w >> p) << (p + 1)) | (w & ((1 << p) - 1))
    return w


def geometry(B):
    run = 16 * B
    pad = run + 16
    gran = run // 16
    return run, pad, 256 * pad, gran, (5 if gran == 8 else 4)


def stage_image(B, n, high, tid):
    """stage byte offset -> ket byte offset of each 16-byte copy of tile tid"""
    run, pad, stage, gran, lobits = geometry(B)
    tq = [0, 1, 2, 3] + sorted(high)
    hh = []
    for t in range(gran):
        h = 0
        for b in range(8 - lobits):
            if (t >> b) & 1:
                h |= 1 << tq[4 + lobits + b]
        hh.append(h * B)
    step = (256 // gran) * pad
    base = tile_expand(tid << 4, high) * B
    img = {}
    for th in range(256):
        hlo = 0
        for b in range(lobits):
            if ((th // gran) >> b) & 1:
                hlo |= 1 << tq[4 + b]
        src0 = hlo * B + (th % gran) * 16
        dst0 = (th // gran) * pad + (th % gran) * 16
        for k in range(gran):
            d, s = dst0 + k * step, src0 + base + hh[k]
            assert 0 <= d and d + 16 <= stage
            assert s % 16 == 0 and 0 <= s and s + 16 <= (B << n)
            assert d not in img
            img[d] = s
    return img, tq


CASES = [(12, list(range(4, 12))), (27, list(range(4, 12))), (27, list(range(12, 20))),
         (27, list(range(19, 27))), (20, [4, 7, 9, 11, 13, 15, 17, 19]),
         (27, [4, 7, 10, 13, 16, 19, 22, 25]), (27, [4, 6, 9, 12, 15, 18, 21, 24])]


@pytest.mark.parametrize("B", [8, 16])
@pytest.mark.parametrize("n,high", CASES)
def test_copies_fill_the_stage_and_reads_find_their_amplitudes(B, n, high):
    run, pad, stage, gran, _ = geometry(B)
    rng = random.Random(n)
    for tid in {0, (1 << (n - 12)) - 1, rng.randrange(1 << (n - 12))}:
        img, tq = stage_image(B, n, high, tid)
        assert len(img) * 16 == 256 * run
        base = tile_expand(tid << 4, high)

        def ket_index(e):
            g = base
            for j in range(12):
                if (e >> j) & 1:
                    g |= 1 << tq[j]
            return g

        def where(e):
            return (e >> 4) * pad + (e & 15) * B

        for e in range(4096):
            at = where(e)
            assert img[at - at % 16] + at % 16 == ket_index(e) * B
        for th in range(256):
            offA = th * pad
            offB = (th >> 4) * 16 * pad + (th & 15) * B
            offC = (th >> 4) * pad + (th & 15) * B
            for r in range(16):
                assert offA + r * B == where((th << 4) | r)
                assert offB + r * pad == where((th & 15) | (r << 4) | ((th >> 4) << 8))
                assert offC + r * 16 * pad == where(th | (r << 8))


@pytest.mark.parametrize("B", [8, 16])
def test_no_bank_conflicts(B):
    """16-byte accesses go to the banks in phases of 8 threads, 8-byte ones in
    phases of 16: each phase must touch distinct 16- (8-) byte bank slots."""
    run, pad, stage, gran, _ = geometry(B)
    for w in range(8):
        ths = list(range(32 * w, 32 * w + 32))
        for q in range(4):
            sub = ths[8 * q:8 * q + 8]
            assert len({(((t // gran) * pad + (t % gran) * 16) % 128) // 16 for t in sub}) == 8
        if B == 8:
            for q in range(4):
                sub = ths[8 * q:8 * q + 8]
                for g in range(8):
                    assert len({((t * pad + g * 16) % 128) // 16 for t in sub}) == 8
            reads = [lambda t, r: (t >> 4) * 16 * pad + (t & 15) * B + r * pad,
                     lambda t, r: (t >> 4) * pad + (t & 15) * B + r * 16 * pad]
            for h in range(2):
                sub = ths[16 * h:16 * h + 16]
                for r in range(16):
                    for f in reads:
                        assert len({(f(t, r) % 128) // 8 for t in sub}) == 16
        else:
            reads = [lambda t, r: t * pad + r * 16,
                     lambda t, r: (t >> 4) * 16 * pad + (t & 15) * B + r * pad,
                     lambda t, r: (t >> 4) * pad + (t & 15) * B + r * 16 * pad]
            for q in range(4):
                sub = ths[8 * q:8 * q + 8]
                for r in range(16):
                    for f in reads:
                        assert len({(f(t, r) % 128) // 16 for t in sub}) == 8


@pytest.mark.parametrize("n,high,grid", [(27, list(range(4, 12)), 304), (27, list(range(19, 27)), 304),
                                         (24, [4, 7, 9, 11, 13, 15, 17, 23], 152), (13, list(range(4, 12)), 152),
                                         (12, list(range(4, 12)), 304), (27, [5, 8, 11, 14, 17, 20, 23, 26], 304)])
def test_tile_base_masked_add(n, high, grid):
    nontile = ((1 << n) - 1) & ~0xF
    for q in high:
        nontile &= ~(1 << q)
    step = tile_expand(grid << 4, high)
    ntiles = 1 << (n - 12)
    for b in range(min(grid, ntiles)):
        nb, i = tile_expand(b << 4, high), 0
        while b + i * grid < ntiles:
            assert nb == tile_expand((b + i * grid) << 4, high)
            nb = ((nb | (~nontile & M64)) + step) & M64 & nontile
            i += 1


def pass_specs(n):
    """The tiled passes of the all-qubit Bloch sums for n >= 12 qubits, as the
    host side of csrc/k_reduce.cu plans them: 12 tile qubits (0..3 and 8 high
    ones), high qubit number i to pass i mod P, fillers from the lowest high
    qubits of other passes, and the mask of tile qubits the pass reports."""
    h = n - 4
    P = (h + 7) // 8
    specs = []
    for p in range(P):
        own = [4 + i for i in range(p, h, P)]
        high = list(own)
        q = 4
        while len(high) < 8:
            if q not in high:
                high.append(q)
            q += 1
        high.sort()
        wmask = (0xF if p == 0 else 0) | sum(1 << (4 + j) for j, q in enumerate(high) if q in own)
        specs.append(([0, 1, 2, 3] + high, wmask))
    return specs


def emulate_bloch_all(psi):
    """The kernel's sums in FP64, tile by tile: thread th of a tile holds its
    run (tile bits 0..3, tile bits 4..11 = th), then the slices with register
    bits = tile bits 4..7 and 8..11; S_j from the register pairs of the slice
    that holds tile bit j; Z sums of the high tile qubits from the threads'
    run totals."""
    n = int(np.log2(psi.size))
    out = np.zeros((n, 4))
    seen = np.zeros(n, dtype=int)
    for tq, wmask in pass_specs(n):
        rest = [q for q in range(n) if q not in tq]
        comb = np.zeros(1 + 3 * 12)
        for tid in range(1 << len(rest)):
            base = sum(((tid >> k) & 1) << q for k, q in enumerate(rest))
            tile = np.array([psi[base + sum(((e >> j) & 1) << tq[j] for j in range(12))] for e in range(4096)])
            runs = tile.reshape(256, 16)                       # [th][r]
            tot_th = (np.abs(runs) ** 2).sum(axis=1)
            comb[0] += tot_th.sum()
            for j in range(4):                                  # slice 1: own run, pairs in r bit j
                r0 = [r for r in range(16) if not (r >> j) & 1]
                x, y = runs[:, r0], runs[:, [r | (1 << j) for r in r0]]
                comb[1 + 3 * j] += (np.abs(y) ** 2).sum()
                s = (np.conj(x) * y).sum()
                comb[2 + 3 * j] += s.real
                comb[3 + 3 * j] += s.imag
            for b in range(8):                                  # Z of tile bit 4 + b from run totals
                comb[1 + 3 * (4 + b)] += tot_th[[th for th in range(256) if (th >> b) & 1]].sum()
            for j in range(4, 12):                              # slices 2 and 3: pairs in tile bit j
                e0 = [e for e in range(4096) if not (e >> j) & 1]
                s = (np.conj(tile[e0]) * tile[[e | (1 << j) for e in e0]]).sum()
                comb[2 + 3 * j] += s.real
                comb[3 + 3 * j] += s.imag
        for j in range(12):
            if (wmask >> j) & 1:
                q = tq[j]
                seen[q] += 1
                out[q] = [comb[0] - comb[1 + 3 * j], comb[1 + 3 * j], comb[2 + 3 * j], comb[3 + 3 * j]]
    assert (seen == 1).all()   # every qubit reported by exactly one pass
    return out


@pytest.mark.parametrize("n", [12, 13, 14])
def test_pass_plan_and_sums_match_the_oracle(n):
    """Every qubit is reported by one pass, and the sums the passes form give
    the oracle's Bloch vectors (r = (2 Re S, 2 Im S, p0 - p1) / (p0 + p1))."""
    import oracle
    rng = np.random.default_rng(n)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    sums = emulate_bloch_all(psi)
    for q in range(n):
        p0, p1, sr, si = sums[q]
        r = np.array([2 * sr, 2 * si, p0 - p1]) / (p0 + p1)
        assert np.max(np.abs(r - oracle.bloch(psi, q))) <= 1e-12, q


@pytest.mark.parametrize("n", [12, 13, 20, 27, 34])
def test_pass_plan_covers_every_qubit_once(n):
    specs = pass_specs(n)
    assert len(specs) == (n - 4 + 7) // 8
    rep = [q for tq, m in specs for j, q in enumerate(tq) if (m >> j) & 1]
    assert sorted(rep) == list(range(n))
    for tq, m in specs:
        assert len(set(tq)) == 12 and max(tq) < n
