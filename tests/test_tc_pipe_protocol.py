"""Barrier protocol of the pipelined tensor-core kernel (k_tc_pipe.cu),
modelled on the CPU with random interleavings of its roles.

The model follows the kernel's roles and mbarrier waits: the TMA producer
(load m into stage m mod S, signalling full[m mod B] after waiting for the
free barrier of the load the stage held before), the converters (complex64:
one group reading tile j; complex128 and complex64 with TF32 operands: four
quarter groups, quarter q of tile j is load 4j + q, plus the all-converter
barrier before the A operand is rewritten), the MMA issuer and the
write-back. A parity wait passes when the
barrier's current phase parity differs from the one waited for, as
mbarrier.try_wait.parity does. Every interleaving must read each load from
its stage after it landed and before the stage is reloaded, and finish.
With the stage ring's barriers shared between quarters (B = S = 3) the model
reproduces the race the per-quarter barriers remove. The model must be kept
in step with the kernel by hand."""
import random

import pytest


class Bar:
    def __init__(self, count):
        self.count = count
        self.pend = count
        self.tx = 0
        self.phase = 0

    def _check(self):
        assert self.pend >= 0 and self.tx >= 0, "barrier underflow"
        if self.pend == 0 and self.tx == 0:
            self.phase += 1
            self.pend = self.count

    def arrive(self):
        self.pend -= 1
        self._check()

    def expect_tx(self, b):
        self.tx += b
        self.pend -= 1
        self._check()

    def complete_tx(self, b):
        self.tx -= b
        self._check()

    def done(self, parity):
        return (self.phase & 1) != parity


def run(wide, J, pd, seed, nbar=None, nstage=None, lenient=None):
    """One random interleaving. lenient (a list) records stage violations
    (an early read, a stage reloaded or overwritten before it was read)
    instead of failing on them, so that the run goes on to show what the
    barriers do next; barrier underflow and deadlock still fail."""
    rng = random.Random(seed)

    def violation(kind, info):
        if lenient is None:
            raise AssertionError(kind, info)
        lenient.append(kind)
    NS, NB, Q = (3, 4, 4) if wide else (2, 2, 1)
    if nbar:
        NB = nbar
    if nstage:
        NS = nstage
    NG = 4 if wide else 1
    full = [Bar(2 if pd else 1) for _ in range(NB)]
    sfree = [Bar(1) for _ in range(NB)]       # a group's threads act as one arrival
    aready = [Bar(NG) for _ in range(2)]
    mma = [Bar(1) for _ in range(2)]
    accf = [Bar(1) for _ in range(2)]
    stage = [None] * NS                        # (load, landed)
    read = set()
    inflight = []
    acc = [None, None]
    abuf = {}
    written = []

    def producer():
        m = 0
        for j in range(J):
            for q in range(Q):
                s = m % NS
                if m >= NS:
                    r = m - NS
                    while not sfree[r % NB].done((r // NB) & 1):
                        yield
                    if r not in read:
                        violation("stage reloaded before it was read", (m, r))
                if not (stage[s] is None or stage[s][0] in read):
                    violation("stage overwritten", m)
                stage[s] = (m, False)
                full[m % NB].expect_tx(1)
                inflight.append((s, m, m % NB))
                if pd:
                    full[m % NB].arrive()
                m += 1
                yield

    def tma():
        while True:
            if inflight and rng.random() < 0.5:
                k = rng.randrange(len(inflight)) if rng.random() < 0.2 else 0
                s, m, b = inflight.pop(k)
                assert stage[s][0] == m
                stage[s] = (m, True)
                full[b].complete_tx(1)
            yield

    bar1 = {"cnt": 0, "gen": 0}

    def barrier_all(n):
        g = bar1["gen"]
        bar1["cnt"] += 1
        if bar1["cnt"] == n:
            bar1["cnt"] = 0
            bar1["gen"] += 1
        while bar1["gen"] == g:
            yield

    def converter(qi):
        for j in range(J):
            b = j & 1
            m = 4 * j + qi if wide else j
            while not full[m % NB].done((m // NB) & 1):
                yield
            if stage[m % NS] != (m, True):
                violation("read before the load landed", (j, qi, stage[m % NS], m))
            read.add(m)
            sfree[m % NB].arrive()
            yield
            if wide:
                if j >= 1:
                    while not mma[(j - 1) & 1].done(((j - 1) >> 1) & 1):
                        yield
                yield from barrier_all(NG)
                ab = 0
            else:
                if j >= 2:
                    while not mma[b].done(((j - 2) >> 1) & 1):
                        yield
                ab = b
            assert abuf.get((ab, qi), (-1, True))[1], "A operand rewritten before the MMAs read it"
            abuf[(ab, qi)] = (j, False)
            aready[ab].arrive()

    def mma_issuer():
        for j in range(J):
            b = j & 1
            ab = 0 if wide else b
            while not aready[ab].done((j & 1) if wide else ((j >> 1) & 1)):
                yield
            if j >= 2:
                while not accf[b].done(((j - 2) >> 1) & 1):
                    yield
            for qi in range(NG):
                assert abuf[(ab, qi)][0] == j, "MMA read another tile's A operand"
            assert acc[b] is None, "accumulator still being written back"
            acc[b] = j
            yield
            for qi in range(NG):
                abuf[(ab, qi)] = (j, True)
            mma[b].arrive()

    def write_back():
        for j in range(J):
            b = j & 1
            while not mma[b].done((j >> 1) & 1):
                yield
            assert acc[b] == j
            written.append(j)
            acc[b] = None
            accf[b].arrive()
            yield

    alive = [producer(), mma_issuer(), write_back()] + [converter(q) for q in range(NG)]
    t = tma()
    steps = 0
    while alive:
        steps += 1
        assert steps < 200000, "no progress (deadlock)"
        if rng.random() < 0.3:
            next(t)
        a = rng.choice(alive)
        try:
            next(a)
        except StopIteration:
            alive.remove(a)
    assert written == list(range(J)) and not inflight


@pytest.mark.parametrize("wide", [False, True])
@pytest.mark.parametrize("pd", [False, True])
def test_protocol_random_interleavings(wide, pd):
    for seed in range(600):
        run(wide, 1 + seed % 7, pd, seed)


@pytest.mark.parametrize("pd", [False, True])
def test_protocol_quarter_tiles_five_stages(pd):
    """Complex64 with TF32 operands: quarter tiles (as complex128) in a ring
    of five stages with eight barrier pairs (two per quarter, by tile
    parity), one A operand. With at least as many pairs as stages, issuing
    load m + B implies load m was read (the producer waited for its stage at
    load m + S), so no waiter can see a barrier complete twice."""
    for seed in range(600):
        run(True, 1 + seed % 7, pd, seed, nstage=5, nbar=8)


def test_shared_stage_barriers_underflow():
    """What the shared-barrier layout does after such an early read: some
    interleavings reload a stage whose load was never read and then complete
    a load's bytes on a barrier phase that has already completed (barrier
    underflow: an mbarrier over-arrived, undefined in PTX, with a bulk copy
    still writing the stage). The first complex128 runs of the kernel with
    that layout returned wrong amplitudes and then a launch failure."""
    found = False
    for seed in range(2000):
        rec = []
        try:
            run(True, 1 + seed % 7, False, seed, nbar=3, lenient=rec)
        except AssertionError as e:
            if str(e.args[0]).startswith("barrier underflow"):
                assert rec, "underflow without an earlier stage violation"
                found = True
                break
    assert found


def test_more_stages_than_barrier_pairs_fails():
    """Five stages on four barrier pairs: the producer's wait for load
    m - 5's stage can find the barrier already past load m - 1 as well (two
    completions, one parity), and loads can be issued onto a barrier whose
    previous phase has not completed: some interleaving deadlocks or
    underflows a barrier."""
    with pytest.raises(AssertionError, match="barrier underflow|deadlock|read before the load landed"):
        for seed in range(600):
            run(True, 1 + seed % 7, False, seed, nstage=5, nbar=4)


def test_shared_stage_barriers_race():
    """Quarters sharing the ring's barriers (three for four quarters): some
    interleaving reads a quarter before its load landed."""
    with pytest.raises(AssertionError, match="read before the load landed"):
        for seed in range(600):
            run(True, 1 + seed % 7, False, seed, nbar=3)


def run7(J, pd, seed, nstage=5, nbar=8, nslot_e=4):
    """One random interleaving of the 7-qubit kernel (k_tc_pipe7.cu): load m =
    8 j + e (eighth e of tile j) into stage m mod S after the free barrier of
    load m - S, signalling full[m mod B]; converter part p reads eighths p
    and p + 4 of each tile, and writes A chunk c once afree[c] shows that the
    MMAs of the previous tile's second half have read it; the MMA issuer
    takes output half h of tile j into slot h once the write-back has read
    slot h of tile j - 1 (accf[h]), waiting for aready[c] per chunk in the
    first half and arriving at afree[c] after each chunk of the second; the
    write-back reads slot 0, then slot 1. With deferred phases the producer
    writes tile j's factors into slot j mod 4 before its second arrival on
    full[0], and the converters of tile j read that slot."""
    rng = random.Random(seed)
    NS, NB = nstage, nbar
    full = [Bar(2 if pd else 1) for _ in range(NB)]
    sfree = [Bar(1) for _ in range(NB)]       # a part's four warps act as one arrival
    aready = [Bar(1) for _ in range(8)]
    afree = [Bar(1) for _ in range(8)]
    mma = [Bar(1) for _ in range(2)]
    accf = [Bar(1) for _ in range(2)]
    stage = [None] * NS
    read = set()
    inflight = []
    slot = [None, None]
    achunk = [None] * 8                        # (tile, read by both halves)
    sE = [None] * nslot_e
    written = []

    def producer():
        m = 0
        for j in range(J):
            for e in range(8):
                s = m % NS
                if m >= NS:
                    r = m - NS
                    while not sfree[r % NB].done((r // NB) & 1):
                        yield
                    assert r in read, ("stage reloaded before it was read", m, r)
                assert stage[s] is None or stage[s][0] in read, ("stage overwritten", m)
                stage[s] = (m, False)
                full[m % NB].expect_tx(1)
                inflight.append((s, m, m % NB))
                if pd:
                    if e == 0:
                        sE[j % nslot_e] = j
                    yield
                    full[m % NB].arrive()
                m += 1
                yield

    def tma():
        while True:
            if inflight and rng.random() < 0.5:
                k = rng.randrange(len(inflight)) if rng.random() < 0.2 else 0
                s, m, b = inflight.pop(k)
                assert stage[s][0] == m
                stage[s] = (m, True)
                full[b].complete_tx(1)
            yield

    def converter(p):
        for j in range(J):
            for hh in range(2):
                c = p + 4 * hh
                m = 8 * j + c
                while not full[m % NB].done((m // NB) & 1):
                    yield
                assert stage[m % NS] == (m, True), ("read before the load landed", j, c)
                if pd:
                    assert sE[j % nslot_e] == j, ("tile factors overwritten", j, c)
                read.add(m)
                sfree[m % NB].arrive()
                yield
                if j >= 1:
                    while not afree[c].done((j - 1) & 1):
                        yield
                assert achunk[c] is None or achunk[c] == (j - 1, True), ("A chunk rewritten before both halves read it",
                                                                         j, c, achunk[c])
                achunk[c] = (j, False)
                yield
                aready[c].arrive()

    def mma_issuer():
        for j in range(J):
            for h in range(2):
                if j >= 1:
                    while not accf[h].done((j - 1) & 1):
                        yield
                assert slot[h] is None, "slot still being written back"
                for c in range(8):
                    if h == 0:
                        while not aready[c].done(j & 1):
                            yield
                    assert achunk[c] == (j, False), ("MMA read another tile's A chunk", j, h, c, achunk[c])
                    yield
                    if h == 1:
                        achunk[c] = (j, True)
                        afree[c].arrive()
                slot[h] = j
                mma[h].arrive()

    def write_back():
        for j in range(J):
            for h in range(2):
                while not mma[h].done(j & 1):
                    yield
                assert slot[h] == j
                yield
                slot[h] = None
                written.append((j, h))
                accf[h].arrive()

    alive = [producer(), mma_issuer(), write_back()] + [converter(p) for p in range(4)]
    t = tma()
    steps = 0
    while alive:
        steps += 1
        assert steps < 400000, "no progress (deadlock)"
        if rng.random() < 0.3:
            next(t)
        a = rng.choice(alive)
        try:
            next(a)
        except StopIteration:
            alive.remove(a)
    assert written == [(j, h) for j in range(J) for h in range(2)] and not inflight


@pytest.mark.parametrize("pd", [False, True])
def test_protocol7_random_interleavings(pd):
    """The 7-qubit kernel's protocol: five stages on eight barrier pairs (one
    per eighth), per-chunk A barriers and two output slots."""
    for seed in range(500):
        run7(1 + seed % 6, pd, seed)


def test_protocol7_needs_a_pair_per_eighth():
    """With fewer barrier pairs than stages (five stages, four pairs) some
    interleaving of the 7-qubit kernel's ring fails."""
    with pytest.raises(AssertionError):
        for seed in range(500):
            run7(1 + seed % 6, False, seed, nbar=4)


def run_tf_split(J, pd, seed, shared_lo=False):
    """The 3xTF32 variant's A handshake in two halves: the MMA issuer takes
    a_lo u_hi first and commits (lo free), then a_hi u_hi and a_hi u_lo and
    commits (the whole tile done); the converters (one group: the quarters
    are read as in `run`, the A stores follow an all-converter barrier) write
    tile j's lo parts once tile j - 1's lo product is done and signal lo
    ready, then its hi parts once tile j - 1's MMAs are done and signal hi
    ready; the MMA waits lo ready before the lo product and hi ready before
    the others. shared_lo: the lo parts wait only for the whole previous
    tile (the one-handshake layout)."""
    rng = random.Random(seed)
    lofree, loready, hiready = Bar(1), Bar(1), Bar(1)
    mma = [Bar(1) for _ in range(2)]
    accf = [Bar(1) for _ in range(2)]
    a_lo = [None, True]       # (tile, read) of the one A operand's lo and hi regions
    a_hi = [None, True]
    acc = [None, None]
    written = []
    state = {"lo_read": -1, "hi_read": -1}

    def converters():
        for j in range(J):
            yield                                        # quarters read, phases, split
            if j >= 1:
                if shared_lo:
                    while not mma[(j - 1) & 1].done(((j - 1) >> 1) & 1):
                        yield
                else:
                    while not lofree.done((j - 1) & 1):
                        yield
            assert state["lo_read"] == j - 1, ("lo rewritten before the MMAs read it", j)
            a_lo[0] = j
            yield
            loready.arrive()
            if j >= 1:
                while not mma[(j - 1) & 1].done(((j - 1) >> 1) & 1):
                    yield
            assert state["hi_read"] == j - 1, ("hi rewritten before the MMAs read it", j)
            a_hi[0] = j
            yield
            hiready.arrive()

    def mma_issuer():
        for j in range(J):
            b = j & 1
            if j >= 2:
                while not accf[b].done(((j - 2) >> 1) & 1):
                    yield
            assert acc[b] is None, "accumulator still being written back"
            while not loready.done(j & 1):
                yield
            assert a_lo[0] == j, ("lo product read another tile's lo parts", j)
            yield
            state["lo_read"] = j
            lofree.arrive()
            while not hiready.done(j & 1):
                yield
            assert a_hi[0] == j, ("hi products read another tile's hi parts", j)
            yield
            state["hi_read"] = j
            acc[b] = j
            mma[b].arrive()

    def write_back():
        for j in range(J):
            b = j & 1
            while not mma[b].done((j >> 1) & 1):
                yield
            assert acc[b] == j
            yield
            acc[b] = None
            written.append(j)
            accf[b].arrive()

    alive = [converters(), mma_issuer(), write_back()]
    steps = 0
    while alive:
        steps += 1
        assert steps < 200000, "no progress (deadlock)"
        a = rng.choice(alive)
        try:
            next(a)
        except StopIteration:
            alive.remove(a)
    assert written == list(range(J))


@pytest.mark.parametrize("shared_lo", [False, True])
def test_protocol_tf32_lo_hi_handshake(shared_lo):
    """The two-half A handshake of the 3xTF32 variant: every interleaving
    writes each half of the one A operand only after the MMAs that read its
    previous contents are done, and finishes."""
    for seed in range(800):
        run_tf_split(1 + seed % 9, False, seed, shared_lo=shared_lo)
