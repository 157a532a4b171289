"""Host logic of the persistent batch form (one launch across all levels), on
the CPU: the producer indices the compiler hands the launch, the scratch-slot
reuse window, and every evaluation order the launch's rules allow.

The launch runs gate g once the gates that last wrote its two operands have
run and every gate two levels above g's level has run (Sec. 7: the gates of a
level are independent; here neighbouring levels also overlap). Programs
compiled for it reuse a scratch slot only two levels after its last read.
The tests model both orders on the compiled program's own listing
(`sfft_program_gates`) and compare what every operand read sees.
"""
import heapq

import numpy as np
import pytest

import paper_1611_08769_gb300 as sf
from oracle import circuit, evaluate
from paper_1611_08769_gb300 import build as sfbuild

NONE = 0xFFFFFFFF
SHAPES = [(8, 1, 8, 4), (16, 1, 16, 8), (4, 4, 8, 4)]


@pytest.fixture(scope="module", autouse=True)
def built():
    sfbuild.build()


def _levels(gates):
    """[start, end) of each level in program order."""
    lev = gates["level"]
    cuts = np.flatnonzero(np.diff(lev)) + 1
    edges = np.concatenate(([0], cuts, [len(gates)]))
    return list(zip(edges[:-1], edges[1:]))


def sequential_reads(gates):
    """Level by level, a level's reads before its writes: for every gate, the
    gate whose write each operand read sees (-1: never written, an input)."""
    ver, seen = {}, np.full((len(gates), 2), -1, np.int64)
    for s, e in _levels(gates):
        for g in range(s, e):
            seen[g, 0] = ver.get(int(gates["a"][g]), -1)
            seen[g, 1] = ver.get(int(gates["b"][g]), -1)
        for g in range(s, e):
            for o in (gates["o0"][g], gates["o1"][g]):
                if o != NONE:
                    ver[int(o)] = g
    return seen


def persistent_reads(gates, deps, seed):
    """An order the persistent launch allows, as hostile as its rules permit:
    always the deepest ready gate next (random among equals). A gate is ready
    once its producers `deps` ran and every gate two levels up ran. Returns
    what each read sees, as sequential_reads."""
    rng = np.random.default_rng(seed)
    n = len(gates)
    lev = gates["level"].astype(np.int64)
    nlev = int(lev.max()) + 1
    left = np.bincount(lev, minlength=nlev)
    consumers = [[] for _ in range(n)]
    unmet = np.zeros(n, np.int64)
    for g in range(n):
        for d in {int(x) for x in deps[g] if x >= 0}:
            consumers[d].append(g)
            unmet[g] += 1
    parked = [[] for _ in range(nlev)]
    heap = []

    def offer(g):
        if lev[g] < 2 or left[lev[g] - 2] == 0:
            heapq.heappush(heap, (-lev[g], rng.random(), g))
        else:
            parked[lev[g]].append(g)

    for g in range(n):
        if unmet[g] == 0:
            offer(g)
    ver, seen, ran = {}, np.full((n, 2), -1, np.int64), 0
    while heap:
        g = heapq.heappop(heap)[2]
        seen[g, 0] = ver.get(int(gates["a"][g]), -1)
        seen[g, 1] = ver.get(int(gates["b"][g]), -1)
        for o in (gates["o0"][g], gates["o1"][g]):
            if o != NONE:
                ver[int(o)] = g
        ran += 1
        left[lev[g]] -= 1
        if left[lev[g]] == 0 and lev[g] + 2 < nlev:
            for p in parked[lev[g] + 2]:
                heapq.heappush(heap, (-lev[p], rng.random(), p))
            parked[lev[g] + 2] = []
        for c in consumers[g]:
            unmet[c] -= 1
            if unmet[c] == 0:
                offer(c)
    assert ran == n, "the persistent rules left gates that can never run"
    return seen


def reuse_distances(gates):
    """For every write to a slot that held an earlier value: its level minus
    the level of the earlier value's last read."""
    last_read, written, dist = {}, set(), []
    for s, e in _levels(gates):
        lvl = int(gates["level"][s])
        for g in range(s, e):
            for r in (gates["a"][g], gates["b"][g]):
                last_read[int(r)] = lvl
        for g in range(s, e):
            for o in (gates["o0"][g], gates["o1"][g]):
                if o == NONE:
                    continue
                o = int(o)
                if o in written and o in last_read:
                    dist.append(lvl - last_read[o])
                written.add(o)
                last_read.pop(o, None)
    return np.array(dist)


def _nib(code, k):
    v = (int(code) >> (4 * k)) & 15
    return v - 16 if v & 8 else v


def plain_outputs(gates, in_bits, n_out):
    """The listing evaluated on bits in program order (out = c0 + c1 a + c2 b
    + c3 A~ b, A~ = 1 - a when complemented): output slot -> bit."""
    reg = {(1 << 30) | i: int(b) for i, b in enumerate(in_bits)}
    for s, e in _levels(gates):
        vals = []
        for g in range(s, e):
            a, b = reg[int(gates["a"][g])], reg[int(gates["b"][g])]
            at = 1 - a if gates["flags"][g] & 1 else a
            for h, o in enumerate((gates["o0"][g], gates["o1"][g])):
                if o != NONE:
                    c = int(gates["code"][g]) >> (16 * h)
                    v = _nib(c, 0) + _nib(c, 1) * a + _nib(c, 2) * b + _nib(c, 3) * at * b
                    assert v in (0, 1)
                    vals.append((int(o), v))
        reg.update(vals)
    return {i: reg[(2 << 30) | i] for i in range(n_out) if (2 << 30) | i in reg}


@pytest.mark.parametrize("N1,N2,F,f", SHAPES)
def test_producers_are_the_last_writers(N1, N2, F, f):
    gates = sf.program_gates(sf.param_set("P2"), N1, N2, F, f, sf.BATCH_PERSISTENT)
    seen = sequential_reads(gates)
    for k, name in enumerate(("dep_a", "dep_b")):
        want = np.where(seen[:, k] < 0, NONE, seen[:, k]).astype(np.uint32)
        assert np.array_equal(gates[name], want), name
    # every producer sits at a lower level
    for name in ("dep_a", "dep_b"):
        d = gates[name]
        m = d != NONE
        assert (gates["level"][d[m]] < gates["level"][m]).all()


@pytest.mark.parametrize("N1,N2,F,f", SHAPES)
def test_slots_are_reused_two_levels_after_their_last_read(N1, N2, F, f):
    p = sf.param_set("P2")
    d2 = reuse_distances(sf.program_gates(p, N1, N2, F, f, sf.BATCH_PERSISTENT))
    d1 = reuse_distances(sf.program_gates(p, N1, N2, F, f))
    assert len(d2) and d2.min() >= 2
    assert len(d1) and d1.min() == 1   # the level-by-level form reuses at once


@pytest.mark.parametrize("N1,N2,F,f", SHAPES)
def test_every_allowed_order_reads_what_level_order_reads(N1, N2, F, f):
    gates = sf.program_gates(sf.param_set("P2"), N1, N2, F, f, sf.BATCH_PERSISTENT)
    seen = sequential_reads(gates)
    for seed in range(3):
        assert np.array_equal(persistent_reads(gates, seen, seed), seen), seed


def test_the_window_alone_does_not_protect_immediate_reuse():
    """The same rules on a program that reuses slots at once (the level-by-
    level compilation): some read sees a later write. This is what the
    two-level reuse gap of the persistent compilation prevents."""
    gates = sf.program_gates(sf.param_set("P2"), 16, 1, 16, 8)
    seen = sequential_reads(gates)
    assert any(not np.array_equal(persistent_reads(gates, seen, s), seen) for s in range(3))


@pytest.mark.parametrize("N1,N2,F,f", SHAPES[:2])
def test_persistent_listing_computes_the_circuit(N1, N2, F, f):
    """The listing compiled for the persistent form, run on random bits,
    gives the oracle circuit's outputs (those written by gates)."""
    gates = sf.program_gates(sf.param_set("P2"), N1, N2, F, f, sf.BATCH_PERSISTENT)
    c = circuit.fft_circuit(N1, N2, F, f)
    bits = np.random.default_rng(N1 * 100 + F).integers(0, 2, len(c.inputs))
    want = evaluate.eval_plain(c, [int(b) for b in bits])
    got = plain_outputs(gates, bits, len(want))
    assert len(got) > 0.9 * len(want)
    assert all(got[i] == want[i] for i in got)


def test_listing_rejects_bad_arguments():
    import ctypes
    p = sf.param_set("P2")
    n = ctypes.c_uint64(0)
    lib = sf.lib()
    assert lib.sfft_program_gates(ctypes.byref(p), 8, 1, 8, 4, 0, None, 0, None) != 0   # no count
    assert lib.sfft_program_gates(ctypes.byref(p), 8, 1, 8, 4, 0, None, 0, ctypes.byref(n)) == 0
    buf = np.zeros(n.value - 1, dtype=sf.GATE_RECORD)
    assert lib.sfft_program_gates(ctypes.byref(p), 8, 1, 8, 4, 0, ctypes.c_void_p(buf.ctypes.data),
                                  n.value - 1, ctypes.byref(n)) != 0                      # short buffer
    with pytest.raises(sf.SfftError):   # linear (exclusive-carry) gates have no persistent schedule
        sf.program_gates(p, 8, 1, 8, 4, sf.BATCH_PERSISTENT | sf.PLAN_XCARRY)
    with pytest.raises(sf.SfftError):   # not a power-of-two FFT
        sf.program_gates(p, 6, 1, 8, 4)
