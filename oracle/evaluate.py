"""Plaintext and encrypted evaluation of a circuit (oracle side).

Plaintext evaluation applies the Boolean truth function of each gate.
Encrypted evaluation applies the compressed GSW gate to ciphertexts, with
the bit-decomposed operand chosen by the depth rule of ``circuit``.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
import numpy as np

from . import gsw
from .circuit import ZERO, ONE

TRUTH = {
    "NOT": lambda a, b: 1 - a,
    "AND": lambda a, b: a & b,
    "XOR": lambda a, b: a ^ b,
    "OR": lambda a, b: a | b,
    "XADD": lambda a, b: _exclusive_sum(a, b),
    "NAND": lambda a, b: 1 - (a & b),
    "SEL1": lambda a, b: a,
    "SEL0": lambda a, b: 0,
}


def _exclusive_sum(a, b):
    if a & b:
        raise AssertionError("XADD applied to two set bits")
    return a + b


def eval_plain(c, in_bits):
    """Values of c.outputs for 0/1 input bits (one per input wire)."""
    val = [None] * len(c.depth)
    for w, bit in zip(c.inputs, in_bits):
        val[w] = int(bit)

    def get(w):
        return 0 if w == ZERO else 1 if w == ONE else val[w]

    for op, a, b, o in c.gates:
        val[o] = TRUTH[op](get(a), None if b is None else get(b))
    return [get(w) for w in c.outputs]


def operands(c, a, b):
    """(A, B): A is the deeper operand, ties keep the first argument."""
    if b is not None and c.d(b) > c.d(a):
        return b, a
    return a, b


def eval_encrypted(c, p, in_cts, keep=None):
    """Ciphertexts of c.outputs given input ciphertexts (list or array).

    Wires are released after their last use so that long circuits fit in
    memory. ``keep`` (optional set of wires) are kept and returned as a dict.
    """
    last = {}
    for idx, (op, a, b, o) in enumerate(c.gates):
        last[a] = idx
        if b is not None:
            last[b] = idx
    outs = set(w for w in c.outputs if w >= 0)
    keep = set(keep or ())
    val = {}
    for w, ct in zip(c.inputs, in_cts):
        val[w] = ct
    zero, one = gsw.zero_ct(p), gsw.one_ct(p)

    def get(w):
        return zero if w == ZERO else one if w == ONE else val[w]

    for idx, (op, a, b, o) in enumerate(c.gates):
        A, B = operands(c, a, b)
        val[o] = gsw.gate(p, get(A), None if B is None else get(B), gsw.GATE_CODES[op])
        for w in (a, b):
            if w is not None and w >= 0 and last.get(w) == idx and w not in outs and w not in keep:
                val.pop(w, None)
    result = np.stack([get(w) for w in c.outputs]) if c.outputs else None
    if keep:
        return result, {w: val[w] for w in keep if w in val}
    return result
