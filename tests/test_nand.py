"""NAND-only circuit (the paper's literal construction): Lemma 4 builds NOT,
AND, OR and XOR from the scheme's NAND gate, and Sec. 7 counts the FFT's
arithmetic in NAND gates (36 F per fixed-point addition, 288 F^2 log F per
fixed-point multiplication, the latter a stated worst case). Every gate that
survives constant folding is a GSW NAND (1, 0, 0, -1), one ciphertext product
each; there are no complement bits and no linear gates.

Pins: the NAND truth table and the code's plaintext identity; each composed
gate exhaustively; the closed forms of every word operation (exhaustive at
F = 4, random at 16 bits); the FFT circuit against the integer FFT; the gate
counts against Sec. 7's bounds and against hand counts of the composition;
encrypted evaluation decrypting to the plaintext circuit with the exact noise
inside the static bound; and the native compiler against the oracle's
independent construction.
"""
import itertools
import math
import random

import numpy as np
import pytest

from oracle import circuit, evaluate, fixedpoint as fx, gsw, noise
from oracle.circuit import ONE, ZERO


def _eval_words(c, xs, F):
    bits = []
    for x in xs:
        bits += fx.to_bits(x, F)
    return fx.from_bits(evaluate.eval_plain(c, bits))


def _ops(c):
    return {g[0] for g in c.gates}


def test_nand_code_is_the_nand_identity():
    c0, c1, c2, c3 = gsw.GATE_CODES["NAND"]
    for a, b in itertools.product((0, 1), repeat=2):
        assert c0 + c1 * a + c2 * b + c3 * a * b == 1 - (a & b) == evaluate.TRUTH["NAND"](a, b)


@pytest.mark.parametrize("gate,fn,nands", [
    ("NOT", lambda a, b: 1 - a, 1),
    ("AND", lambda a, b: a & b, 2),
    ("OR", lambda a, b: a | b, 3),
    ("XOR", lambda a, b: a ^ b, 4),
])
def test_composed_gates_exhaustive(gate, fn, nands):
    c = circuit.Circuit(nand=True)
    a, b = c.new_input(), c.new_input()
    out = c.NOT(a) if gate == "NOT" else getattr(c, gate)(a, b)
    c.outputs = [out]
    assert _ops(c) == {"NAND"} and len(c.gates) == nands
    for x, y in itertools.product((0, 1), repeat=2):
        assert evaluate.eval_plain(c, [x, y]) == [fn(x, y)]


def test_half_and_full_adder_exhaustive():
    c = circuit.Circuit(nand=True)
    a, b, d = c.new_input(), c.new_input(), c.new_input()
    s, k = c.HA(a, b)
    assert len(c.gates) == 5           # t shared by the XOR and the AND
    s3, k3 = c.FA(a, b, d)
    assert len(c.gates) == 5 + 13      # two half adders and a three-gate OR
    c.outputs = [s, k, s3, k3]
    assert _ops(c) == {"NAND"}
    for x, y, z in itertools.product((0, 1), repeat=3):
        o = evaluate.eval_plain(c, [x, y, z])
        assert o[0] + 2 * o[1] == x + y and o[2] + 2 * o[3] == x + y + z


def test_constants_fold_before_decomposition():
    c = circuit.Circuit(nand=True)
    x = c.new_input()
    assert c.AND(x, ONE) == x and c.AND(ZERO, x) == ZERO and c.OR(x, ZERO) == x
    assert c.OR(ONE, x) == ONE and c.XOR(ZERO, x) == x and c.NOT(ONE) == ZERO
    assert c.HA(x, ZERO) == (x, ZERO) and not c.gates
    nx = c.XOR(x, ONE)                 # XOR with 1 is a NOT: NAND(x, x)
    assert c.gates == [("NAND", x, x, nx)]


def test_variants_are_exclusive():
    with pytest.raises(ValueError):
        circuit.Circuit(xcarry=True, nand=True)


@pytest.mark.parametrize("kind", ["add", "sub"])
def test_add_sub_exhaustive_f4(kind):
    F = 4
    c = circuit.word_circuit(kind, F, nand=True)
    assert _ops(c) == {"NAND"}
    for x, y in itertools.product(range(-8, 8), repeat=2):
        want = fx.wrap(x + y if kind == "add" else x - y, F)
        assert _eval_words(c, [x, y], F) == want, (x, y)


@pytest.mark.parametrize("f", [0, 1, 2, 3])
def test_mul_exhaustive_f4(f):
    F = 4
    for w in range(-8, 8):
        c = circuit.word_circuit("mul", F, f, w, nand=True)
        for x in range(-8, 8):
            assert _eval_words(c, [x, 0], F) == fx.wrap(math.floor(x * w / 2 ** f), F), (x, w, f)


def test_word_ops_random_16bit():
    F, f = 16, 8
    rng = random.Random(78)
    lo, hi = -(1 << (F - 1)), (1 << (F - 1)) - 1
    add, sub = circuit.word_circuit("add", F, nand=True), circuit.word_circuit("sub", F, nand=True)
    for _ in range(30):
        x, y = rng.randint(lo, hi), rng.randint(lo, hi)
        assert _eval_words(add, [x, y], F) == fx.wrap(x + y, F)
        assert _eval_words(sub, [x, y], F) == fx.wrap(x - y, F)
    for _ in range(3):
        w = rng.randint(-(1 << f), 1 << f)
        mul = circuit.word_circuit("mul", F, f, w, nand=True)
        for _ in range(4):
            x = rng.randint(lo, hi)
            assert _eval_words(mul, [x, 0], F) == fx.wrap(math.floor(x * w / 2 ** f), F)


@pytest.mark.parametrize("F", [4, 8, 16])
def test_gate_counts_within_section7_bounds(F):
    # ripple adder: a half adder (5) then F - 1 full adders (13), the final
    # carry pruned: 13 F - 13 after the dead last OR is removed; Sec. 7 bounds
    # it by 36 F
    add = circuit.stats(circuit.word_circuit("add", F, nand=True))
    assert add["NAND"] == add["products"] == 13 * F - 13 <= 36 * F
    # constant multiplication, worst plaintext over a sample: Sec. 7's
    # 288 F^2 log F is a loose worst case
    rng = random.Random(F)
    ws = [-(1 << (F - 1)), (1 << (F - 1)) - 1, -1] + [rng.randint(-(1 << (F - 1)), (1 << (F - 1)) - 1)
                                                       for _ in range(3)]
    worst = max(circuit.stats(circuit.word_circuit("mul", F, F // 2, w, nand=True))["NAND"] for w in ws)
    assert 0 < worst <= 288 * F * F * math.log2(F)


def test_products_and_noise_against_the_arithmetised_circuit():
    N, F, f = 8, 8, 4
    paper = circuit.stats(circuit.fft_circuit(N, 1, F, f))
    c = circuit.fft_circuit(N, 1, F, f, nand=True)
    st = circuit.stats(c)
    assert st["NOT"] == st["AND"] == st["XOR"] == st["OR"] == st["XADD"] == 0
    # every logical gate costs at least one NAND product
    assert st["products"] > paper["products"] and st["depth"] > paper["depth"]
    assert noise.smallest_ell(c, 1, 1) > noise.smallest_ell(circuit.fft_circuit(N, 1, F, f), 1, 1)


@pytest.mark.parametrize("N1,N2,F,f", [(8, 1, 8, 4), (4, 4, 8, 3)])
def test_fft_circuit_equals_integer_fft(N1, N2, F, f):
    c = circuit.fft_circuit(N1, N2, F, f, nand=True)
    rng = random.Random(N1 * 7 + N2)
    lo, hi = -(1 << (F - 2)), (1 << (F - 2)) - 1
    re = [rng.randint(lo, hi) for _ in range(N1 * N2)]
    im = [rng.randint(lo, hi) for _ in range(N1 * N2)]
    bits = []
    for r, i in zip(re, im):
        bits += fx.to_bits(r, F) + fx.to_bits(i, F)
    out = evaluate.eval_plain(c, bits)
    words = [fx.from_bits(out[k * F:(k + 1) * F]) for k in range(2 * N1 * N2)]
    want = fx.fft_int(re, im, F, f) if N2 == 1 else fx.fft2_int(re, im, N1, N2, F, f)
    assert (words[0::2], words[1::2]) == tuple(want)


def test_encrypted_fft_noisy_leveled_parameters():
    N, F, f = 2, 4, 1
    c = circuit.fft_circuit(N, 1, F, f, nand=True)
    ell = noise.smallest_ell(c, n=1, chi=1)
    p = gsw.Params(1, ell, 2 * ell, 1)
    bounds = noise.wire_bounds(c, p)
    keys = gsw.Keys(p, seed=9)
    re, im = [6, -4], [-2, 7]
    cts, bits = [], []
    for k, (r, i) in enumerate(zip(re, im)):
        for part, v in enumerate((r, i)):
            for b, bit in enumerate(fx.to_bits(v, F)):
                cts.append(gsw.encrypt(keys, bit, 3, (k * 2 + part) * F + b))
                bits.append(bit)
    out = evaluate.eval_encrypted(c, p, cts)
    plain = evaluate.eval_plain(c, bits)
    assert [gsw.decrypt(keys, ct) for ct in out] == plain
    for w, ct, mu in zip(c.outputs, out, plain):
        assert max(map(abs, gsw.noise(keys, ct, mu))) <= bounds[w]
    words = [fx.from_bits(plain[k * F:(k + 1) * F]) for k in range(2 * N)]
    assert (words[0::2], words[1::2]) == fx.fft_int(re, im, F, f)


@pytest.mark.parametrize("N1,N2,F,f", [(2, 1, 4, 1), (8, 1, 8, 4), (4, 4, 8, 3)])
def test_native_program_matches_oracle(N1, N2, F, f):
    import paper_1611_08769_gb300 as sf
    sp = sf.param_set("P0")
    c = circuit.fft_circuit(N1, N2, F, f, nand=True)
    st = circuit.stats(c)
    info = sf.circuit_info(sp, N1, N2, F, f, nand=True)
    assert info["products"] == st["products"] and info["levels"] == st["depth"]
    assert info["gates_xadd"] == 0
    assert sf.min_ell(N1, N2, F, f, 1, 1, nand=True) == noise.smallest_ell(c, 1, 1)
    rng = random.Random(N1 * 5 + F)
    for _ in range(3):
        bits = [rng.randint(0, 1) for _ in range(len(c.inputs))]
        got = sf.program_eval_plain(sp, N1, N2, F, f, np.array(bits, np.uint8), nand=True)
        assert list(got) == evaluate.eval_plain(c, bits)


def test_native_rejects_both_variants():
    import paper_1611_08769_gb300 as sf
    assert sf.min_ell(8, 1, 8, 4, 1, 1, xcarry=True, nand=True) == 0
    with pytest.raises(sf.SfftError):
        sf.circuit_info(sf.param_set("P0"), 8, 1, 8, 4, xcarry=True, nand=True)
