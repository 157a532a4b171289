"""Exclusive-carry full adder (circuit variant, not the paper's): the carry of
FA = HA, HA, carry is the sum of the two half-adder carries, which are never
both 1 (Lemma 6's OR agrees with it on every input it meets). As a GSW gate it
is linear, (0, 1, 1, 0), with no ciphertext product, and its noise adds.

Pins: truth tables and the closed forms of every word operation (exhaustive at
F = 4, random wider), the FFT circuit against the integer FFT, encrypted
evaluation decrypting to the plaintext circuit with the exact noise inside the
static bound, the static bound never above the paper circuit's, and the native
compiler's program (levels with linear phases, slots, fix-ups) against the
oracle's independent construction.
"""
import itertools
import math
import random

import numpy as np
import pytest

from oracle import circuit, evaluate, fixedpoint as fx, gsw, noise


def _eval_words(c, xs, F):
    bits = []
    for x in xs:
        bits += fx.to_bits(x, F)
    return fx.from_bits(evaluate.eval_plain(c, bits))


def test_full_adder_exhaustive_and_carries_exclusive():
    c = circuit.Circuit(xcarry=True)
    a, b, d = c.new_input(), c.new_input(), c.new_input()
    s, cy = c.FA(a, b, d)
    c.outputs = [s, cy]
    assert [g[0] for g in c.gates].count("XADD") == 1
    for x, y, z in itertools.product((0, 1), repeat=3):
        out = evaluate.eval_plain(c, [x, y, z])    # XADD raises on two set bits
        assert out[0] + 2 * out[1] == x + y + z


def test_xadd_folding_and_depth():
    c = circuit.Circuit(xcarry=True)
    x, y = c.new_input(), c.new_input()
    Z, O = circuit.ZERO, circuit.ONE
    assert c.XADD(x, Z) == x and c.XADD(Z, x) == x and c.XADD(O, x) == O
    s, k = c.HA(x, y)
    w = c.XADD(k, x)
    assert c.gates[-1][0] == "XADD" and c.depth[w] == max(c.depth[k], c.depth[x])


@pytest.mark.parametrize("kind", ["add", "sub"])
def test_add_sub_exhaustive_f4(kind):
    F = 4
    c = circuit.word_circuit(kind, F, xcarry=True)
    for x, y in itertools.product(range(-8, 8), repeat=2):
        want = fx.wrap(x + y if kind == "add" else x - y, F)
        assert _eval_words(c, [x, y], F) == want, (x, y)


@pytest.mark.parametrize("f", [0, 1, 2, 3])
def test_mul_exhaustive_f4(f):
    F = 4
    for w in range(-8, 8):
        c = circuit.word_circuit("mul", F, f, w, xcarry=True)
        for x in range(-8, 8):
            assert _eval_words(c, [x, 0], F) == fx.wrap(math.floor(x * w / 2 ** f), F), (x, w, f)


def test_word_ops_random_16bit():
    F, f = 16, 8
    rng = random.Random(77)
    lo, hi = -(1 << (F - 1)), (1 << (F - 1)) - 1
    add, sub = circuit.word_circuit("add", F, xcarry=True), circuit.word_circuit("sub", F, xcarry=True)
    for _ in range(30):
        x, y = rng.randint(lo, hi), rng.randint(lo, hi)
        assert _eval_words(add, [x, y], F) == fx.wrap(x + y, F)
        assert _eval_words(sub, [x, y], F) == fx.wrap(x - y, F)
    for _ in range(4):
        w = rng.randint(-(1 << f), 1 << f)
        mul = circuit.word_circuit("mul", F, f, w, xcarry=True)
        for _ in range(5):
            x = rng.randint(lo, hi)
            assert _eval_words(mul, [x, 0], F) == fx.wrap(math.floor(x * w / 2 ** f), F)


@pytest.mark.parametrize("N1,N2,F,f", [(8, 1, 8, 4), (4, 4, 8, 3)])
def test_fft_circuit_equals_integer_fft(N1, N2, F, f):
    c = circuit.fft_circuit(N1, N2, F, f, xcarry=True)
    rng = random.Random(N1 * 5 + N2)
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


def test_fewer_products_and_never_more_noise():
    N, F, f = 8, 8, 4
    paper = circuit.fft_circuit(N, 1, F, f)
    var = circuit.fft_circuit(N, 1, F, f, xcarry=True)
    sp, sv = circuit.stats(paper), circuit.stats(var)
    # every OR becomes an XADD, every other gate is unchanged; the products
    # drop by the distinct OR products (identical ORs shared one product)
    assert sv["XADD"] == sp["OR"] and sv["OR"] == 0
    assert all(sv[k] == sp[k] for k in ("AND", "XOR", "NOT"))
    assert sv["products"] < sp["products"]
    for ell in (160, 224):
        p = gsw.Params(1, ell, 2 * ell, 1)
        assert noise.max_bound(var, p) <= noise.max_bound(paper, p)
    assert noise.smallest_ell(var, 1, 1) < noise.smallest_ell(paper, 1, 1)


def test_encrypted_fft_noisy_leveled_parameters():
    N, F, f = 2, 4, 1
    c = circuit.fft_circuit(N, 1, F, f, xcarry=True)
    ell = noise.smallest_ell(c, n=1, chi=1)
    p = gsw.Params(1, ell, 2 * ell, 1)
    bounds = noise.wire_bounds(c, p)
    keys = gsw.Keys(p, seed=8)
    re, im = [5, -3], [1, -6]
    cts, bits = [], []
    for k, (r, i) in enumerate(zip(re, im)):
        for part, v in enumerate((r, i)):
            for b, bit in enumerate(fx.to_bits(v, F)):
                cts.append(gsw.encrypt(keys, bit, 2, (k * 2 + part) * F + b))
                bits.append(bit)
    out = evaluate.eval_encrypted(c, p, cts)
    plain = evaluate.eval_plain(c, bits)
    assert [gsw.decrypt(keys, ct) for ct in out] == plain
    for w, ct, mu in zip(c.outputs, out, plain):
        assert max(map(abs, gsw.noise(keys, ct, mu))) <= bounds[w]
    words = [fx.from_bits(plain[k * F:(k + 1) * F]) for k in range(2 * N)]
    assert (words[0::2], words[1::2]) == fx.fft_int(re, im, F, f)


@pytest.mark.parametrize("N1,N2,F,f", [(8, 1, 8, 4), (4, 4, 8, 3), (16, 1, 8, 4)])
def test_native_program_matches_oracle(N1, N2, F, f):
    import paper_1611_08769_gb300 as sf
    sp = sf.param_set("P0")
    c = circuit.fft_circuit(N1, N2, F, f, xcarry=True)
    info = sf.circuit_info(sp, N1, N2, F, f, xcarry=True)
    assert info["products"] == circuit.stats(c)["products"]
    assert sf.min_ell(N1, N2, F, f, 1, 1, xcarry=True) == noise.smallest_ell(c, 1, 1)
    rng = random.Random(N1 * 3 + F)
    for _ in range(4):
        bits = [rng.randint(0, 1) for _ in range(len(c.inputs))]
        got = sf.program_eval_plain(sp, N1, N2, F, f, np.array(bits, np.uint8), xcarry=True)
        assert list(got) == evaluate.eval_plain(c, bits)
