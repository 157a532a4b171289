"""Encrypted-operand multiplier (a variant: the paper multiplies by plaintext
twiddles and notes in Sec. 4 that a plaintext constant's bits show through the
Wallace tree). Both words are sign-extended to T = f + F bits and every
partial product is an AND of two ciphertext bits; Lemma 8's Wallace stages and
Lemma 9's middle bits follow unchanged. With encrypted twiddles the FFT takes
one table W_M^k, k < M/2, M = max(N1, N2), as inputs after the signal.

Pins: the closed form floor(x y / 2^f) mod 2^F (exhaustive at F = 4 for every
f, random at 16 and 24 bits), commutativity of the value, the FFT with
encrypted twiddles against the integer FFT (1-D, square and non-square 2-D,
every gate variant), encrypted evaluation decrypting to the closed form with
the exact noise inside the static bound, and the native compiler (circuits,
smallest ell, device program, twiddle table, errors) against the oracle.
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


def _closed(x, y, F, f):
    return fx.wrap(math.floor(x * y / 2 ** f), F)


@pytest.mark.parametrize("f", [0, 1, 2, 3])
def test_mule_exhaustive_f4(f):
    F = 4
    c = circuit.word_circuit("mule", F, f)
    for x, y in itertools.product(range(-8, 8), repeat=2):
        assert _eval_words(c, [x, y], F) == _closed(x, y, F, f), (x, y, f)


@pytest.mark.parametrize("F,f", [(16, 8), (24, 12)])
def test_mule_random_wide(F, f):
    c = circuit.word_circuit("mule", F, f)
    rng = random.Random(F)
    lo, hi = -(1 << (F - 1)), (1 << (F - 1)) - 1
    for _ in range(12):
        x, y = rng.randint(lo, hi), rng.randint(lo, hi)
        got = _eval_words(c, [x, y], F)
        assert got == _closed(x, y, F, f) == _eval_words(c, [y, x], F)
    for x, y in ((lo, lo), (lo, -1), (hi, hi), (0, lo), (-1, -1)):   # extremes and wrap
        assert _eval_words(c, [x, y], F) == _closed(x, y, F, f)


def test_mule_agrees_with_constant_multiplier():
    F, f = 8, 4
    rng = random.Random(5)
    e = circuit.word_circuit("mule", F, f)
    for _ in range(10):
        w = rng.randint(-128, 127)
        m = circuit.word_circuit("mul", F, f, w)
        for _ in range(4):
            x = rng.randint(-128, 127)
            assert _eval_words(e, [x, w], F) == _eval_words(m, [x, 0], F)


def test_mule_partial_products_are_ands_of_inputs():
    F, f = 4, 1
    c = circuit.word_circuit("mule", F, f)
    xs, ys = set(c.inputs[:F]), set(c.inputs[F:])
    first = [g for g in c.gates if g[1] in xs | ys or g[2] in xs | ys]
    # every gate on an input is a partial product x_a y_b with a + b < T
    T = f + F
    for op, a, b, _ in first:
        assert op == "AND" and a in xs and b in ys
        assert sorted(c.inputs).index(a) + sorted(c.inputs).index(b) - F < T


def _fft_bits(c, re, im, tw, F):
    bits = []
    for r, i in zip(re, im):
        bits += fx.to_bits(r, F) + fx.to_bits(i, F)
    for wr, wi in tw:
        bits += fx.to_bits(wr, F) + fx.to_bits(wi, F)
    assert len(bits) == len(c.inputs)
    return bits


@pytest.mark.parametrize("N1,N2,F,f,var", [
    (8, 1, 8, 4, {}), (16, 1, 8, 4, {}), (4, 4, 8, 3, {}), (2, 8, 8, 3, {}), (8, 2, 8, 3, {}),
    (8, 1, 8, 4, {"xcarry": True}), (4, 1, 8, 4, {"nand": True})])
def test_fft_encrypted_twiddles_equals_integer_fft(N1, N2, F, f, var):
    c = circuit.fft_circuit(N1, N2, F, f, enc_twiddle=True, **var)
    M = max(N1, N2)
    rng = random.Random(N1 * 11 + N2)
    lo, hi = -(1 << (F - 2)), (1 << (F - 2)) - 1
    re = [rng.randint(lo, hi) for _ in range(N1 * N2)]
    im = [rng.randint(lo, hi) for _ in range(N1 * N2)]
    out = evaluate.eval_plain(c, _fft_bits(c, re, im, circuit.twiddles(M, f), F))
    words = [fx.from_bits(out[k * F:(k + 1) * F]) for k in range(2 * N1 * N2)]
    want = fx.fft_int(re, im, F, f) if N2 == 1 else fx.fft2_int(re, im, N1, N2, F, f)
    assert (words[0::2], words[1::2]) == tuple(want)


def test_encrypted_twiddles_need_room_for_one():
    with pytest.raises(ValueError):
        circuit.fft_circuit(4, 1, 8, 7, enc_twiddle=True)   # 2^7 does not fit 8 signed bits
    circuit.fft_circuit(4, 1, 8, 6, enc_twiddle=True)


def test_encrypted_word_multiply_noisy_parameters():
    F, f = 4, 1
    c = circuit.word_circuit("mule", F, f)
    ell = noise.smallest_ell(c, n=1, chi=1)
    p = gsw.Params(1, ell, 2 * ell, 1)
    bounds = noise.wire_bounds(c, p)
    keys = gsw.Keys(p, seed=12)
    for k, (x, y) in enumerate([(-8, 7), (5, -3), (-1, -1)]):
        bits = fx.to_bits(x, F) + fx.to_bits(y, F)
        cts = [gsw.encrypt(keys, b, 6, k * 2 * F + j) for j, b in enumerate(bits)]
        out = evaluate.eval_encrypted(c, p, cts)
        dec = [gsw.decrypt(keys, ct) for ct in out]
        assert fx.from_bits(dec) == _closed(x, y, F, f)
        for w, ct, mu in zip(c.outputs, out, dec):
            assert max(map(abs, gsw.noise(keys, ct, mu))) <= bounds[w]


def test_encrypted_fft_with_encrypted_twiddles():
    N, F, f = 2, 4, 1
    c = circuit.fft_circuit(N, 1, F, f, enc_twiddle=True)
    ell = noise.smallest_ell(c, n=1, chi=1)
    p = gsw.Params(1, ell, 2 * ell, 1)
    keys = gsw.Keys(p, seed=13)
    re, im = [3, -4], [-2, 1]
    bits = _fft_bits(c, re, im, circuit.twiddles(N, f), F)
    cts = [gsw.encrypt(keys, b, 7, j) for j, b in enumerate(bits)]
    out = evaluate.eval_encrypted(c, p, cts)
    dec = [gsw.decrypt(keys, ct) for ct in out]
    assert dec == evaluate.eval_plain(c, bits)
    words = [fx.from_bits(dec[k * F:(k + 1) * F]) for k in range(2 * N)]
    assert (words[0::2], words[1::2]) == fx.fft_int(re, im, F, f)


# ----------------------------------------------------------- native vs oracle

@pytest.mark.parametrize("N1,N2,F,f,var", [
    (2, 1, 4, 1, {}), (8, 1, 8, 4, {}), (4, 4, 8, 3, {}), (2, 8, 8, 3, {}),
    (8, 1, 8, 4, {"xcarry": True}), (2, 1, 4, 1, {"nand": True})])
def test_native_fft_program_matches_oracle(N1, N2, F, f, var):
    import paper_1611_08769_gb300 as sf
    sp = sf.param_set("P0")
    c = circuit.fft_circuit(N1, N2, F, f, enc_twiddle=True, **var)
    st = circuit.stats(c)
    info = sf.circuit_info(sp, N1, N2, F, f, enc_twiddle=True, **var)
    assert info["inputs"] == len(c.inputs) and info["outputs"] == len(c.outputs)
    assert info["products"] == st["products"] and info["levels"] == st["depth"]
    assert sf.min_ell(N1, N2, F, f, 1, 1, enc_twiddle=True, **var) == noise.smallest_ell(c, 1, 1)
    rng = random.Random(N1 * 13 + F)
    for _ in range(3):
        bits = [rng.randint(0, 1) for _ in range(len(c.inputs))]
        got = sf.program_eval_plain(sp, N1, N2, F, f, np.array(bits, np.uint8), enc_twiddle=True,
                                    **var)
        assert list(got) == evaluate.eval_plain(c, bits)


@pytest.mark.parametrize("kind,F,f", [("add", 8, 4), ("sub", 8, 4), ("mule", 4, 1), ("mule", 8, 4),
                                      ("mule", 16, 8)])
def test_native_word_program_matches_oracle(kind, F, f):
    import paper_1611_08769_gb300 as sf
    op = {"add": sf.WORD_ADD, "sub": sf.WORD_SUB, "mule": sf.WORD_MUL}[kind]
    sp = sf.param_set("P0")
    count = 5
    c = circuit.word_circuit(kind, F, f)
    info = sf.word_circuit_info(sp, op, count, F, f)
    assert info["inputs"] == 2 * count * F and info["outputs"] == count * F
    assert info["products"] == count * circuit.stats(c)["products"]
    assert sf.word_min_ell(op, F, f) == noise.smallest_ell(c, 1, 1)
    rng = random.Random(F + op)
    xs = [(rng.randint(-(1 << (F - 1)), (1 << (F - 1)) - 1), rng.randint(-(1 << (F - 1)), (1 << (F - 1)) - 1))
          for _ in range(count)]
    bits = []
    for x, y in xs:
        bits += fx.to_bits(x, F) + fx.to_bits(y, F)
    got = sf.word_program_eval_plain(sp, op, count, F, f, np.array(bits, np.uint8))
    for k, (x, y) in enumerate(xs):
        want = {"add": fx.wrap(x + y, F), "sub": fx.wrap(x - y, F), "mule": _closed(x, y, F, f)}[kind]
        assert fx.from_bits([int(v) for v in got[k * F:(k + 1) * F]]) == want


def test_native_twiddle_table_and_errors():
    import paper_1611_08769_gb300 as sf
    for M, f in ((2, 4), (16, 8), (256, 12)):
        wr, wi = sf.twiddles(M, f)
        assert list(zip(wr.tolist(), wi.tolist())) == circuit.twiddles(M, f)
    sp = sf.param_set("P0")
    assert sf.min_ell(4, 1, 8, 7, 1, 1, enc_twiddle=True) == 0
    with pytest.raises(sf.SfftError):
        sf.circuit_info(sp, 4, 1, 8, 7, enc_twiddle=True)
    with pytest.raises(sf.SfftError):
        sf.word_circuit_info(sp, 9, 1, 8, 4)
    with pytest.raises(sf.SfftError):
        sf.word_circuit_info(sp, sf.WORD_MUL, 0, 8, 4)
    with pytest.raises(sf.SfftError):
        sf.twiddles(6, 4)


def test_native_circuit_size_bounds():
    import paper_1611_08769_gb300 as sf
    sp = sf.param_set("P0")
    F, f = 16, 8
    limit = (1 << 28) // ((f + F) * (f + F))
    assert sf.word_circuit_info(sp, sf.WORD_ADD, 1, F, f)["outputs"] == F
    with pytest.raises(sf.SfftError):
        sf.word_circuit_info(sp, sf.WORD_ADD, limit + 1, F, f)
    with pytest.raises(sf.SfftError):
        sf.refresh_circuit_info(sf.param_set("P1", 1056), 1 << 20)
