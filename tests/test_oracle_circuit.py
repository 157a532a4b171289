"""Pins of the oracle's gate circuit and fixed-point FFT.

* Half/full adder truth tables, exhaustively.
* F = 4: every ADD, SUB (all 256 operand pairs) and every constant MUL
  (all x, all w, f = 0..3) against (x+y), (x-y), floor(x w / 2^f) mod 2^F.
* Random wider words (F = 8..24) against the same closed forms.
* The plaintext FFT circuit against the closed-form integer DIT FFT, 1-D and 2-D.
* Quantised twiddles against hand-worked values (tests/golden/twiddles_n8_f4.txt).
* The FP64 DFT against numpy's FFT; the fixed-point FFT error against the
  paper's Theorem 2 bound in the paper's own setting (32-bit words, 16
  fraction bits, signals in [0, 1], N = 8 .. 128).
* Gate counts within the paper's complexity bounds (Sec. 7).
"""
import itertools
import math
import random

import numpy as np
import pytest

from oracle import circuit, evaluate, fixedpoint as fx


def _eval_words(c, xs, F):
    bits = []
    for x in xs:
        bits += fx.to_bits(x, F)
    return fx.from_bits(evaluate.eval_plain(c, bits))


def test_half_and_full_adder_exhaustive():
    c = circuit.Circuit()
    a, b, d = c.new_input(), c.new_input(), c.new_input()
    s, cy = c.HA(a, b)
    s3, cy3 = c.FA(a, b, d)
    c.outputs = [s, cy, s3, cy3]
    for x, y, z in itertools.product((0, 1), repeat=3):
        out = evaluate.eval_plain(c, [x, y, z])
        assert out[0] + 2 * out[1] == x + y
        assert out[2] + 2 * out[3] == x + y + z


def test_constant_inputs_fold():
    c = circuit.Circuit()
    x = c.new_input()
    Z, O = circuit.ZERO, circuit.ONE
    assert c.AND(x, O) == x and c.AND(O, x) == x and c.AND(x, Z) == Z
    assert c.XOR(x, Z) == x and c.OR(x, Z) == x and c.OR(O, x) == O
    n = c.XOR(x, O)
    assert c.gates[-1] == ("NOT", x, None, n)
    assert c.NOT(Z) == O and c.NOT(O) == Z


@pytest.mark.parametrize("kind", ["add", "sub"])
def test_add_sub_exhaustive_f4(kind):
    F = 4
    c = circuit.word_circuit(kind, F)
    for x, y in itertools.product(range(-8, 8), repeat=2):
        want = fx.wrap(x + y if kind == "add" else x - y, F)
        assert _eval_words(c, [x, y], F) == want, (x, y)


@pytest.mark.parametrize("f", [0, 1, 2, 3])
def test_mul_exhaustive_f4(f):
    F = 4
    for w in range(-8, 8):
        c = circuit.word_circuit("mul", F, f, w)
        for x in range(-8, 8):
            got = _eval_words(c, [x, 0], F)
            assert got == fx.wrap(math.floor(x * w / 2 ** f), F), (x, w, f)


@pytest.mark.parametrize("F,f", [(8, 4), (12, 5), (16, 8), (24, 12)])
def test_word_ops_random(F, f):
    rng = random.Random(F * 31 + f)
    lo, hi = -(1 << (F - 1)), (1 << (F - 1)) - 1
    add, sub = circuit.word_circuit("add", F), circuit.word_circuit("sub", F)
    for _ in range(30):
        x, y = rng.randint(lo, hi), rng.randint(lo, hi)
        assert _eval_words(add, [x, y], F) == fx.wrap(x + y, F)
        assert _eval_words(sub, [x, y], F) == fx.wrap(x - y, F)
    for _ in range(6):
        w = rng.randint(-(1 << f), 1 << f)
        mul = circuit.word_circuit("mul", F, f, w)
        for _ in range(5):
            x = rng.randint(lo, hi)
            assert _eval_words(mul, [x, 0], F) == fx.wrap(math.floor(x * w / 2 ** f), F)


def test_mul_fix_closed_form_is_floor():
    for x, w, f in [(-7, 3, 2), (5, -5, 1), (-8, -8, 3), (7, 7, 0)]:
        assert fx.mul_fix(x, w, 8, f) == fx.wrap(math.floor(x * w / 2 ** f), 8)


def test_twiddles_hand_worked(golden):
    tw = circuit.twiddles(8, 4)
    for k, wr, wi in golden("twiddles_n8_f4.txt"):
        assert tw[k] == (wr, wi)


def _plain_fft_via_circuit(c, re, im, F):
    bits = []
    for r, i in zip(re, im):
        bits += fx.to_bits(r, F) + fx.to_bits(i, F)
    out = evaluate.eval_plain(c, bits)
    words = [fx.from_bits(out[k * F:(k + 1) * F]) for k in range(2 * len(re))]
    return words[0::2], words[1::2]


@pytest.mark.parametrize("N,F,f", [(2, 8, 4), (4, 8, 4), (8, 8, 4), (16, 12, 6), (32, 16, 8)])
def test_fft_circuit_equals_integer_fft(N, F, f):
    c = circuit.fft_circuit(N, 1, F, f)
    rng = random.Random(N)
    lo, hi = -(1 << (F - 1)), (1 << (F - 1)) - 1
    for _ in range(3):
        re = [rng.randint(lo, hi) for _ in range(N)]
        im = [rng.randint(lo, hi) for _ in range(N)]
        assert _plain_fft_via_circuit(c, re, im, F) == fx.fft_int(re, im, F, f)


@pytest.mark.parametrize("N1,N2", [(4, 4), (2, 8), (8, 2)])
def test_fft2d_circuit_equals_integer_fft(N1, N2):
    F, f = 10, 4
    c = circuit.fft_circuit(N1, N2, F, f)
    rng = random.Random(N1 * 10 + N2)
    re = [rng.randint(-512, 511) for _ in range(N1 * N2)]
    im = [rng.randint(-512, 511) for _ in range(N1 * N2)]
    assert _plain_fft_via_circuit(c, re, im, F) == fx.fft2_int(re, im, N1, N2, F, f)


def test_dft_fp64_matches_numpy():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(16) + 1j * rng.standard_normal(16)
    Xr, Xi = fx.dft_fp64(list(x.real), list(x.imag))
    ref = np.fft.fft(x)
    assert np.allclose(np.array(Xr) + 1j * np.array(Xi), ref, atol=1e-12)
    img = rng.standard_normal(32) + 1j * rng.standard_normal(32)
    Yr, Yi = fx.dft2_fp64(list(img.real), list(img.imag), 4, 8)
    ref2 = np.fft.fft2(img.reshape(4, 8)).reshape(-1)
    assert np.allclose(np.array(Yr) + 1j * np.array(Yi), ref2, atol=1e-12)


@pytest.mark.parametrize("N", [8, 16, 32, 64, 128])
def test_theorem2_error_bound_paper_setting(N):
    """Sec. 6 setting: 32-bit words, 16 fraction bits, signals in [0, 1]."""
    F, f = 32, 16
    rng = random.Random(N)
    worst = 0.0
    for _ in range(5):
        x = [rng.random() for _ in range(N)]
        re = [fx.quantize(v, F, f) for v in x]
        im = [0] * N
        assert not fx.fft_int_overflows(re, im, F, f)
        gr, gi = fx.fft_int(re, im, F, f)
        Xr, Xi = fx.dft_fp64(x, [0.0] * N)
        err = max(max(abs(gr[k] / 2 ** f - Xr[k]), abs(gi[k] / 2 ** f - Xi[k])) for k in range(N))
        worst = max(worst, err)
    bound = fx.error_bound(N, f, 1.0)
    assert worst <= bound, (worst, bound)
    # Table 1 reports per-point errors of order 1e-5 .. 1e-4 for N = 8 .. 128
    assert worst < 1e-2


def test_gate_counts_within_paper_bounds():
    """Sec. 7: adder <= 36F NAND, multiplier <= 288 F^2 log F NAND; products <= NANDs."""
    for F in (8, 16, 24):
        add = circuit.stats(circuit.word_circuit("add", F))
        assert add["products"] <= 36 * F
        # HA at bit 0 (1 product), F-2 full adders (3 each), top FA without its carry OR (2)
        assert add["products"] == 3 * F - 3
        for w in (-(1 << (F // 2)), (1 << (F // 2)) - 3, 5):
            mul = circuit.stats(circuit.word_circuit("mul", F, F // 2, w))
            assert mul["products"] <= 288 * F * F * math.log2(F)
