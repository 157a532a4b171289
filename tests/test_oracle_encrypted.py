"""Encrypted evaluation on the oracle decrypts to the plaintext circuit.

Theorem 1's proof composes Lemmas 1-3: encryption, gate-by-gate evaluation
and decryption. Here the encrypted FFT circuit, evaluated on the oracle's
compressed GSW ciphertexts, must decrypt to the plaintext circuit's output
bit for bit, in the noise-free toy parameters and in a noisy leveled set
whose q is sized by the static noise bound. The measured noise of every
output must stay inside that bound.
"""
import random

import numpy as np
import pytest

from oracle import circuit, evaluate, fixedpoint as fx, gsw, noise


def _encrypt_signal(keys, re, im, F, enc_seed):
    cts, bits = [], []
    for k, (r, i) in enumerate(zip(re, im)):
        for part, v in enumerate((r, i)):
            for b, bit in enumerate(fx.to_bits(v, F)):
                cts.append(gsw.encrypt(keys, bit, enc_seed, (k * 2 + part) * F + b))
                bits.append(bit)
    return cts, bits


def test_encrypted_fft_8pt_toy_parameters():
    N, F, f = 8, 8, 4
    p = gsw.Params(1, 32, 64, 0)
    keys = gsw.Keys(p, seed=0)
    rng = random.Random(0)
    re = [fx.quantize(rng.uniform(-1, 1), F, f) for _ in range(N)]
    im = [0] * N
    c = circuit.fft_circuit(N, 1, F, f)
    cts, bits = _encrypt_signal(keys, re, im, F, enc_seed=0)
    out = evaluate.eval_encrypted(c, p, cts)
    dec = [gsw.decrypt(keys, ct) for ct in out]
    assert dec == evaluate.eval_plain(c, bits)
    words = [fx.from_bits(dec[k * F:(k + 1) * F]) for k in range(2 * N)]
    assert (words[0::2], words[1::2]) == fx.fft_int(re, im, F, f)


def test_encrypted_fft_noisy_leveled_parameters():
    N, F, f = 2, 4, 1
    c = circuit.fft_circuit(N, 1, F, f)
    ell = noise.smallest_ell(c, n=1, chi=1)
    p = gsw.Params(1, ell, 2 * ell, 1)
    bounds = noise.wire_bounds(c, p)
    assert max(bounds) < p.q // 4
    keys = gsw.Keys(p, seed=3)
    re, im = [3, -5], [-2, 7]
    cts, bits = _encrypt_signal(keys, re, im, F, enc_seed=1)
    out = evaluate.eval_encrypted(c, p, cts)
    plain = evaluate.eval_plain(c, bits)
    assert [gsw.decrypt(keys, ct) for ct in out] == plain
    for w, ct, mu in zip(c.outputs, out, plain):
        e = gsw.noise(keys, ct, mu)
        assert max(map(abs, e)) <= bounds[w]
    words = [fx.from_bits(plain[k * F:(k + 1) * F]) for k in range(2 * N)]
    assert (words[0::2], words[1::2]) == fx.fft_int(re, im, F, f)


def test_operand_order_changes_ciphertext_not_plaintext():
    """Why the depth rule must be canonical: swapping A and B changes bits."""
    p = gsw.Params(1, 32, 64, 0)
    keys = gsw.Keys(p, seed=1)
    a = gsw.encrypt(keys, 1, 2, 0)
    b = gsw.encrypt(keys, 1, 2, 1)
    ab = gsw.gate(p, a, b, gsw.GATE_CODES["AND"])
    ba = gsw.gate(p, b, a, gsw.GATE_CODES["AND"])
    assert not np.array_equal(ab, ba)
    assert gsw.decrypt(keys, ab) == gsw.decrypt(keys, ba) == 1
