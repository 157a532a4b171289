"""Pins of the oracle's PRNG and GSW scheme against things other than itself.

* SplitMix64 against its published reference outputs.
* The compressed GSW form against the literal N x N GSW definition
  (Enc, every gate code, two levels deep): BitDecomp^-1 of the literal
  ciphertext must equal the compressed one bit for bit.
* Dec(Enc(b)) = b; gate truth tables on encrypted inputs.
* The measured noise of a gate output equals the closed form
  c1 e_A + c2 e_B + c3 (mu_B e_A + BitDecomp(A') e_B) exactly, and stays within
  the static bound; with chi = 0 it is identically zero.
* BitDecomp by byte unpacking equals BitDecomp by integer shifts; the matrix
  product equals a brute-force big-integer sum.
"""
import itertools
import random

import numpy as np
import pytest

from oracle import gsw, prng


def test_splitmix64_reference_outputs(golden):
    for seed, k, value in golden("splitmix64.txt"):
        assert prng.out(seed, k) == value
        assert int(prng.words(seed, k, 1)[0]) == value


def test_stream_vectorised_matches_scalar():
    state = prng.ct_key(7, 11)
    w = prng.words(state, 3, 50)
    assert [int(x) for x in w] == [prng.out(state, 3 + i) for i in range(50)]


TINY = gsw.Params(1, 32, 64, 1)       # Ng = 64: literal form feasible


@pytest.fixture(scope="module")
def tiny_keys():
    return gsw.Keys(TINY, seed=5)


def test_key_relation(tiny_keys):
    """A s = e (the defining property of the public key)."""
    p, k = TINY, tiny_keys
    for r in range(p.m):
        assert sum(k.A[r][j] * k.s[j] for j in range(p.n + 1)) % p.q == k.e[r] % p.q
    assert all(-p.chi <= e <= p.chi for e in k.e)


def test_bitdecomp_two_routes(tiny_keys):
    ct = gsw.encrypt(tiny_keys, 1, enc_seed=1, ct_index=0)
    b = gsw.bits(ct)
    vals = gsw.from_limbs(ct)
    for i in range(0, TINY.Ng, 7):
        assert list(b[i]) == gsw.bitdecomp_vec(vals[i], TINY)


def test_product_brute_force():
    p = gsw.Params(1, 64, 32, 0)
    rng = np.random.default_rng(0)
    A = rng.integers(0, 2**32, size=(p.Ng, 2, p.L), dtype=np.uint64).astype(np.uint32)
    B = rng.integers(0, 2**32, size=(p.Ng, 2, p.L), dtype=np.uint64).astype(np.uint32)
    got = gsw.from_limbs(gsw.product(A, B, p.L))
    Av, Bv = gsw.from_limbs(A), gsw.from_limbs(B)
    for i in (0, 5, p.Ng - 1):
        bits = gsw.bitdecomp_vec(Av[i], p)
        for j in range(2):
            want = sum(bits[k] * int(Bv[k, j]) for k in range(p.Ng)) % p.q
            assert got[i, j] == want


def test_literal_equals_compressed(tiny_keys):
    """Literal GSW (Flatten of N x N integer matrices) == compressed form."""
    k, p = tiny_keys, TINY
    lit = {}
    comp = {}
    for idx, mu in enumerate((0, 1, 1)):
        lit[idx] = gsw.literal_encrypt(k, mu, enc_seed=9, ct_index=idx)
        comp[idx] = gsw.encrypt(k, mu, enc_seed=9, ct_index=idx)
        assert np.array_equal(gsw.literal_to_compressed(lit[idx], p), comp[idx])
        assert gsw.literal_decrypt(k, lit[idx]) == mu == gsw.decrypt(k, comp[idx])
    # every gate code on (0, 1), then a second level on its output
    for name in ("AND", "XOR", "OR", "NAND", "NOT"):
        code = gsw.GATE_CODES[name]
        B_l = None if name == "NOT" else lit[1]
        B_c = None if name == "NOT" else comp[1]
        L1 = gsw.literal_gate(lit[0], B_l, code, p)
        C1 = gsw.gate(p, comp[0], B_c, code)
        assert np.array_equal(gsw.literal_to_compressed(L1, p), C1), name
        L2 = gsw.literal_gate(L1, lit[2], gsw.GATE_CODES["AND"], p)
        C2 = gsw.gate(p, C1, comp[2], gsw.GATE_CODES["AND"])
        assert np.array_equal(gsw.literal_to_compressed(L2, p), C2), name


def test_trivial_ciphertexts_are_flatten_of_identity():
    p = TINY
    ident = [[1 if i == j else 0 for j in range(p.Ng)] for i in range(p.Ng)]
    assert np.array_equal(gsw.literal_to_compressed(gsw.flatten(ident, p), p), gsw.one_ct(p))
    assert np.array_equal(gsw.bits(gsw.one_ct(p)), np.eye(p.Ng, dtype=np.uint8))


@pytest.mark.parametrize("params", [gsw.Params(1, 32, 64, 0), gsw.Params(1, 64, 128, 1),
                                    gsw.Params(2, 32, 96, 1)])
def test_dec_enc_identity(params):
    keys = gsw.Keys(params, seed=17)
    rng = random.Random(1)
    for idx in range(40):
        mu = rng.randint(0, 1)
        assert gsw.decrypt(keys, gsw.encrypt(keys, mu, enc_seed=4, ct_index=idx)) == mu


TRUTH = {"AND": lambda a, b: a & b, "XOR": lambda a, b: a ^ b, "OR": lambda a, b: a | b,
         "NAND": lambda a, b: 1 - (a & b), "NOR": lambda a, b: 1 - (a | b),
         "XNOR": lambda a, b: 1 - (a ^ b)}


@pytest.mark.parametrize("chi", [0, 1])
def test_gate_truth_tables_encrypted(chi):
    p = gsw.Params(1, 64, 128, chi)
    keys = gsw.Keys(p, seed=2)
    cts = {(mu, r): gsw.encrypt(keys, mu, 3, 2 * mu + r) for mu in (0, 1) for r in (0, 1)}
    for name, fn in TRUTH.items():
        for a, b in itertools.product((0, 1), repeat=2):
            out = gsw.gate(p, cts[(a, 0)], cts[(b, 1)], gsw.GATE_CODES[name])
            assert gsw.decrypt(keys, out) == fn(a, b), (name, a, b)
    for a in (0, 1):
        assert gsw.decrypt(keys, gsw.gate(p, cts[(a, 0)], None, gsw.GATE_CODES["NOT"])) == 1 - a


def test_noise_closed_form_and_bound():
    p = gsw.Params(1, 64, 128, 1)
    keys = gsw.Keys(p, seed=8)
    fresh = p.m * p.chi
    for mu_a, mu_b in itertools.product((0, 1), repeat=2):
        A = gsw.encrypt(keys, mu_a, 6, 10 + mu_a)
        B = gsw.encrypt(keys, mu_b, 6, 20 + mu_b)
        eA, eB = gsw.noise(keys, A, mu_a), gsw.noise(keys, B, mu_b)
        assert max(map(abs, eA)) <= fresh and max(map(abs, eB)) <= fresh
        bitA = gsw.bits(A).astype(object)
        for name in ("AND", "XOR", "OR", "NAND"):
            c0, c1, c2, c3 = gsw.GATE_CODES[name]
            out = gsw.gate(p, A, B, (c0, c1, c2, c3))
            mu = TRUTH[name](mu_a, mu_b)
            e = gsw.noise(keys, out, mu)
            want = [c1 * eA[i] + c2 * eB[i] + c3 * (mu_b * eA[i] + sum(int(bitA[i, k]) * eB[k]
                                                                       for k in range(p.Ng)))
                    for i in range(p.Ng)]
            assert e == want, name
            bound = (abs(c1) + abs(c3)) * fresh + (abs(c2) + abs(c3) * p.Ng) * fresh
            assert max(map(abs, e)) <= bound


def test_noise_free_parameters_have_zero_noise():
    p = gsw.Params(1, 32, 64, 0)
    keys = gsw.Keys(p, seed=0)
    A = gsw.encrypt(keys, 1, 0, 0)
    B = gsw.encrypt(keys, 1, 0, 1)
    out = gsw.gate(p, gsw.gate(p, A, B, gsw.GATE_CODES["XOR"]), A, gsw.GATE_CODES["OR"])
    assert all(x == 0 for x in gsw.noise(keys, out, 1))
    assert all(x == 0 for x in gsw.noise(keys, A, 1))


def test_constant_folding_is_bit_exact():
    """AND(x,1)=x, XOR(x,1)=NOT x, OR(x,1)=1, AND(x,0)=0 on ciphertexts, both operand orders."""
    p = gsw.Params(1, 64, 128, 1)
    keys = gsw.Keys(p, seed=4)
    x = gsw.encrypt(keys, 1, 1, 0)
    one, zero = gsw.one_ct(p), gsw.zero_ct(p)
    notx = gsw.gate(p, x, None, gsw.GATE_CODES["NOT"])
    C = gsw.GATE_CODES
    for A, B in ((x, one), (one, x)):
        assert np.array_equal(gsw.gate(p, A, B, C["AND"]), x)
        assert np.array_equal(gsw.gate(p, A, B, C["XOR"]), notx)
        assert np.array_equal(gsw.gate(p, A, B, C["OR"]), one)
    for A, B in ((x, zero), (zero, x)):
        assert np.array_equal(gsw.gate(p, A, B, C["AND"]), zero)
        assert np.array_equal(gsw.gate(p, A, B, C["XOR"]), x)
        assert np.array_equal(gsw.gate(p, A, B, C["OR"]), x)
    assert np.array_equal(gsw.gate(p, notx, None, C["NOT"]), x)
