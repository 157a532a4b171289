"""Ciphertext refresh (bootstrapping by homomorphic decryption; the paper's
Sec. 5 ends by pointing at refreshing without a construction).

Pins: the truncated sum S against the exact phase (2^tau S = x - R mod q with
0 <= R < rows 2^tau), the refreshed bit against exact decryption for every
phase noise in [-q/8, q/4) (sampled, including both edges), the selectors
against the definition of K'_r, the refresh circuit's plaintext evaluation
against the closed form, encrypted refresh of noisy ciphertexts decrypting to
their bit with the exact noise inside the static bound and below q/8 (so the
output can be refreshed again), and the native compiler against the oracle.
"""
import random

import numpy as np
import pytest

from oracle import circuit, evaluate, gsw, noise, refresh


def _row_with_phase(p, keys, x, rng):
    """A public row c with <c, s> = x (mod q): c_1..c_n random, c_0 solves."""
    row = [0] + [rng.randrange(p.q) for _ in range(p.n)]
    acc = sum(row[j] * keys.s[j] for j in range(1, p.n + 1))
    row[0] = (x - acc) % p.q
    return row


def _phase(p, keys, row):
    return sum(row[j] * keys.s[j] for j in range(p.n + 1)) % p.q


@pytest.mark.parametrize("n,ell", [(1, 64), (2, 64), (1, 224)])
def test_truncated_sum_tracks_the_phase(n, ell):
    p = gsw.Params(n, ell, (n + 1) * ell, 1)
    keys = gsw.Keys(p, seed=n + ell)
    sigma = refresh.key_bits(keys)
    rows, pbits, tau = refresh.shape(p)
    assert 2 ** pbits >= 8 * rows and len(sigma) == rows
    rng = random.Random(ell)
    for _ in range(50):
        row = [rng.randrange(p.q) for _ in range(n + 1)]
        S = row[0] >> tau
        for j in range(1, n + 1):
            for b in range(ell):
                S += sigma[1 + (j - 1) * ell + b] * (((row[j] << b) % p.q) >> tau)
        R = (_phase(p, keys, row) - (S << tau)) % p.q
        assert 0 <= R < rows << tau


@pytest.mark.parametrize("n,ell", [(1, 64), (2, 96), (1, 224)])
def test_refreshed_bit_equals_decryption(n, ell):
    p = gsw.Params(n, ell, (n + 1) * ell, 1)
    keys = gsw.Keys(p, seed=3 * ell + n)
    sigma = refresh.key_bits(keys)
    rng = random.Random(n * ell)
    q = p.q
    edges = [-q // 8, -q // 8 + 1, -1, 0, 1, q // 4 - 1, q // 8 - 1]
    for mu in (0, 1):
        for e in edges + [rng.randrange(-q // 8, q // 4) for _ in range(40)]:
            row = _row_with_phase(p, keys, (mu * q // 2 + e) % q, rng)
            assert refresh.refreshed_bit(p, row, sigma) == mu, (mu, e)


def test_selectors_are_bits_of_the_truncated_terms():
    p = gsw.Params(2, 64, 192, 1)
    rows, pbits, tau = refresh.shape(p)
    rng = random.Random(4)
    row = [rng.randrange(p.q) for _ in range(p.n + 1)]
    K = [row[0] >> tau] + [((row[j] << b) % p.q) >> tau for j in range(1, p.n + 1)
                           for b in range(p.ell)]
    for k, col in enumerate(refresh.selectors(p, row)):
        present = {r for r, _ in col}
        for r, beta in col:
            assert beta == (K[r] >> k) & 1
        for r in set(range(rows)) - present:     # left out only where statically zero
            assert (K[r] >> k) & 1 == 0
            assert r > 0 and tau + k - (r - 1) % p.ell < 0


@pytest.mark.parametrize("xcarry", [False, True])
def test_circuit_equals_closed_form(xcarry):
    p = gsw.Params(1, 64, 128, 1)
    keys = gsw.Keys(p, seed=17)
    sigma = refresh.key_bits(keys)
    rng = random.Random(18)
    rows_list = [[rng.randrange(p.q) for _ in range(p.n + 1)] for _ in range(6)]
    for mu in (0, 1):   # phases on and near the decision edges
        for e in (-p.q // 8, p.q // 4 - 1):
            rows_list.append(_row_with_phase(p, keys, (mu * p.q // 2 + e) % p.q, rng))
    c = refresh.refresh_circuit(p, rows_list, xcarry=xcarry)
    assert len(c.outputs) == len(rows_list)
    got = evaluate.eval_plain(c, sigma)
    assert got == [refresh.refreshed_bit(p, row, sigma) for row in rows_list]
    # random key bits too: the circuit computes the closed form for any sigma
    for _ in range(3):
        s2 = [1] + [rng.randint(0, 1) for _ in range(len(sigma) - 1)]
        assert evaluate.eval_plain(c, s2) == [refresh.refreshed_bit(p, r, s2) for r in rows_list]


def test_structure_does_not_depend_on_the_selectors():
    p = gsw.Params(1, 64, 128, 1)
    rng = random.Random(2)
    a = refresh.refresh_circuit(p, [[rng.randrange(p.q), rng.randrange(p.q)]])
    b = refresh.refresh_circuit(p, [None])
    strip = [(op[:3] if op.startswith("SEL") else op, x, y, o) for op, x, y, o in a.gates]
    assert strip == [(op[:3] if op.startswith("SEL") else op, x, y, o) for op, x, y, o in b.gates]


def _noisy_ciphertext(keys, mu, seed):
    """Encrypt mu, then grow its noise: AND with fresh encryptions of 1."""
    p = keys.p
    ct = gsw.encrypt(keys, mu, seed, 0)
    for i in range(1, 4):
        one = gsw.encrypt(keys, 1, seed, i)
        ct = gsw.gate(p, one, ct, gsw.GATE_CODES["AND"])   # noise grows by ~Ng per step
    return ct


def test_encrypted_refresh_smallest_ell():
    xcarry = True
    ell = refresh.min_ell(1, 1, xcarry=xcarry)
    p = gsw.Params(1, ell, 2 * ell, 1)
    keys = gsw.Keys(p, seed=31)
    bk = refresh.bootstrap_key(keys, enc_seed=77)
    cts, mus = [], []
    for k, mu in enumerate((1, 0)):
        ct = _noisy_ciphertext(keys, mu, 100 + k)
        assert max(map(abs, gsw.noise(keys, ct, mu))) < p.q // 8
        cts.append(ct)
        mus.append(mu)
    c = refresh.refresh_circuit(p, [refresh.public_row(ct, p) for ct in cts], xcarry=xcarry)
    out = evaluate.eval_encrypted(c, p, bk)
    bound = noise.max_bound(refresh.refresh_circuit(p, [None], xcarry=xcarry), p)
    assert bound < p.q // 8
    for ct, mu in zip(out, mus):
        assert gsw.decrypt(keys, ct) == mu
        assert max(map(abs, gsw.noise(keys, ct, mu))) <= bound


def test_min_ell_is_smallest_with_output_below_q_over_8():
    for xcarry in (False, True):
        ell = refresh.min_ell(1, 1, xcarry=xcarry)
        for e in (ell - 32, ell):
            p = gsw.Params(1, e, 2 * e, 1)
            b = noise.max_bound(refresh.refresh_circuit(p, [None], xcarry=xcarry), p)
            assert (b < p.q // 8) == (e == ell)


# ----------------------------------------------------------- native vs oracle

@pytest.mark.parametrize("n,ell,xcarry", [(1, 64, False), (1, 64, True), (2, 64, False),
                                          (1, 224, False)])
def test_native_refresh_program_matches_oracle(n, ell, xcarry):
    import paper_1611_08769_gb300 as sf
    sp = sf.Params(n, ell, (n + 1) * ell, 1)
    p = gsw.Params(n, ell, (n + 1) * ell, 1)
    count = 4
    rng = random.Random(n * 1000 + ell)
    keys = sf.keygen(sp, 6)
    ko = gsw.Keys(p, 6)
    kb = keys.key_bits()
    assert list(kb) == refresh.key_bits(ko)
    rows = [[rng.randrange(p.q) for _ in range(n + 1)] for _ in range(count - 2)]
    for mu in (0, 1):   # phases on the decision edges
        rows.append(_row_with_phase(p, ko, (mu * p.q // 2 - p.q // 8) % p.q, rng))
    c = refresh.refresh_circuit(p, rows, xcarry=xcarry)
    worst = refresh.refresh_circuit(p, [None] * count, xcarry=xcarry)
    info = sf.refresh_circuit_info(sp, count, xcarry=xcarry)
    st = circuit.stats(c)
    assert info["inputs"] == n * ell + 1 and info["outputs"] == count
    assert info["products"] == st["products"] == circuit.stats(worst)["products"]
    # levels: the multiplicative depth, more where a level's width is capped
    assert info["levels"] >= st["depth"] and info["max_level_width"] <= 4096
    assert info["noise_bits"] == noise.max_bound(worst, p).bit_length()
    h_rows = np.array([gsw.to_limbs(np.array(r, dtype=object), p.L).reshape(-1) for r in rows],
                      dtype=np.uint32)
    got = sf.refresh_eval_plain(sp, kb, h_rows, xcarry=xcarry)
    assert list(got) == evaluate.eval_plain(c, list(kb))
    assert list(got) == [refresh.refreshed_bit(p, r, [int(v) for v in kb]) for r in rows]


def test_native_refresh_min_ell_matches_oracle():
    import paper_1611_08769_gb300 as sf
    for xcarry in (False, True):
        assert sf.refresh_min_ell(1, 1, xcarry=xcarry) == refresh.min_ell(1, 1, xcarry=xcarry)


def test_native_refresh_rejects_both_gate_variants():
    import paper_1611_08769_gb300 as sf
    with pytest.raises(sf.SfftError):
        sf.refresh_circuit_info(sf.Params(1, 64, 128, 1), 1, xcarry=True, nand=True)
    assert sf.refresh_min_ell(1, 1, xcarry=True, nand=True) == 0
