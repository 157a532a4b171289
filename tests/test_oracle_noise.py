"""The oracle's static noise bound, pinned in both directions (CPU only).

Upper side: hand-derived bounds of a small gate chain (tests/golden/
noise_bound_chain.txt, worked in its comments) must equal the oracle's.
Lower side: the per-gate bound is attained, exactly, by constructed
ciphertexts, so an overestimate (a factor Ng on the wrong operand, a fresh
noise counted twice) fails as surely as an underestimate. GSW'13 is the scheme
Sec. 3 names; Sec. 7 gives the N x N ciphertext size behind the Ng factor.
"""
import numpy as np
import pytest

from oracle import circuit, gsw, noise


def test_chain_bounds_match_hand_derivation(golden):
    rows = golden("noise_bound_chain.txt")
    p = gsw.Params(1, 64, 128, 1)
    c = circuit.Circuit()
    x, y, z = c.new_input(), c.new_input(), c.new_input()
    s, cy = c.HA(x, y)
    t = c.AND(s, z)
    o = c.OR(cy, t)
    E = noise.wire_bounds(c, p)
    got = {0: E[x], 1: E[y], 2: E[z], 3: E[cy], 4: E[s], 5: E[t], 6: E[o]}
    assert got == {r[0]: r[1] for r in rows}


class _Key:
    """A GSW key with a chosen secret t (n = 1): s = (1, -t), v = Powersof2(s)."""

    def __init__(self, p, t):
        self.p = p
        self.t = [t]
        self.s = [1, (-t) % p.q]
        self.v = [(1 << b) * self.s[j] % p.q for j in range(p.n + 1) for b in range(p.ell)]


def _ct(p, key, mu, noise_of_row, rng, row0_all_ones=False):
    """Compressed ciphertext with row i = (x_i, y_i), x_i - t y_i = mu v_i + e_i."""
    rows = []
    for i in range(p.Ng):
        if row0_all_ones and i == 0:
            rows.append([p.q - 1, p.q - 1])
            continue
        y = int(rng.integers(0, 2**63)) % p.q
        xv = (mu * key.v[i] + noise_of_row(i) + key.t[0] * y) % p.q
        rows.append([xv, y])
    return gsw.to_limbs(np.array(rows, dtype=object), p.L)


@pytest.mark.parametrize("code", [(0, 0, 0, 1), (1, 0, 0, -1), (0, 1, 0, 1), (0, 0, 1, 1),
                                  (0, 2, 1, 3), (0, 0, 0, -2)])
def test_gate_bound_is_attained(code):
    """Row 0 of A' all ones (every bit of BitDecomp(A') set), mu_B = 1, every
    row of B at noise +E_B and A at +E_A: with coefficients of one sign the
    noise of row 0 is (|c1| + |c3|) E_A + (|c2| + |c3| Ng) E_B exactly."""
    p = gsw.Params(1, 64, 128, 1)
    EA, EB = 5, 3
    # row 0 of the all-ones A' has phase t - 1 = mu_A v_0 + e_0 with v_0 = 1:
    # t = 2 + EA gives mu_A = 1 and noise exactly EA there
    key = _Key(p, 2 + EA)
    rng = np.random.default_rng(1)
    A = _ct(p, key, 1, lambda i: EA, rng, row0_all_ones=True)
    B = _ct(p, key, 1, lambda i: EB, rng)
    assert gsw.noise(key, A, 1) == [EA] * p.Ng
    assert gsw.noise(key, B, 1) == [EB] * p.Ng
    out = gsw.gate(p, A, B, code)
    c0, c1, c2, c3 = code
    mu = c0 + c1 + c2 + c3   # the gate's (integer) message at mu_A = mu_B = 1
    e = gsw.noise(key, out, mu)
    bound = noise.gate_bound(code, EA, EB, p.Ng)
    assert max(abs(v) for v in e) == bound
    assert abs(e[0]) == bound
    assert bound == (abs(c1) + abs(c3)) * EA + (abs(c2) + abs(c3) * p.Ng) * EB


def test_fresh_bound_is_attained():
    """R A with every R entry 1 and every key error +chi: noise m chi."""
    p = gsw.Params(1, 64, 16, 1)
    key = _Key(p, 12345)
    rng = np.random.default_rng(2)
    Bcol = [int(rng.integers(0, 2**63)) % p.q for _ in range(p.m)]
    A = [[(b * key.t[0] + p.chi) % p.q, b] for b in Bcol]   # A = [B t + e | B], e = +chi
    RA = [[sum(A[k][j] for k in range(p.m)) % p.q for j in range(2)] for _ in range(p.Ng)]
    ct = gsw.to_limbs(np.array(RA, dtype=object), p.L)
    assert gsw.noise(key, ct, 0) == [noise.fresh_bound(p)] * p.Ng
    assert noise.fresh_bound(p) == p.m * p.chi
