"""Ciphertext refresh by homomorphic decryption (oracle side).

The paper evaluates a leveled circuit and, at the end of its noise analysis
(Sec. 5), points at refreshing ciphertexts so that evaluation could go on
indefinitely, without giving a construction. This module states the
construction used here, a reading of that remark.

Decryption of a compressed ciphertext reads row ell - 1, c = (c_0, ..., c_n),
and its phase x = <c, s> mod q with s = (1, -t). Let sigma_0 = 1 and, for
j >= 1, sigma_{j,b} be bit b of s_j = -t_j mod q. Then

    x = sum_r K_r sigma_r  (mod q),   K_0 = c_0,   K_{j,b} = c_j 2^b mod q,

over the rows r = 0 and r = (j, b), rows = n ell + 1 in all. Only the top bits
of x decide the rounding. With p = ceil(log2 rows) + 3, tau = ell - p and
K'_r = floor(K_r / 2^tau),

    S = sum_r K'_r sigma_r  (mod 2^p)   satisfies   2^tau S = x - R (mod q),

with 0 <= R < rows 2^tau <= q/8. The refreshed bit is [S's top two bits
differ], i.e. [q/4 <= 2^tau S < 3q/4], which equals the decryption of x = mu
q/2 + e whenever e lies in [-q/8, q/4); |e| < q/8 suffices.

Bit k of K'_{j,b} is bit tau + k - b of c_j (zero when that index is
negative) and bit k of K'_0 is bit tau + k of c_0: the selectors are bits of
the refreshed ciphertext itself, public to the evaluator.

Circuit (for each refreshed ciphertext): the bootstrapping key holds GSW
encryptions of sigma_r (same key). Column k < p of the sum receives SEL(BK_r,
bit k of K'_r), the linear gate beta * C, for r = 0 then r = (j, b) in (j, b)
order, leaving out the statically zero selectors; Lemma 8's Wallace stages
and an ADD_p (carries out of bit p - 1 dropped) give S; the output is
XOR(S_{p-1}, S_{p-2}). SEL gates are never folded, so the circuit's
structure, and with it every ciphertext bit, is the same for every beta.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
import math

from . import gsw, noise
from .circuit import Circuit


def shape(p):
    """(rows, pbits, tau) of the refresh sum for parameters p (the truncation
    stated in this module's docstring)."""
    rows = p.n * p.ell + 1
    pbits = math.ceil(math.log2(rows)) + 3
    if pbits > p.ell:
        raise ValueError("ell too small to refresh")
    return rows, pbits, p.ell - pbits


def key_bits(keys):
    """sigma_r in row order: 1, then bit b of s_j (j = 1..n, b = 0..ell-1);
    s = (1, -t) is GSW'13's secret vector (Sec. 3)."""
    p = keys.p
    out = [1]
    for j in range(1, p.n + 1):
        out += [(keys.s[j] >> b) & 1 for b in range(p.ell)]
    return out


def bootstrap_key(keys, enc_seed):
    """GSW encryptions (Sec. 3) of every sigma_r (ciphertext index r under
    enc_seed): the bootstrapping key."""
    return [gsw.encrypt(keys, bit, enc_seed, r) for r, bit in enumerate(key_bits(keys))]


def selectors(p, row):
    """For each column k < p: [(r, beta)] with beta = bit k of K'_r, for the
    public row c = row (n + 1 ints); rows whose selector is statically zero
    are left out."""
    rows, pbits, tau = shape(p)
    cols = []
    for k in range(pbits):
        col = [(0, (row[0] >> (tau + k)) & 1)]
        for j in range(1, p.n + 1):
            for b in range(p.ell):
                if tau + k - b >= 0:
                    col.append((1 + (j - 1) * p.ell + b, (row[j] >> (tau + k - b)) & 1))
        cols.append(col)
    return cols


def refresh_circuit(p, rows_list, xcarry=False, nand=False):
    """Circuit refreshing one ciphertext per entry of rows_list (its public
    row ell - 1 as n + 1 ints; None selects every key ciphertext, the
    worst case used for the static noise bound). Inputs: the bootstrapping
    key; outputs: one refreshed bit per entry."""
    nrows, pbits, _ = shape(p)
    c = Circuit(xcarry, nand)
    bk = [c.new_input() for _ in range(nrows)]
    for row in rows_list:
        cols = []
        for k, col in enumerate(selectors(p, row if row is not None else [0] * (p.n + 1))):
            cols.append([c.SEL(bk[r], 1 if row is None else beta) for r, beta in col])
        S = c._wallace(cols)
        c.outputs.append(c.XOR(S[pbits - 1], S[pbits - 2]))
    c.prune()
    return c


def public_row(ct, p):
    """Row ell - 1 of a compressed ciphertext as n + 1 Python ints: the row
    that decryption reads (Sec. 3)."""
    return [int(v) for v in gsw.from_limbs(ct[p.ell - 1])]


def refreshed_bit(p, row, sigma):
    """Closed form of the refresh: [top two bits of S differ], S computed
    from the definitions with Python integers."""
    _, pbits, tau = shape(p)
    S = row[0] >> tau
    r = 1
    for j in range(1, p.n + 1):
        for b in range(p.ell):
            S += sigma[r] * (((row[j] << b) % p.q) >> tau)
            r += 1
    S %= 1 << pbits
    return ((S >> (pbits - 1)) ^ (S >> (pbits - 2))) & 1


def min_ell(n, chi, xcarry=False, nand=False, limit=8192):
    """Smallest ell (multiple of 32, m = Ng) at which the refresh circuit's
    static output bound stays below q/8, so that its output can be
    refreshed again; 0 if none up to limit."""
    ell = 32
    while ell <= limit:
        p = gsw.Params(n, ell, (n + 1) * ell, chi)
        try:
            c = refresh_circuit(p, [None], xcarry, nand)
        except ValueError:
            ell += 32
            continue
        if noise.max_bound(c, p) < p.q // 8:
            return ell
        ell += 32
    return 0
