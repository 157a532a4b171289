"""GSW'13 leveled FHE, as used by the paper (Sec. 3), in two forms.

The paper names Gentry-Sahai-Waters (CRYPTO 2013) as its scheme and lists its
four evaluation capabilities (addition, constant multiplication, ciphertext
multiplication, NAND) without restating it (Sec. 3); Sec. 7 notes that a
ciphertext is an N x N matrix and that a NAND costs an N x N matrix product.
The definitions below restate GSW'13 Sec. 3:

    q = 2^ell, Ng = (n+1) ell
    BitDecomp(a)      bits of every element of a, LSB first, element by element
    BitDecomp^-1(x)_j = sum_b 2^b x_{j ell + b}  mod q   (x any integers)
    Flatten(X)        = BitDecomp(BitDecomp^-1(X))
    Powersof2(s)_{j ell + b} = 2^b s_j
    KeyGen: t <- Z_q^n, s = (1, -t), B <- Z_q^{m x n}, e <- chi^m,
            A = [B t + e | B]            (so A s = e)
    Enc(mu): R <- {0,1}^{Ng x m},  C = Flatten(mu I + BitDecomp(R A))
    Dec:     x = <C_{ell-1}, v>, v = Powersof2(s);  mu = [q/4 <= x < 3q/4]
    Gate (c0,c1,c2,c3) on C1, C2:  Flatten(c0 I + c1 C1 + c2 C2 + c3 C1 C2)

Compressed form (what both the oracle and the GPU store): a ciphertext is
kept as C' = BitDecomp^-1(C), an Ng x (n+1) matrix over Z_q (Ng^2 bits).
Because BitDecomp^-1(X) = X P with the gadget matrix P[j ell + b][j] = 2^b,
and BitDecomp(C') = C for a flattened C:

    Enc:  C' = R A + mu P                       (mod q)
    Gate: C' = c0 P + c1 A' + c2 B' + c3 BitDecomp(A') B'   (mod q)
    Dec:  x = <C'_{ell-1}, s>                   (mod q)

``literal_*`` implements the N x N binary form for tiny parameters; the tests
check that BitDecomp^-1 of every literal ciphertext equals the compressed one.

Storage: a compressed ciphertext is a uint32 array of shape (Ng, n+1, L),
L = ell/32 limbs per Z_q element, least significant limb first. Row i read as
one little-endian bit string is exactly row i of BitDecomp(C').

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
import numpy as np

from . import prng

GATE_CODES = {
    # (c0, c1, c2, c3): plaintext identities c0 + c1 a + c2 b + c3 ab
    "NOT": (1, -1, 0, 0),   # 1 - a
    "AND": (0, 0, 0, 1),    # ab
    "NAND": (1, 0, 0, -1),  # 1 - ab  (GSW'13's own gate)
    "OR": (0, 1, 1, -1),    # a + b - ab
    "XOR": (0, 1, 1, -2),   # a + b - 2ab
    "NOR": (1, -1, -1, 1),  # 1 - a - b + ab
    "XNOR": (1, -1, -1, 2),  # 1 - a - b + 2ab
    # a + b for two bits that are never both 1 (the carries of a full adder):
    # linear, no product; equals OR on every input it is applied to
    "XADD": (0, 1, 1, 0),
    # beta C for a public bit beta (refresh: a bootstrapping-key ciphertext
    # selected by a bit of the refreshed ciphertext); linear
    "SEL1": (0, 1, 0, 0),
    "SEL0": (0, 0, 0, 0),
}


class Params:
    """Scheme parameters (n, ell, m, chi); chi = B means e uniform in [-B, B]."""

    def __init__(self, n, ell, m, chi):
        if ell % 32 != 0 or ell <= 0:
            raise ValueError("ell must be a positive multiple of 32")
        self.n, self.ell, self.m, self.chi = int(n), int(ell), int(m), int(chi)
        self.q = 1 << self.ell
        self.L = self.ell // 32
        self.Ng = (self.n + 1) * self.ell

    def __repr__(self):
        return f"Params(n={self.n}, ell={self.ell}, m={self.m}, chi={self.chi})"


# ----------------------------------------------------------------------------
# Z_q elements <-> limbs
# ----------------------------------------------------------------------------

def to_limbs(values, L):
    """Python ints (array-like, any shape) in [0, q) -> uint32 (..., L)."""
    vals = np.asarray(values, dtype=object)
    out = np.zeros(vals.shape + (L,), dtype=np.uint32)
    for idx in np.ndindex(vals.shape):
        v = int(vals[idx])
        for l in range(L):
            out[idx + (l,)] = (v >> (32 * l)) & 0xFFFFFFFF
    return out


def from_limbs(limbs):
    """uint32 (..., L) -> object array (...) of Python ints."""
    limbs = np.asarray(limbs, dtype=np.uint32)
    shape = limbs.shape[:-1]
    out = np.empty(shape, dtype=object)
    for idx in np.ndindex(shape):
        v = 0
        for l, w in enumerate(limbs[idx]):
            v |= int(w) << (32 * l)
        out[idx] = v
    return out


def _digits16(ct):
    """uint32 limbs (..., L) -> int64 16-bit digits (..., 2L), low first."""
    lo = (ct & np.uint32(0xFFFF)).astype(np.int64)
    hi = (ct >> np.uint32(16)).astype(np.int64)
    return np.stack([lo, hi], axis=-1).reshape(ct.shape[:-1] + (2 * ct.shape[-1],))


def _normalize16(S, L):
    """Integers given as sum_d S[..., d] 2^(16 d) (int64, any sign) -> limbs mod 2^(32 L).

    Plain carry propagation digit by digit; numpy's >> on int64 is a floor
    shift, so negative sums wrap exactly as the mod-q definition requires.
    """
    D = S.shape[-1]
    digits = np.zeros(S.shape, dtype=np.int64)
    carry = np.zeros(S.shape[:-1], dtype=np.int64)
    for d in range(D):
        v = S[..., d] + carry
        digits[..., d] = v & 0xFFFF
        carry = v >> 16
    digits = digits.reshape(S.shape[:-1] + (L, 2))
    return (digits[..., 0] | (digits[..., 1] << 16)).astype(np.uint32)


def bits(ct):
    """BitDecomp of every row of a compressed ciphertext -> (Ng, Ng) uint8."""
    Ng = ct.shape[0]
    b = np.unpackbits(np.ascontiguousarray(ct).astype("<u4").view(np.uint8), bitorder="little")
    return b.reshape(Ng, -1)


def gadget(p):
    """P with P[j ell + b][j] = 2^b, shape (Ng, n+1, L)."""
    G = np.zeros((p.Ng, p.n + 1, p.L), dtype=np.uint32)
    for i in range(p.Ng):
        j, b = divmod(i, p.ell)
        G[i, j, b // 32] = np.uint32(1 << (b % 32))
    return G


def zero_ct(p):
    """Trivial encryption of 0 (the zero matrix)."""
    return np.zeros((p.Ng, p.n + 1, p.L), dtype=np.uint32)


def one_ct(p):
    """Trivial encryption of 1 (the gadget P, i.e. Flatten(I))."""
    return gadget(p)


def product(A, Bm, L):
    """BitDecomp(A) . Bm mod 2^(32 L), rows of Bm being Z_q vectors.

    A: (Ng, n+1, L) limbs.  Bm: (K, c, L) limbs with K = Ng.  The matrix
    product is carried out in float64 on 16-bit digits: every partial sum is
    an integer below K * 2^16 < 2^53, so BLAS returns it exactly.
    """
    bitm = bits(A).astype(np.float64)
    K, c = Bm.shape[0], Bm.shape[1]
    Bd = _digits16(Bm).reshape(K, c * 2 * L).astype(np.float64)
    S = np.rint(bitm @ Bd).astype(np.int64).reshape(A.shape[0], c, 2 * L)
    return _normalize16(S, L)


def lincomb(terms, L):
    """sum_k c_k X_k mod 2^(32 L) for small integer c_k and limb arrays X_k."""
    S = None
    for c, X in terms:
        if c == 0:
            continue
        t = c * _digits16(X)
        S = t if S is None else S + t
    if S is None:
        raise ValueError("empty linear combination")
    return _normalize16(S, L)


def gate(p, A, B, code):
    """Compressed GSW gate: c0 P + c1 A + c2 B + c3 BitDecomp(A) B  (mod q).

    ``A`` is the bit-decomposed (left) operand. For a unary gate pass B=None.
    """
    c0, c1, c2, c3 = code
    terms = [(c0, gadget(p)), (c1, A)]
    if B is not None:
        terms.append((c2, B))
    if c3 != 0:
        terms.append((c3, product(A, B, p.L)))
    if all(c == 0 for c, _ in terms):
        return zero_ct(p)
    return lincomb(terms, p.L)


# ----------------------------------------------------------------------------
# Keys, encryption, decryption (compressed form)
# ----------------------------------------------------------------------------

def _zq_from_stream(state, index, p):
    """Element number ``index`` of the uniform Z_q stream ``state``."""
    W = (p.ell + 63) // 64
    v = 0
    for w in range(W):
        v |= prng.out(state, index * W + w) << (64 * w)
    return v & (p.q - 1)


class Keys:
    """Secret t (and s = (1, -t)), public A = [B t + e | B], and the error e."""

    def __init__(self, p, seed):
        self.p = p
        kt = prng.key(seed, prng.DOMAIN_T)
        kb = prng.key(seed, prng.DOMAIN_B)
        ke = prng.key(seed, prng.DOMAIN_E)
        self.t = [_zq_from_stream(kt, j, p) for j in range(p.n)]
        self.s = [1] + [(-tj) % p.q for tj in self.t]
        self.Bmat = [[_zq_from_stream(kb, r * p.n + j, p) for j in range(p.n)] for r in range(p.m)]
        width = 2 * p.chi + 1
        self.e = [(prng.out(ke, r) % width) - p.chi for r in range(p.m)]
        A = []
        for r in range(p.m):
            b = (sum(self.Bmat[r][j] * self.t[j] for j in range(p.n)) + self.e[r]) % p.q
            A.append([b] + list(self.Bmat[r]))
        self.A = A                                   # m x (n+1) Python ints
        self.A_limbs = to_limbs(np.array(A, dtype=object), p.L)  # (m, n+1, L)
        self.v = [(1 << b) * self.s[j] % p.q for j in range(p.n + 1) for b in range(p.ell)]


def r_matrix(p, enc_seed, ct_index):
    """R in {0,1}^{Ng x m}: bit (i m + k) of the ciphertext's stream, LSB first."""
    nbits = p.Ng * p.m
    w = prng.words(prng.ct_key(enc_seed, ct_index), 0, (nbits + 63) // 64)
    b = np.unpackbits(w.astype("<u8").view(np.uint8), bitorder="little")[:nbits]
    return b.reshape(p.Ng, p.m)


def encrypt(keys, mu, enc_seed, ct_index):
    """C' = R A + mu P (mod q) for the bit ``mu`` (GSW Enc, compressed)."""
    p = keys.p
    R = r_matrix(p, enc_seed, ct_index).astype(np.float64)
    Ad = _digits16(keys.A_limbs).reshape(p.m, (p.n + 1) * 2 * p.L).astype(np.float64)
    S = np.rint(R @ Ad).astype(np.int64).reshape(p.Ng, p.n + 1, 2 * p.L)
    if mu:
        S = S + _digits16(gadget(p))
    return _normalize16(S, p.L)


def phase(keys, ct, row):
    """<C'_row, s> mod q."""
    p = keys.p
    vals = from_limbs(ct[row])
    return sum(int(vals[j]) * keys.s[j] for j in range(p.n + 1)) % p.q


def decrypt(keys, ct):
    """mu = 1 iff q/4 <= <C'_{ell-1}, s> < 3q/4 (v_{ell-1} = q/2)."""
    p = keys.p
    x = phase(keys, ct, p.ell - 1)
    return 1 if p.q // 4 <= x < 3 * p.q // 4 else 0


def noise(keys, ct, mu):
    """Exact noise vector e = C' s - mu v, centred into (-q/2, q/2]."""
    p = keys.p
    vals = from_limbs(ct)
    e = []
    for i in range(p.Ng):
        x = (sum(int(vals[i, j]) * keys.s[j] for j in range(p.n + 1)) - mu * keys.v[i]) % p.q
        if x > p.q // 2:
            x -= p.q
        e.append(x)
    return e


# ----------------------------------------------------------------------------
# Literal N x N form (tiny parameters only): the pin of the compressed form
# ----------------------------------------------------------------------------

def bitdecomp_vec(vec, p):
    return [(int(vec[j]) >> b) & 1 for j in range(len(vec)) for b in range(p.ell)]


def bitdecomp_inv_vec(x, p):
    k = len(x) // p.ell
    return [sum(int(x[j * p.ell + b]) << b for b in range(p.ell)) % p.q for j in range(k)]


def flatten(X, p):
    return [bitdecomp_vec(bitdecomp_inv_vec(row, p), p) for row in X]


def literal_encrypt(keys, mu, enc_seed, ct_index):
    p = keys.p
    R = r_matrix(p, enc_seed, ct_index)
    RA = [[sum(int(R[i, k]) * keys.A[k][j] for k in range(p.m)) % p.q for j in range(p.n + 1)]
          for i in range(p.Ng)]
    M = [bitdecomp_vec(row, p) for row in RA]
    for i in range(p.Ng):
        M[i][i] += mu
    return flatten(M, p)


def literal_gate(C1, C2, code, p):
    c0, c1, c2, c3 = code
    N = p.Ng
    out = []
    for i in range(N):
        row = []
        for j in range(N):
            v = c0 * (1 if i == j else 0) + c1 * C1[i][j]
            if C2 is not None:
                v += c2 * C2[i][j]
                if c3:
                    v += c3 * sum(C1[i][k] * C2[k][j] for k in range(N))
            row.append(v)
        out.append(row)
    return flatten(out, p)


def literal_decrypt(keys, C):
    p = keys.p
    x = sum(C[p.ell - 1][k] * keys.v[k] for k in range(p.Ng)) % p.q
    return 1 if p.q // 4 <= x < 3 * p.q // 4 else 0


def literal_to_compressed(C, p):
    """BitDecomp^-1 of every row -> (Ng, n+1, L) limbs."""
    return to_limbs(np.array([bitdecomp_inv_vec(row, p) for row in C], dtype=object), p.L)
