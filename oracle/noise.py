"""Static worst-case noise bound of a circuit under the compressed GSW gate.

Multiplying C' s out for a gate c0 P + c1 A' + c2 B' + c3 BitDecomp(A') B'
(messages mu_A, mu_B in {0,1}, noises e_A, e_B) gives the noise
    c1 e_A + c2 e_B + c3 (mu_B e_A + BitDecomp(A') e_B),
so with |BitDecomp(A') e_B| <= Ng |e_B| the infinity norm is at most
    (|c1| + |c3|) E_A + (|c2| + |c3| Ng) E_B.
Fresh ciphertexts carry R e with R binary, |R e| <= m chi. Trivial constants
carry none. Decryption is correct while the noise stays below q/4 (the
decision regions of Dec are [q/4, 3q/4) around q/2 and its complement around
0). This is the "noise management" the paper leaves to the scheme (Sec. 5
closes by pointing at refreshing); the leveled reading sizes q from it.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from . import gsw
from .evaluate import operands


def fresh_bound(p):
    """Noise bound of a fresh encryption R A + mu P: R e with R binary, m chi."""
    return p.m * p.chi


def gate_bound(code, EA, EB, Ng):
    """Noise bound of the compressed gate (c0, c1, c2, c3) on operands with
    bounds EA (the bit-decomposed operand A) and EB."""
    c0, c1, c2, c3 = code
    return (abs(c1) + abs(c3)) * EA + (abs(c2) + abs(c3) * Ng) * EB


def wire_bounds(c, p):
    """Exact integer noise bound of every wire (list indexed by wire)."""
    E = [0] * len(c.depth)
    for w in c.inputs:
        E[w] = fresh_bound(p)

    def get(w):
        return 0 if w < 0 else E[w]

    for op, a, b, o in c.gates:
        A, B = operands(c, a, b)
        EB = 0 if B is None else get(B)
        E[o] = gate_bound(gsw.GATE_CODES[op], get(A), EB, p.Ng)
    return E


def max_bound(c, p):
    E = wire_bounds(c, p)
    return max(E) if E else 0


def smallest_ell(c, n, chi, m_of_ell=None, limit=8192):
    """Smallest ell (multiple of 32) with max wire bound < q/4; m = Ng unless given."""
    ell = 32
    while ell <= limit:
        Ng = (n + 1) * ell
        m = Ng if m_of_ell is None else m_of_ell(ell)
        p = gsw.Params(n, ell, m, chi)
        if max_bound(c, p) < p.q // 4:
            return ell
        ell += 32
    return None
