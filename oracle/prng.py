"""Counter-based SplitMix64 streams for keys and encryption randomness.

The paper does not say how its randomness is drawn (Sec. 3 only cites the
scheme). To make two independent implementations produce the same keys and
ciphertexts, every random value is a pure function of (seed, domain, counter):

    mix64(z)        the SplitMix64 output finaliser (Steele, Lea, Flood,
                    OOPSLA 2014; the 64-bit variant with shifts 30/27/31)
    out(state, k)   = mix64(state + (k+1) * GAMMA)   (k-th output of the
                    SplitMix64 generator started at ``state``)
    key(seed, d)    = mix64(seed XOR d * TAG_MUL)     for domain d

Domains: 1 = secret t, 2 = public matrix B, 3 = error e, 4 = encryption
matrices R. The R key of ciphertext number c is out(key(encseed, 4), c).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
TAG_MUL = 0xD1B54A32D192ED03

DOMAIN_T, DOMAIN_B, DOMAIN_E, DOMAIN_R = 1, 2, 3, 4


def mix64(z):
    """SplitMix64 finaliser on a Python int (mod 2^64)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def out(state, k):
    """k-th (0-based) output of SplitMix64 seeded with ``state``."""
    return mix64((state + (k + 1) * GAMMA) & MASK64)


def key(seed, domain):
    return mix64((seed ^ ((domain * TAG_MUL) & MASK64)) & MASK64)


def ct_key(enc_seed, ct_index):
    """Stream key of the R matrix of ciphertext number ``ct_index``."""
    return out(key(enc_seed, DOMAIN_R), ct_index)


def words(state, start, count):
    """Outputs start .. start+count-1 of the stream ``state`` as uint64 array.

    Same function as ``out`` applied elementwise, written with numpy uint64
    (wrapping) arithmetic so that large R matrices are generated quickly.
    """
    k = np.arange(start, start + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(state) + (k + np.uint64(1)) * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z
