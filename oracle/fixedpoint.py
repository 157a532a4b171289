"""Fixed-point arithmetic, closed-form integer FFT, FP64 DFT, error bound.

* Quantisation (Sec. 4 fixed point; Sec. 5 "truncation"): raw = floor(x 2^f),
  kept as an F-bit two's-complement word (wraps mod 2^F).
* Fixed-point product (Lemma 9): the middle bits [f, f+F) of the 2F-style
  product, i.e. floor(x w / 2^f) mod 2^F for signed x, w.
* The closed-form integer FFT applies exactly those word operations in the
  radix-2 DIT order of Sec. 4; the gate circuit must reproduce it bit for bit.
* ``dft_fp64`` is the O(N^2) definition of the DFT in double precision.
* ``error_bound`` is Theorem 2: Delta (N/2)(log N + X_b + 1), Delta = 2^-f.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
import math

from .circuit import bitrev, twiddles


def wrap(v, F):
    """Signed value of v mod 2^F."""
    v %= 1 << F
    return v - (1 << F) if v >= 1 << (F - 1) else v


def quantize(x, F, f):
    return wrap(math.floor(x * (1 << f)), F)


def to_bits(v, F):
    return [(v >> i) & 1 for i in range(F)]      # Python >> on negatives: two's complement


def from_bits(bits):
    F = len(bits)
    return wrap(sum(b << i for i, b in enumerate(bits)), F)


def mul_fix(x, w, F, f):
    return wrap((x * w) >> f, F)


def fft_int(re, im, F, f):
    """Integer radix-2 DIT FFT with the circuit's word operations."""
    N = len(re)
    logN = N.bit_length() - 1
    tw = twiddles(N, f)
    a = [(re[bitrev(i, logN)], im[bitrev(i, logN)]) for i in range(N)]
    m = 2
    while m <= N:
        h = m // 2
        for k in range(0, N, m):
            for j in range(h):
                Wr, Wi = tw[j * (N // m)]
                (ur, ui), (xr, xi) = a[k + j], a[k + j + h]
                tr = wrap(mul_fix(xr, Wr, F, f) - mul_fix(xi, Wi, F, f), F)
                ti = wrap(mul_fix(xi, Wr, F, f) + mul_fix(xr, Wi, F, f), F)
                a[k + j] = (wrap(ur + tr, F), wrap(ui + ti, F))
                a[k + j + h] = (wrap(ur - tr, F), wrap(ui - ti, F))
        m *= 2
    return [x[0] for x in a], [x[1] for x in a]


def fft2_int(re, im, N1, N2, F, f):
    """Row-column 2-D integer FFT, sample k = r * N2 + c: rows, then columns."""
    re, im = list(re), list(im)
    if N2 > 1:
        for r in range(N1):
            sl = slice(r * N2, (r + 1) * N2)
            re[sl], im[sl] = fft_int(re[sl], im[sl], F, f)
    if N1 > 1:
        for col in range(N2):
            idx = [r * N2 + col for r in range(N1)]
            cr, ci = fft_int([re[i] for i in idx], [im[i] for i in idx], F, f)
            for r, i in enumerate(idx):
                re[i], im[i] = cr[r], ci[r]
    return re, im


def dft_fp64(re, im):
    """X_k = sum_n x_n exp(-2 pi i k n / N), straight from the definition."""
    N = len(re)
    Xr, Xi = [], []
    for k in range(N):
        sr = si = 0.0
        for n in range(N):
            ang = -2.0 * math.pi * ((k * n) % N) / N
            c, s = math.cos(ang), math.sin(ang)
            sr += re[n] * c - im[n] * s
            si += re[n] * s + im[n] * c
        Xr.append(sr)
        Xi.append(si)
    return Xr, Xi


def dft2_fp64(re, im, N1, N2):
    re, im = list(re), list(im)
    for r in range(N1):
        sl = slice(r * N2, (r + 1) * N2)
        re[sl], im[sl] = dft_fp64(re[sl], im[sl])
    for col in range(N2):
        idx = [r * N2 + col for r in range(N1)]
        cr, ci = dft_fp64([re[i] for i in idx], [im[i] for i in idx])
        for r, i in enumerate(idx):
            re[i], im[i] = cr[r], ci[r]
    return re, im


def error_bound(N, f, Xb):
    """Theorem 2: Delta * (N/2) * (log2 N + X_b + 1)."""
    return 2.0 ** (-f) * (N / 2) * (math.log2(N) + Xb + 1)


def fft_int_overflows(re, im, F, f):
    """True if the exact (unwrapped) integer DIT FFT leaves the F-bit range."""
    N = len(re)
    logN = N.bit_length() - 1
    tw = twiddles(N, f)
    lo, hi = -(1 << (F - 1)), (1 << (F - 1)) - 1
    a = [(re[bitrev(i, logN)], im[bitrev(i, logN)]) for i in range(N)]
    m = 2
    while m <= N:
        h = m // 2
        for k in range(0, N, m):
            for j in range(h):
                Wr, Wi = tw[j * (N // m)]
                (ur, ui), (xr, xi) = a[k + j], a[k + j + h]
                vals = [(xr * Wr) >> f, (xi * Wi) >> f, (xi * Wr) >> f, (xr * Wi) >> f]
                tr = vals[0] - vals[1]
                ti = vals[2] + vals[3]
                new = [ur + tr, ui + ti, ur - tr, ui - ti]
                if any(v < lo or v > hi for v in vals + [tr, ti] + new):
                    return True
                a[k + j], a[k + j + h] = (new[0], new[1]), (new[2], new[3])
        m *= 2
    return False
