"""Seeded synthetic workloads (plain doubles and request mixes, no FHE arithmetic).

These generators are the only code shared by the oracle-based tests and the
GPU path's tests and benchmark. They draw plaintext signals and request
parameters from numpy's PCG64 with fixed seeds; quantisation, encryption and
everything after it happen on each side separately.

Stand-ins for the paper's data (Sec. 6): its random 1-D signals and its ten
16 x 16 test images are not published, so seeded uniform signals and
uniform-pixel images of the same shapes replace them.
"""
from dataclasses import dataclass, field
from typing import List

import numpy as np


def signal_1d(N, lo, hi, seed):
    """Real signal of N samples uniform in [lo, hi); imaginary part zero."""
    rng = np.random.default_rng(seed)
    re = rng.uniform(lo, hi, size=N)
    return re.astype(np.float64), np.zeros(N, dtype=np.float64)


def image_2d(N1, N2, seed):
    """N1 x N2 image of integer pixels uniform in 0..255, mapped to p / 255."""
    rng = np.random.default_rng(seed)
    pix = rng.integers(0, 256, size=N1 * N2)
    return (pix / 255.0).astype(np.float64), np.zeros(N1 * N2, dtype=np.float64)


@dataclass
class Request:
    """One encrypted-FFT request of a batch or a serving trace."""
    N1: int
    N2: int
    F: int
    f: int
    key_set: int
    seed: int
    arrival_s: float = 0.0
    re: np.ndarray = field(default=None, repr=False)
    im: np.ndarray = field(default=None, repr=False)


def batch_requests(count=256, seed=4, sizes=(16, 32, 64, 128), widths=(16, 24), key_sets=4):
    """Independent 1-D FFTs: N uniform over ``sizes``, F over ``widths``, f = F/2,
    inputs uniform in [-1, 1), key set uniform over ``key_sets``."""
    rng = np.random.default_rng(seed)
    out: List[Request] = []
    for r in range(count):
        N = int(rng.choice(sizes))
        F = int(rng.choice(widths))
        ks = int(rng.integers(0, key_sets))
        s = int(rng.integers(0, 2**31))
        re, im = signal_1d(N, -1.0, 1.0, s)
        out.append(Request(N, 1, F, F // 2, ks, s, 0.0, re, im))
    return out


def serving_trace(count, rate_per_s, seed=5, key_sets=8, F=16):
    """Poisson arrivals of a mix of 1-D (N in 8..256) and 2-D (8x8..32x32) FFTs.

    1-D requests use 8 fraction bits and inputs in [-1, 1); 2-D requests are
    images in [0, 1] with log2(pixels) + 2 integer bits.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out: List[Request] = []
    for r in range(count):
        t += float(rng.exponential(1.0 / rate_per_s))
        ks = int(rng.integers(0, key_sets))
        s = int(rng.integers(0, 2**31))
        if rng.random() < 0.75:
            N = int(rng.choice([8, 16, 32, 64, 128, 256]))
            re, im = signal_1d(N, -1.0, 1.0, s)
            out.append(Request(N, 1, F, F // 2, ks, s, t, re, im))
        else:
            n = int(rng.choice([8, 16, 32]))
            int_bits = int(np.log2(n * n)) + 2
            re, im = image_2d(n, n, s)
            out.append(Request(n, n, F, F - int_bits, ks, s, t, re, im))
    return out
