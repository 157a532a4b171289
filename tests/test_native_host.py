"""The native library on the host (no GPU): symbol table, circuit compiler,
keys, host encryption and decryption, each against the oracle.

The native circuit compiler is an independent C++ implementation of the same
canonical circuit; here its plaintext run of the compiled device program
(levels, scratch slots, fix-ups, adjusted coefficients) must equal the
oracle's plaintext circuit, and its statistics and static noise bound must
equal the oracle's.
"""
import os
import random
import re

import numpy as np
import pytest

import paper_1611_08769_gb300 as sf
from oracle import circuit, evaluate, fixedpoint as fx, gsw, noise
from paper_1611_08769_gb300 import build as sfbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    sfbuild.build()


def header_functions():
    txt = open(os.path.join(ROOT, "include", "sfft.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sfft_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = sf.native.lib()
    names = header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
        assert name in sf.native.SIGNATURES, f"{name} not bound in native.py"


def test_version_string():
    assert "sm_103a" in sf.version()


@pytest.mark.parametrize("N1,N2,F,f", [(2, 1, 4, 1), (8, 1, 8, 4), (16, 1, 12, 6), (4, 4, 8, 3),
                                       (4, 2, 6, 2)])
def test_compiled_program_matches_oracle_circuit(N1, N2, F, f):
    p = sf.param_set("P0")
    oc = circuit.fft_circuit(N1, N2, F, f)
    rng = random.Random(N1 * 100 + N2 * 10 + F)
    for _ in range(4):
        bits = [rng.randint(0, 1) for _ in range(len(oc.inputs))]
        want = evaluate.eval_plain(oc, bits)
        got = sf.program_eval_plain(p, N1, N2, F, f, bits)
        assert list(got) == want


@pytest.mark.parametrize("N1,N2,F,f", [(8, 1, 8, 4), (32, 1, 16, 8), (4, 4, 10, 4)])
def test_circuit_statistics_match_oracle(N1, N2, F, f):
    oc = circuit.fft_circuit(N1, N2, F, f)
    st = circuit.stats(oc)
    info = sf.circuit_info(sf.param_set("P0"), N1, N2, F, f)
    assert info["products"] == st["products"]
    assert info["levels"] == st["depth"]
    assert info["inputs"] == info["outputs"] == 2 * F * N1 * N2


@pytest.mark.parametrize("N1,N2,F,f", [(2, 1, 4, 1), (8, 1, 8, 4), (4, 4, 8, 3)])
def test_min_ell_and_noise_bound_match_oracle(N1, N2, F, f):
    oc = circuit.fft_circuit(N1, N2, F, f)
    ell = noise.smallest_ell(oc, n=1, chi=1)
    assert sf.min_ell(N1, N2, F, f, n=1, chi=1) == ell
    p = gsw.Params(1, ell, 2 * ell, 1)
    info = sf.circuit_info(sf.Params(1, ell, 2 * ell, 1), N1, N2, F, f)
    assert info["noise_bits"] == noise.max_bound(oc, p).bit_length()
    assert info["noise_ok"] == 1


@pytest.mark.parametrize("n,ell,m,chi", [(1, 32, 64, 0), (1, 64, 128, 1), (2, 32, 96, 1)])
def test_keys_and_host_encryption_match_oracle(n, ell, m, chi):
    ok = gsw.Keys(gsw.Params(n, ell, m, chi), seed=11)
    nk = sf.keygen(sf.Params(n, ell, m, chi), 11)
    assert np.array_equal(nk.public().reshape(ok.A_limbs.shape), ok.A_limbs)
    F, f = 4, 1
    re_, im_ = [0.75, -1.5], [2.25, -0.5]
    cts = sf.encrypt_bits(nk, re_, im_, F, f, enc_seed=3)
    k = 0
    for s in range(2):
        for part, x in enumerate((re_[s], im_[s])):
            for b, bit in enumerate(fx.to_bits(fx.quantize(x, F, f), F)):
                want = gsw.encrypt(ok, bit, 3, k)
                assert np.array_equal(cts[k].reshape(want.shape), want), (s, part, b)
                k += 1


def test_host_decryption_matches_oracle():
    p = gsw.Params(1, 64, 128, 1)
    ok = gsw.Keys(p, seed=2)
    nk = sf.keygen(sf.Params(1, 64, 128, 1), 2)
    F, f = 6, 2
    vals = [(1.25, -3.0), (-7.5, 0.5)]
    cts = []
    for s, (r, i) in enumerate(vals):
        for part, x in enumerate((r, i)):
            for b, bit in enumerate(fx.to_bits(fx.quantize(x, F, f), F)):
                cts.append(gsw.encrypt(ok, bit, 9, (2 * s + part) * F + b).reshape(-1))
    arr = np.stack(cts)
    W = (p.n + 1) * p.L
    rows = arr[:, (p.ell - 1) * W:p.ell * W]
    re_, im_, raw = sf.decrypt(nk, rows, W, 2, F, f)
    assert list(raw) == [fx.quantize(x, F, f) for pair in vals for x in pair]
    assert list(re_) == [v[0] for v in vals] and list(im_) == [v[1] for v in vals]
    flat = arr.reshape(-1)[(p.ell - 1) * W:]      # row ell-1 of ciphertext 0 onwards
    re2, im2, raw2 = sf.decrypt(nk, flat, arr.shape[1], 2, F, f)
    assert list(raw2) == list(raw)


def test_invalid_arguments_fail_loudly():
    with pytest.raises(sf.SfftError):
        sf.circuit_info(sf.param_set("P0"), 6, 1, 8, 4)      # not a power of two
    with pytest.raises(sf.SfftError):
        sf.circuit_info(sf.Params(1, 40), 8, 1, 8, 4)        # ell not a multiple of 32
    with pytest.raises(sf.SfftError):
        sf.keygen(sf.Params(0, 32), 1)
