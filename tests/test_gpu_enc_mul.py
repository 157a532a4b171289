"""GPU parity of the encrypted-operand multiplier (word plans and the FFT with
encrypted twiddles) against the oracle, ciphertext for ciphertext."""
import math
import random

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1611_08769_gb300 as sf  # noqa: E402
from oracle import circuit, evaluate, fixedpoint as fx, gsw  # noqa: E402
from paper_1611_08769_gb300 import build as sfbuild  # noqa: E402
from synthetic import image_2d, signal_1d  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sfbuild.build()


def _run(plan, d_in):
    info = plan.info
    out = torch.zeros((info["outputs"], info["ct_words"]), dtype=torch.int32, device="cuda")
    scratch = torch.empty(max(1, info["scratch_bytes"] // 4), dtype=torch.int32, device="cuda")
    plan.eval_fft(d_in, out, scratch)
    plan.check()
    return out.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("flags", [0, sf.PLAN_INT_KERNEL])
def test_word_multiply_bit_exact(flags):
    """8 encrypted 8-bit 4.4 products at the smallest noisy ell, both kernels."""
    op, F, f, count = sf.WORD_MUL, 8, 4, 8
    sp = sf.param_set("P1", sf.word_min_ell(op, F, f))
    p = gsw.Params(sp.n, sp.ell, sp.m, sp.chi)
    rng = random.Random(21)
    xs = [rng.randint(-128, 127) for _ in range(count)]
    ys = [rng.randint(-128, 127) for _ in range(count)]
    keys = sf.keygen(sp, 8)
    d_in = torch.zeros((2 * count * F, sf.ct_words(sp)), dtype=torch.int32, device="cuda")
    sf.encrypt_bits_device(sp, torch.from_numpy(keys.public().view(np.int32)).cuda(),
                           [x / 2 ** f for x in xs], [y / 2 ** f for y in ys], F, f, 3, d_in)
    plan = sf.Plan.words(sp, op, count, F, f, flags)
    got = _run(plan, d_in).reshape(count * F, p.Ng, p.n + 1, p.L)
    ko = gsw.Keys(p, 8)
    c = circuit.word_circuit("mule", F, f)
    for k, (x, y) in enumerate(zip(xs, ys)):
        bits = fx.to_bits(x, F) + fx.to_bits(y, F)
        cts = [gsw.encrypt(ko, b, 3, 2 * k * F + j) for j, b in enumerate(bits)]
        want = evaluate.eval_encrypted(c, p, cts)
        assert np.array_equal(got[k * F:(k + 1) * F], want), k
        dec = [gsw.decrypt(ko, ct) for ct in want]
        assert fx.from_bits(dec) == fx.wrap(math.floor(x * y / 2 ** f), F)


@pytest.mark.parametrize("pset,N1,N2,F,f,flags", [
    ("P1", 2, 1, 4, 1, 0), ("P1", 2, 1, 4, 1, sf.PLAN_INT_KERNEL), ("P0", 4, 4, 8, 3, 0)])
def test_fft_encrypted_twiddles_bit_exact(pset, N1, N2, F, f, flags):
    ell = sf.min_ell(N1, N2, F, f, n=1, chi=1, enc_twiddle=True) if pset == "P1" else None
    sp = sf.param_set(pset, ell)
    p = gsw.Params(sp.n, sp.ell, sp.m, sp.chi)
    re_, im_ = signal_1d(N1, -1, 1, 9) if N2 == 1 else image_2d(N1, N2, 9)
    M = max(N1, N2)
    wr, wi = sf.twiddles(M, f)
    re_all = list(re_) + [w / 2 ** f for w in wr.tolist()]
    im_all = list(im_) + [w / 2 ** f for w in wi.tolist()]
    keys = sf.keygen(sp, 9)
    n_in = (N1 * N2 + M // 2) * 2 * F
    d_in = torch.zeros((n_in, sf.ct_words(sp)), dtype=torch.int32, device="cuda")
    sf.encrypt_bits_device(sp, torch.from_numpy(keys.public().view(np.int32)).cuda(),
                           re_all, im_all, F, f, 5, d_in)
    plan = sf.Plan(sp, N1, N2, F, f, flags | sf.PLAN_ENC_TWIDDLE)
    assert plan.info["inputs"] == n_in
    got = _run(plan, d_in).reshape(N1 * N2 * 2 * F, p.Ng, p.n + 1, p.L)
    ko = gsw.Keys(p, 9)
    c = circuit.fft_circuit(N1, N2, F, f, enc_twiddle=True)
    bits = []
    for r, i in zip(re_all, im_all):
        bits += fx.to_bits(fx.quantize(r, F, f), F) + fx.to_bits(fx.quantize(i, F, f), F)
    cts = [gsw.encrypt(ko, b, 5, j) for j, b in enumerate(bits)]
    want = evaluate.eval_encrypted(c, p, cts)
    assert np.array_equal(got, want)
    dec = [gsw.decrypt(ko, ct) for ct in got]
    assert dec == evaluate.eval_plain(c, bits)
