"""GPU parity of ciphertext refresh: the bootstrapping key encrypted on the
device, noisy ciphertexts produced by a GPU word plan, refreshed on both gate
kernels and compared ciphertext for ciphertext with the oracle."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1611_08769_gb300 as sf  # noqa: E402
from oracle import circuit, evaluate, fixedpoint as fx, gsw, noise, refresh  # noqa: E402
from paper_1611_08769_gb300 import build as sfbuild  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sfbuild.build()


def _buffers(info):
    out = torch.zeros((info["outputs"], info["ct_words"]), dtype=torch.int32, device="cuda")
    scratch = torch.empty(max(1, info["scratch_bytes"] // 4), dtype=torch.int32, device="cuda")
    return out, scratch


_ORACLE = {}   # xcarry -> (sources, plain bits, refreshed ciphertexts): shared by both kernels


@pytest.mark.parametrize("xcarry,flags", [(True, 0), (True, sf.PLAN_INT_KERNEL), (False, 0)])
def test_refresh_bit_exact(xcarry, flags):
    variant = sf.PLAN_XCARRY if xcarry else 0
    ell = sf.refresh_min_ell(1, 1, xcarry=xcarry)
    sp = sf.param_set("P1", ell)
    p = gsw.Params(sp.n, sp.ell, sp.m, sp.chi)
    keys = sf.keygen(sp, 41)
    d_pub = torch.from_numpy(keys.public().view(np.int32)).cuda()
    cw = sf.ct_words(sp)

    # noisy sources: two 4-bit 2.1 encrypted products (outputs of a GPU word plan)
    F, f, xs, ys = 4, 1, [-7, 5], [3, -6]
    d_in = torch.zeros((2 * len(xs) * F, cw), dtype=torch.int32, device="cuda")
    sf.encrypt_bits_device(sp, d_pub, [x / 2 ** f for x in xs], [y / 2 ** f for y in ys], F, f,
                           2, d_in)
    mul = sf.Plan.words(sp, sf.WORD_MUL, len(xs), F, f, variant)
    src, scratch = _buffers(mul.info)
    mul.eval_fft(d_in, src, scratch)
    mul.check()

    # bootstrapping key, refresh of every source bit
    kb = keys.key_bits()
    d_bk = torch.zeros((len(kb), cw), dtype=torch.int32, device="cuda")
    sf.encrypt_raw_bits_device(sp, d_pub, kb, 9, d_bk)
    count = src.shape[0]
    plan = sf.Plan.refresher(sp, count, flags | variant)
    out, scratch2 = _buffers(plan.info)
    plan.refresh(d_bk, src, out, scratch2)
    plan.check()
    got = out.cpu().numpy().view(np.uint32).reshape(count, p.Ng, p.n + 1, p.L)

    # oracle: same sources, key and bootstrapping key
    ko = gsw.Keys(p, 41)
    bk = refresh.bootstrap_key(ko, 9)
    if xcarry not in _ORACLE:
        wc = circuit.word_circuit("mule", F, f, xcarry=xcarry)
        srcs, bits = [], []
        for k, (x, y) in enumerate(zip(xs, ys)):
            b = fx.to_bits(x, F) + fx.to_bits(y, F)
            cts = [gsw.encrypt(ko, v, 2, 2 * k * F + j) for j, v in enumerate(b)]
            srcs += list(evaluate.eval_encrypted(wc, p, cts))
            bits += fx.to_bits(fx.wrap(math.floor(x * y / 2 ** f), F), F)
        rc = refresh.refresh_circuit(p, [refresh.public_row(ct, p) for ct in srcs], xcarry=xcarry)
        _ORACLE[xcarry] = (srcs, bits, evaluate.eval_encrypted(rc, p, bk))
    srcs, bits, want = _ORACLE[xcarry]
    assert np.array_equal(src.cpu().numpy().view(np.uint32).reshape(count, p.Ng, p.n + 1, p.L),
                          np.stack(srcs))
    assert np.array_equal(d_bk.cpu().numpy().view(np.uint32).reshape(len(kb), p.Ng, p.n + 1, p.L),
                          np.stack(bk))
    assert np.array_equal(got, want)
    bound = noise.max_bound(refresh.refresh_circuit(p, [None], xcarry=xcarry), p)
    for ct, mu in zip(got, bits):
        assert gsw.decrypt(ko, ct) == mu
        assert max(map(abs, gsw.noise(ko, ct, mu))) <= bound < p.q // 8


def test_refresh_at_full_size():
    """Refresh at the ell of the 64-point 16-bit workload (1056) in the launch
    configuration the bench times: too large for the oracle to evaluate gate
    by gate, so the outputs are checked by the properties the construction
    guarantees: each decrypts (oracle keys) to its source bit and its exact
    noise is within the static bound, which is below q/8."""
    ell = sf.min_ell(64, 1, 16, 8, n=1, chi=1)
    assert ell == 1056
    sp = sf.param_set("P1", ell)
    p = gsw.Params(sp.n, sp.ell, sp.m, sp.chi)
    keys = sf.keygen(sp, 77)
    d_pub = torch.from_numpy(keys.public().view(np.int32)).cuda()
    cw = sf.ct_words(sp)
    kb = keys.key_bits()
    d_bk = torch.zeros((len(kb), cw), dtype=torch.int32, device="cuda")
    sf.encrypt_raw_bits_device(sp, d_pub, kb, 3, d_bk)
    bits = np.array([1, 0, 1, 1], dtype=np.uint8)
    d_src = torch.zeros((len(bits), cw), dtype=torch.int32, device="cuda")
    sf.encrypt_raw_bits_device(sp, d_pub, bits, 4, d_src)
    plan = sf.Plan.refresher(sp, len(bits))
    assert plan.info["gate_kernel"] == sf.KERNEL_TC
    out, scratch = _buffers(plan.info)
    plan.refresh(d_bk, d_src, out, scratch)
    plan.check()
    got = out.cpu().numpy().view(np.uint32).reshape(len(bits), p.Ng, p.n + 1, p.L)
    ko = gsw.Keys(p, 77)
    bound = 1 << plan.info["noise_bits"]   # every output's noise is below it
    assert bound <= p.q // 8
    for ct, mu in zip(got, bits):
        assert gsw.decrypt(ko, ct) == mu
        assert max(map(abs, gsw.noise(ko, ct, int(mu)))) < bound
