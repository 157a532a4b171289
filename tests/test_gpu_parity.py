"""GPU parity: the CUDA path against the CPU oracle, bit for bit.

Ciphertext arithmetic is integer mod 2^ell, so every comparison here is
exact equality of uint32 limbs (no tolerance).
"""
import random

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1611_08769_gb300 as sf  # noqa: E402
from oracle import circuit, evaluate, fixedpoint as fx, gsw, noise  # noqa: E402
from paper_1611_08769_gb300 import build as sfbuild  # noqa: E402
from synthetic import image_2d, signal_1d  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sfbuild.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def host(t, shape):
    return t.cpu().numpy().view(np.uint32).reshape(shape)


CODES = {"XOR": (0, 1, 1, -2), "AND": (0, 0, 0, 1), "OR": (0, 1, 1, -1), "NAND": (1, 0, 0, -1),
         "MIX": (1, -1, 2, 3)}


GATE_CASES = [(1, 32, sf.KERNEL_INT), (1, 128, sf.KERNEL_INT), (1, 224, sf.KERNEL_INT),
              (2, 64, sf.KERNEL_INT), (1, 1056, sf.KERNEL_INT),
              (1, 128, sf.KERNEL_TC), (1, 224, sf.KERNEL_TC), (2, 64, sf.KERNEL_TC),
              (1, 1056, sf.KERNEL_TC), (1, 1216, sf.KERNEL_TC), (1, 1440, sf.KERNEL_TC),
              (1, 1984, sf.KERNEL_AUTO)]


@pytest.mark.parametrize("n,ell,kernel", GATE_CASES)
def test_gate_level_matches_oracle(n, ell, kernel):
    p = gsw.Params(n, ell, (n + 1) * ell, 0)
    sp = sf.Params(n, ell)
    shape = (p.Ng, n + 1, p.L)
    # ell 1056 and 1216: 24 gates of 17 and 19 tiles, more than one tile per CTA of the
    # persistent kernel (152 SMs), so both accumulator slots are compared; ell 1440: 8 gates
    # of 23 tiles, one A-tile buffer reloaded between a CTA's items (288 digit columns)
    G = 37 if ell <= 256 else (24 if ell <= 1216 else (8 if ell <= 1440 else 3))
    rng = np.random.default_rng(ell + n)
    A = rng.integers(0, 2**32, size=(G,) + shape, dtype=np.uint64).astype(np.uint32)
    B = rng.integers(0, 2**32, size=(G,) + shape, dtype=np.uint64).astype(np.uint32)
    names = list(CODES)
    code0, code1, flags = [], [], []
    for g in range(G):
        code0.append(sf.pack_code(*CODES[names[g % len(names)]]))
        code1.append(sf.pack_code(*CODES[names[(g + 2) % len(names)]]))
        flags.append((g % 2) | (2 if g % 3 else 0))
    dA, dB = dev(A), dev(B)
    o0 = torch.zeros_like(dA)
    o1 = torch.zeros_like(dA)
    sf.gate_level(sp, dA, dB, o0, o1, code0, code1, flags, kernel=kernel)
    torch.cuda.synchronize()
    got0, got1 = host(o0, A.shape), host(o1, A.shape)
    for g in range(G):
        Aval = gsw.gate(p, A[g], None, gsw.GATE_CODES["NOT"]) if flags[g] & 1 else A[g]
        for code, got, on in ((code0[g], got0, True), (code1[g], got1, bool(flags[g] & 2))):
            if not on:
                continue
            c = [((code >> (4 * k)) & 15) - (16 if (code >> (4 * k)) & 8 else 0) for k in range(4)]
            terms = [(c[0], gsw.gadget(p)), (c[1], A[g]), (c[2], B[g]),
                     (c[3], gsw.product(Aval, B[g], p.L))]
            want = gsw.lincomb(terms, p.L)
            assert np.array_equal(got[g], want), (g, c)


@pytest.mark.parametrize("name,ell", [("P0", None), ("P2", None), ("P1", 224)])
def test_device_encryption_matches_oracle(name, ell):
    sp = sf.param_set(name, ell)
    p = gsw.Params(sp.n, sp.ell, sp.m, sp.chi)
    keys = sf.keygen(sp, 7)
    ok = gsw.Keys(p, 7)
    re_, im_ = signal_1d(2, -1, 1, 3)
    F, f = 4, 2
    out = torch.zeros((2 * 2 * F, sf.ct_words(sp)), dtype=torch.int32, device="cuda")
    sf.encrypt_bits_device(sp, dev(keys.public()), re_, im_, F, f, 5, out)
    torch.cuda.synchronize()
    got = host(out, (2 * 2 * F, p.Ng, p.n + 1, p.L))
    for k in range(2):
        for part, x in enumerate((re_[k], im_[k])):
            for b, bit in enumerate(fx.to_bits(fx.quantize(x, F, f), F)):
                idx = (2 * k + part) * F + b
                assert np.array_equal(got[idx], gsw.encrypt(ok, bit, 5, idx)), idx


def _run_plan(sp, N1, N2, F, f, d_in, flags=0):
    plan = sf.Plan(sp, N1, N2, F, f, flags)
    info = plan.info
    out = torch.zeros((info["outputs"], info["ct_words"]), dtype=torch.int32, device="cuda")
    scratch = torch.empty(max(1, info["scratch_bytes"] // 4), dtype=torch.int32, device="cuda")
    plan.eval_fft(d_in, out, scratch)
    plan.check()
    return plan, out


def _oracle_fft(p, keys_o, re_, im_, N1, N2, F, f, enc_seed):
    c = circuit.fft_circuit(N1, N2, F, f)
    cts, bits = [], []
    for k in range(N1 * N2):
        for part, x in enumerate((re_[k], im_[k])):
            for b, bit in enumerate(fx.to_bits(fx.quantize(x, F, f), F)):
                cts.append(gsw.encrypt(keys_o, bit, enc_seed, (2 * k + part) * F + b))
                bits.append(bit)
    return c, bits, evaluate.eval_encrypted(c, p, cts)


def test_fft_8pt_toy_parameters_bit_exact():
    """8-point FFT, 8-bit 4.4 words, inputs U[-1,1), imag 0, toy parameters, seeds 0."""
    N, F, f = 8, 8, 4
    sp = sf.param_set("P0")
    p = gsw.Params(sp.n, sp.ell, sp.m, sp.chi)
    re_, im_ = signal_1d(N, -1, 1, 0)
    keys = sf.keygen(sp, 0)
    d_in = torch.zeros((N * 2 * F, sf.ct_words(sp)), dtype=torch.int32, device="cuda")
    sf.encrypt_bits_device(sp, dev(keys.public()), re_, im_, F, f, 0, d_in)
    plan, out = _run_plan(sp, N, 1, F, f, d_in)
    got = host(out, (N * 2 * F, p.Ng, p.n + 1, p.L))
    c, bits, want = _oracle_fft(p, gsw.Keys(p, 0), re_, im_, N, 1, F, f, 0)
    assert np.array_equal(got, want)
    W = (p.n + 1) * p.L
    rows = got.reshape(len(got), -1)[:, (p.ell - 1) * W:p.ell * W]
    _, _, raw = sf.decrypt(keys, rows, W, N, F, f)
    q = [fx.quantize(x, F, f) for x in re_]
    er, ei = fx.fft_int(q, [0] * N, F, f)
    assert list(raw) == [v for k in range(N) for v in (er[k], ei[k])]


@pytest.mark.parametrize("flags", [0, sf.PLAN_INT_KERNEL])
def test_fft_noisy_leveled_parameters_bit_exact(flags):
    """Noisy chi = 1 scheme with ell sized by the static bound (8-pt, 8-bit);
    tensor-core kernel (default) and integer kernel."""
    N, F, f = 8, 8, 4
    ell = sf.min_ell(N, 1, F, f, n=1, chi=1)
    sp = sf.param_set("P1", ell)
    p = gsw.Params(sp.n, sp.ell, sp.m, sp.chi)
    re_, im_ = signal_1d(N, -1, 1, 1)
    keys = sf.keygen(sp, 1)
    d_in = torch.zeros((N * 2 * F, sf.ct_words(sp)), dtype=torch.int32, device="cuda")
    sf.encrypt_bits_device(sp, dev(keys.public()), re_, im_, F, f, 2, d_in)
    plan, out = _run_plan(sp, N, 1, F, f, d_in, flags)
    got = host(out, (N * 2 * F, p.Ng, p.n + 1, p.L))
    ko = gsw.Keys(p, 1)
    c, bits, want = _oracle_fft(p, ko, re_, im_, N, 1, F, f, 2)
    assert np.array_equal(got, want)
    assert [gsw.decrypt(ko, ct) for ct in got] == evaluate.eval_plain(c, bits)


@pytest.mark.parametrize("flags", [0, sf.PLAN_INT_KERNEL])
def test_fft_exclusive_carry_variant_bit_exact(flags):
    """The exclusive-carry circuit (linear carry gates between product levels)
    at its own smallest ell, noisy chi = 1: tensor-core and integer kernels."""
    N, F, f = 8, 8, 4
    ell = sf.min_ell(N, 1, F, f, n=1, chi=1, xcarry=True)
    sp = sf.param_set("P1", ell)
    p = gsw.Params(sp.n, sp.ell, sp.m, sp.chi)
    re_, im_ = signal_1d(N, -1, 1, 6)
    keys = sf.keygen(sp, 6)
    d_in = torch.zeros((N * 2 * F, sf.ct_words(sp)), dtype=torch.int32, device="cuda")
    sf.encrypt_bits_device(sp, dev(keys.public()), re_, im_, F, f, 4, d_in)
    plan, out = _run_plan(sp, N, 1, F, f, d_in, flags | sf.PLAN_XCARRY)
    assert plan.info["gates_xadd"] > 0
    got = host(out, (N * 2 * F, p.Ng, p.n + 1, p.L))
    ko = gsw.Keys(p, 6)
    c = circuit.fft_circuit(N, 1, F, f, xcarry=True)
    cts, bits = [], []
    xr = [fx.quantize(float(x), F, f) for x in re_]
    xi = [fx.quantize(float(x), F, f) for x in im_]
    for k in range(N):
        for part, v in enumerate((xr[k], xi[k])):
            for b, bit in enumerate(fx.to_bits(v, F)):
                cts.append(gsw.encrypt(ko, bit, 4, (k * 2 + part) * F + b))
                bits.append(bit)
    want = evaluate.eval_encrypted(c, p, cts)
    assert np.array_equal(got, want)
    assert [gsw.decrypt(ko, ct) for ct in got] == evaluate.eval_plain(c, bits)


@pytest.mark.parametrize("pset,N1,N2,F,f,flags", [
    ("P1", 2, 1, 4, 1, 0), ("P1", 2, 1, 4, 1, sf.PLAN_INT_KERNEL), ("P0", 4, 4, 8, 3, 0)])
def test_fft_nand_variant_bit_exact(pset, N1, N2, F, f, flags):
    """The NAND-only circuit (every gate a GSW NAND product; Lemma 4): noisy
    chi = 1 at its own smallest ell (tensor-core and integer kernels), and a
    2-D transform at the toy parameters, through the plan and the graph-replayed
    batch."""
    ell = sf.min_ell(N1, N2, F, f, n=1, chi=1, nand=True) if pset == "P1" else None
    sp = sf.param_set(pset, ell)
    p = gsw.Params(sp.n, sp.ell, sp.m, sp.chi)
    re_, im_ = (signal_1d(N1, -1, 1, 7) if N2 == 1 else image_2d(N1, N2, 7))
    keys = sf.keygen(sp, 7)
    n_in = N1 * N2 * 2 * F
    d_in = torch.zeros((n_in, sf.ct_words(sp)), dtype=torch.int32, device="cuda")
    sf.encrypt_bits_device(sp, dev(keys.public()), re_, im_, F, f, 4, d_in)
    plan, out = _run_plan(sp, N1, N2, F, f, d_in, flags | sf.PLAN_NAND)
    assert plan.info["gates_xor"] > 0 and plan.info["gates_xadd"] == 0
    got = host(out, (n_in, p.Ng, p.n + 1, p.L))
    ko = gsw.Keys(p, 7)
    c = circuit.fft_circuit(N1, N2, F, f, nand=True)
    assert plan.info["products"] == circuit.stats(c)["products"]
    cts, bits = [], []
    for k in range(N1 * N2):
        for part, x in enumerate((re_[k], im_[k])):
            for b, bit in enumerate(fx.to_bits(fx.quantize(x, F, f), F)):
                cts.append(gsw.encrypt(ko, bit, 4, (2 * k + part) * F + b))
                bits.append(bit)
    want = evaluate.eval_encrypted(c, p, cts)
    assert np.array_equal(got, want)
    assert [gsw.decrypt(ko, ct) for ct in got] == evaluate.eval_plain(c, bits)

    batch = sf.Batch(sp, [(N1, N2, F, f)], flags | sf.PLAN_NAND)
    bi = batch.info
    d_out = torch.zeros((bi["outputs"], bi["ct_words"]), dtype=torch.int32, device="cuda")
    scratch = torch.empty(max(1, bi["scratch_bytes"] // 4), dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    for _ in range(2):   # capture, then replay
        batch.eval(d_in, d_out, scratch, stream)
    batch.check(stream)
    torch.cuda.synchronize()
    assert np.array_equal(host(d_out, (n_in, p.Ng, p.n + 1, p.L)), want)


def test_fft_2d_toy_parameters_bit_exact():
    N1, N2, F, f = 4, 4, 8, 3
    sp = sf.param_set("P0")
    p = gsw.Params(sp.n, sp.ell, sp.m, sp.chi)
    re_, im_ = image_2d(N1, N2, 3)
    keys = sf.keygen(sp, 3)
    d_in = torch.zeros((N1 * N2 * 2 * F, sf.ct_words(sp)), dtype=torch.int32, device="cuda")
    sf.encrypt_bits_device(sp, dev(keys.public()), re_, im_, F, f, 4, d_in)
    plan, out = _run_plan(sp, N1, N2, F, f, d_in)
    got = host(out, (N1 * N2 * 2 * F, p.Ng, p.n + 1, p.L))
    c, bits, want = _oracle_fft(p, gsw.Keys(p, 3), re_, im_, N1, N2, F, f, 4)
    assert np.array_equal(got, want)


def test_eval_fft_host_matches_device_path():
    N, F, f = 4, 6, 2
    sp = sf.param_set("P2")
    re_, im_ = signal_1d(N, -1, 1, 9)
    keys = sf.keygen(sp, 9)
    cw = sf.ct_words(sp)
    d_in = torch.zeros((N * 2 * F, cw), dtype=torch.int32, device="cuda")
    sf.encrypt_bits_device(sp, dev(keys.public()), re_, im_, F, f, 1, d_in)
    plan, out = _run_plan(sp, N, 1, F, f, d_in)
    h_in = d_in.cpu().pin_memory()
    h_out = torch.zeros_like(h_in).pin_memory()
    d_in2, d_out2 = torch.zeros_like(d_in), torch.zeros_like(out)
    scratch = torch.empty(max(1, plan.info["scratch_bytes"] // 4), dtype=torch.int32, device="cuda")
    plan.eval_fft_host(h_in, h_out, d_in2, d_out2, scratch)
    assert torch.equal(h_out, out.cpu())


def test_scratch_too_small_is_rejected():
    sp = sf.param_set("P0")
    plan = sf.Plan(sp, 4, 1, 6, 2)
    cw = plan.info["ct_words"]
    d_in = torch.zeros((plan.info["inputs"], cw), dtype=torch.int32, device="cuda")
    out = torch.zeros_like(d_in)
    small = torch.empty(8, dtype=torch.int32, device="cuda")
    with pytest.raises(sf.SfftError):
        plan.eval_fft(d_in, out, small)
