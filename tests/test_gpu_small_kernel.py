"""GPU parity of the small-ciphertext tensor-core kernel (Ng <= 256).

Every comparison is exact equality of uint32 limbs against the CPU oracle
(ciphertext arithmetic is integer mod 2^ell). The gate counts exceed the
number of SMs several times over, so every CTA runs several gates through its
shared-memory ring, its tensor-memory A stages and its accumulator slots, and
the last round is ragged.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1611_08769_gb300 as sf  # noqa: E402
from oracle import circuit, evaluate, fixedpoint as fx, gsw  # noqa: E402
from paper_1611_08769_gb300 import build as sfbuild  # noqa: E402
from synthetic import signal_1d  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sfbuild.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def host(t, shape):
    return t.cpu().numpy().view(np.uint32).reshape(shape)


CODES = [(0, 1, 1, -2), (0, 0, 0, 1), (0, 1, 1, -1), (1, 0, 0, -1), (1, -1, 2, 3), (-3, 7, -8, 5)]


def _oracle_gate(p, A, B, code, comp):
    Aval = gsw.gate(p, A, None, gsw.GATE_CODES["NOT"]) if comp else A
    terms = [(code[0], gsw.gadget(p)), (code[1], A), (code[2], B),
             (code[3], gsw.product(Aval, B, p.L))]
    return gsw.lincomb(terms, p.L)


def _run_level(n, ell, G, kernel, seed, extreme=False):
    p = gsw.Params(n, ell, (n + 1) * ell, 0)
    sp = sf.Params(n, ell)
    shape = (G, p.Ng, n + 1, p.L)
    rng = np.random.default_rng(seed)
    if extreme:   # all-ones operands: every digit sum at its maximum Ng * 255
        A = np.full(shape, 0xFFFFFFFF, dtype=np.uint32)
        B = np.full(shape, 0xFFFFFFFF, dtype=np.uint32)
    else:
        A = rng.integers(0, 2**32, size=shape, dtype=np.uint64).astype(np.uint32)
        B = rng.integers(0, 2**32, size=shape, dtype=np.uint64).astype(np.uint32)
    code0 = [sf.pack_code(*CODES[g % len(CODES)]) for g in range(G)]
    code1 = [sf.pack_code(*CODES[(g + 3) % len(CODES)]) for g in range(G)]
    flags = [(g % 2) | (2 if g % 3 else 0) for g in range(G)]
    dA, dB = dev(A), dev(B)
    o0 = torch.full_like(dA, -1)
    o1 = torch.full_like(dA, -1)
    sf.gate_level(sp, dA, dB, o0, o1, code0, code1, flags, kernel=kernel)
    torch.cuda.synchronize()
    return p, A, B, code0, code1, flags, host(o0, shape), host(o1, shape)


def _unpack(code):
    return [((code >> (4 * k)) & 15) - (16 if (code >> (4 * k)) & 8 else 0) for k in range(4)]


@pytest.mark.parametrize("n,ell,G", [(1, 128, 461), (1, 64, 333), (1, 96, 170), (2, 64, 310),
                                     (3, 32, 157), (1, 128, 1), (1, 128, 153),
                                     (1, 32, 401), (2, 32, 229), (3, 64, 211), (7, 32, 173)])
def test_small_kernel_gate_level_matches_oracle(n, ell, G):
    p, A, B, code0, code1, flags, got0, got1 = _run_level(n, ell, G, sf.KERNEL_SM, 7 * ell + n + G)
    for g in range(G):
        comp = bool(flags[g] & 1)
        assert np.array_equal(got0[g], _oracle_gate(p, A[g], B[g], _unpack(code0[g]), comp)), g
        if flags[g] & 2:
            assert np.array_equal(got1[g], _oracle_gate(p, A[g], B[g], _unpack(code1[g]), comp)), g


@pytest.mark.parametrize("kind", ["ha", "or"])
def test_small_kernel_half_adder_and_or_gates(kind):
    """The codes the FFT circuits mostly use (half adder: XOR and AND from one
    product; OR alone), with and without a complemented A, against the oracle."""
    n, ell, G = 1, 128, 400
    p = gsw.Params(n, ell, (n + 1) * ell, 0)
    shape = (G, p.Ng, n + 1, p.L)
    rng = np.random.default_rng(17 if kind == "ha" else 18)
    A = rng.integers(0, 2**32, size=shape, dtype=np.uint64).astype(np.uint32)
    B = rng.integers(0, 2**32, size=shape, dtype=np.uint64).astype(np.uint32)
    A[3] = 0xFFFFFFFF   # maximal digit sums in one gate
    B[3] = 0xFFFFFFFF
    xor, and_, or_ = (0, 1, 1, -2), (0, 0, 0, 1), (0, 1, 1, -1)
    c0 = xor if kind == "ha" else or_
    code0 = [sf.pack_code(*c0)] * G
    code1 = [sf.pack_code(*and_)] * G
    flags = [(g % 2) | (2 if kind == "ha" else 0) for g in range(G)]
    dA, dB = dev(A), dev(B)
    o0 = torch.full_like(dA, -1)
    o1 = torch.full_like(dA, -1)
    sf.gate_level(sf.Params(n, ell), dA, dB, o0, o1, code0, code1, flags, kernel=sf.KERNEL_SM)
    torch.cuda.synchronize()
    got0, got1 = host(o0, shape), host(o1, shape)
    for g in range(G):
        comp = bool(flags[g] & 1)
        assert np.array_equal(got0[g], _oracle_gate(p, A[g], B[g], c0, comp)), g
        if kind == "ha":
            assert np.array_equal(got1[g], _oracle_gate(p, A[g], B[g], and_, comp)), g
        else:
            assert (got1[g] == 0xFFFFFFFF).all()   # no second output written


def test_small_kernel_extreme_digit_sums():
    """All-ones operands: every digit sum reaches Ng * 255 (the exactness bound)."""
    p, A, B, code0, code1, flags, got0, got1 = _run_level(1, 128, 160, sf.KERNEL_SM, 1, extreme=True)
    for g in range(0, 160, 7):
        comp = bool(flags[g] & 1)
        assert np.array_equal(got0[g], _oracle_gate(p, A[g], B[g], _unpack(code0[g]), comp)), g


def test_small_kernel_equals_general_kernels():
    """The same level on the small, the general tensor-core and the integer
    kernel: identical outputs."""
    outs = [_run_level(1, 128, 300, k, 5)[6:] for k in (sf.KERNEL_SM, sf.KERNEL_TC, sf.KERNEL_INT)]
    for o in outs[1:]:
        assert np.array_equal(outs[0][0], o[0])
        assert np.array_equal(outs[0][1], o[1])


def test_small_kernel_is_the_default_at_p2():
    sp = sf.param_set("P2")
    plan = sf.Plan(sp, 8, 1, 8, 4)
    assert plan.info["gate_kernel"] == sf.KERNEL_SM
    assert plan.info["tc_columns"] == 32
    forced = sf.Plan(sp, 8, 1, 8, 4, sf.PLAN_TC_KERNEL)
    assert forced.info["gate_kernel"] == sf.KERNEL_TC
    assert forced.info["scratch_bytes"] > plan.info["scratch_bytes"]   # the B expansion region


def test_fft_p2_small_kernel_bit_exact():
    """16-point 8-bit FFT at P2 through the plan (small kernel) == the oracle."""
    N, F, f = 16, 8, 4
    sp = sf.param_set("P2")
    p = gsw.Params(sp.n, sp.ell, sp.m, sp.chi)
    re_, im_ = signal_1d(N, -1, 1, 11)
    keys = sf.keygen(sp, 11)
    d_in = torch.zeros((N * 2 * F, sf.ct_words(sp)), dtype=torch.int32, device="cuda")
    sf.encrypt_bits_device(sp, dev(keys.public()), re_, im_, F, f, 3, d_in)
    plan = sf.Plan(sp, N, 1, F, f)
    assert plan.info["gate_kernel"] == sf.KERNEL_SM
    out = torch.zeros((plan.info["outputs"], plan.info["ct_words"]), dtype=torch.int32, device="cuda")
    scratch = torch.empty(max(1, plan.info["scratch_bytes"] // 4), dtype=torch.int32, device="cuda")
    plan.eval_fft(d_in, out, scratch)
    plan.check()
    got = host(out, (N * 2 * F, p.Ng, p.n + 1, p.L))
    ko = gsw.Keys(p, 11)
    c = circuit.fft_circuit(N, 1, F, f)
    cts, bits = [], []
    for k in range(N):
        for part, x in enumerate((re_[k], im_[k])):
            for b, bit in enumerate(fx.to_bits(fx.quantize(x, F, f), F)):
                cts.append(gsw.encrypt(ko, bit, 3, (2 * k + part) * F + b))
                bits.append(bit)
    want = evaluate.eval_encrypted(c, p, cts)
    assert np.array_equal(got, want)
    assert [gsw.decrypt(ko, ct) for ct in got] == evaluate.eval_plain(c, bits)
