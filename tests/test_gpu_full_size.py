"""Full-size parity: the default bench workload (64-point FFT of 16-bit 8.8 words at the
noisy leveled parameters, ell = 1056 from the static noise bound) through the evaluator and
launch configuration the bench times (the level-merged program replayed as one CUDA graph,
tensor-core product). The encrypted run is too large for the oracle to evaluate gate by gate
(~3,400 s on 16 cores), so every one of the 2048 output ciphertexts is decrypted with the
oracle's keys and compared with the oracle's closed-form integer FFT of the same quantized
inputs, and the exact noise of sampled outputs is checked against the static bound; and,
level by level, over a thousand sampled gates are recomputed by the oracle from the GPU's
own stored inputs and compared ciphertext for ciphertext. The 16 x 16 image workload (ell
992) is checked by decrypting every output. The same
runs for the exclusive-carry circuit variant at its own smallest ell (768)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1611_08769_gb300 as sf  # noqa: E402
from oracle import fixedpoint as fx, gsw  # noqa: E402
from paper_1611_08769_gb300 import build as sfbuild  # noqa: E402
from synthetic import image_2d, signal_1d  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sfbuild.build()


class _Row:
    """A ciphertext of which only row `row` is present (decryption reads no other)."""

    def __init__(self, row, data):
        self.row, self.data = row, data

    def __getitem__(self, i):
        assert i == self.row
        return self.data


@pytest.mark.parametrize("xcarry,ell_expected", [(False, 1056), (True, 768)])
def test_full_size_fft_decrypts_to_closed_form(xcarry, ell_expected):
    N, F, f = 64, 16, 8
    ell = sf.min_ell(N, 1, F, f, n=1, chi=1, xcarry=xcarry)
    assert ell == ell_expected
    sp = sf.param_set("P1", ell)
    p = gsw.Params(sp.n, sp.ell, sp.m, sp.chi)
    key_seed, enc_seed = 21, 5
    re_, im_ = signal_1d(N, -8.0, 8.0, 13)

    keys = sf.keygen(sp, key_seed)
    pub = torch.from_numpy(keys.public().view(np.int32)).cuda()
    batch = sf.Batch(sp, [(N, 1, F, f)], sf.PLAN_XCARRY if xcarry else 0)
    info = batch.info
    assert info["gate_kernel"] == sf.KERNEL_TC and info["noise_ok"] == 1
    cw = sf.ct_words(sp)
    d_in = torch.empty((info["inputs"], cw), dtype=torch.int32, device="cuda")
    sf.encrypt_bits_device(sp, pub, re_, im_, F, f, enc_seed, d_in)
    d_out = torch.zeros((info["outputs"], cw), dtype=torch.int32, device="cuda")
    scratch = torch.empty(max(1, info["scratch_bytes"] // 4), dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    for _ in range(2):   # the first call captures the graph, the second replays it
        batch.eval(d_in, d_out, scratch, stream)
    batch.check(stream)
    torch.cuda.synchronize()

    # decryption rows (row ell - 1 of every output ciphertext), oracle keys
    cts = d_out.view(info["outputs"], p.Ng, p.n + 1, p.L)
    rows = cts[:, p.ell - 1].cpu().numpy().view(np.uint32)
    ko = gsw.Keys(p, key_seed)
    got = [gsw.decrypt(ko, _Row(p.ell - 1, rows[c])) for c in range(info["outputs"])]

    # closed form: integer DIT FFT of the quantized inputs; output word (2k + part), bits LSB first
    xr = [fx.quantize(float(x), F, f) for x in re_]
    xi = [fx.quantize(float(x), F, f) for x in im_]
    yr, yi = fx.fft_int(xr, xi, F, f)
    want = []
    for k in range(N):
        for v in (yr[k], yi[k]):
            want.extend(fx.to_bits(v, F))
    assert got == want

    # exact noise of sampled outputs below the static bound
    bound = 1 << info["noise_bits"]
    for c in (0, 1, 777, 2047):
        full = cts[c].cpu().numpy().view(np.uint32)
        e = gsw.noise(ko, full, got[c])
        assert max(abs(x) for x in e) < bound


def _code(c):
    return [((c >> (4 * k)) & 15) - (16 if (c >> (4 * k)) & 8 else 0) for k in range(4)]


def _oracle_gate(p, A, B, code, comp):
    """c0 P + c1 A + c2 B + c3 BitDecomp(A~) B with A~ = P - A when comp."""
    Aval = gsw.gate(p, A, None, gsw.GATE_CODES["NOT"]) if comp else A
    terms = [(code[0], gsw.gadget(p)), (code[1], A), (code[2], B)]
    if code[3]:
        terms.append((code[3], gsw.product(Aval, B, p.L)))
    if all(c == 0 for c, _ in terms):
        return gsw.zero_ct(p)
    return gsw.lincomb(terms, p.L)


def test_full_size_sampled_gates_match_oracle():
    """The default bench workload (64 points, 16-bit 8.8, noisy ell 1056) level
    by level on the tensor-core kernel: at every one of its 178 levels the
    first, the last and seven random products (at least 1000 in all) are
    recomputed by the oracle from the GPU's own stored inputs and compared
    ciphertext for ciphertext with the GPU's outputs (the sampled-gate check
    at full size). Levels of up to 2341 products are 17 tiles per gate, so the
    persistent kernel's loop over several tiles per CTA and both of its
    accumulator slots are exercised."""
    N, F, f = 64, 16, 8
    ell = sf.min_ell(N, 1, F, f, n=1, chi=1)
    assert ell == 1056
    sp = sf.param_set("P1", ell)
    p = gsw.Params(sp.n, sp.ell, sp.m, sp.chi)
    keys = sf.keygen(sp, 31)
    pub = torch.from_numpy(keys.public().view(np.int32)).cuda()
    re_, im_ = signal_1d(N, -8.0, 8.0, 17)
    plan = sf.Plan(sp, N, 1, F, f)
    info = plan.info
    assert info["gate_kernel"] == sf.KERNEL_TC
    cw = sf.ct_words(sp)
    d_in = torch.empty((info["inputs"], cw), dtype=torch.int32, device="cuda")
    sf.encrypt_bits_device(sp, pub, re_, im_, F, f, 9, d_in)
    d_out = torch.zeros((info["outputs"], cw), dtype=torch.int32, device="cuda")
    scratch = torch.empty(max(1, info["scratch_bytes"] // 4), dtype=torch.int32, device="cuda")
    slots = scratch[:info["scratch_slots"] * cw].view(info["scratch_slots"], cw)
    regions = {0: slots, 1: d_in, 2: d_out}

    def fetch(ref):
        t = regions[int(ref) >> 30][int(ref) & 0x3FFFFFFF]
        return t.cpu().numpy().view(np.uint32).reshape(p.Ng, p.n + 1, p.L)

    rng = np.random.default_rng(3)
    checked = 0
    for lev in range(info["levels"]):
        desc, code, flags, npr = plan.level(lev)
        assert npr > 0
        pick = {0, npr - 1} | set(rng.choice(npr, size=min(npr, 7), replace=False).tolist())
        pick = sorted(pick)
        ins = [(fetch(desc[g, 0]), fetch(desc[g, 1])) for g in pick]
        plan.eval_levels(lev, lev + 1, d_in, d_out, scratch)
        plan.check()
        for (A, B), g in zip(ins, pick):
            comp = bool(flags[g] & 1)
            for k, ref in ((0, desc[g, 2]), (1, desc[g, 3])):
                if ref == 0xFFFFFFFF:
                    continue
                want = _oracle_gate(p, A, B, _code((int(code[g]) >> (16 * k)) & 0xFFFF), comp)
                assert np.array_equal(fetch(ref), want), (lev, g, k)
            checked += 1
    assert checked >= 1000, checked
    plan.eval_levels(info["levels"], info["levels"], d_in, d_out, scratch)   # output fix-ups
    plan.check()
    # the stepped run ends where the one-call evaluation does
    d_out2 = torch.zeros_like(d_out)
    plan.eval_fft(d_in, d_out2, scratch)
    plan.check()
    assert torch.equal(d_out, d_out2)


def test_full_size_image_fft_decrypts_to_closed_form():
    """The 16 x 16 image workload (10.6 words, noisy ell 992 from the static
    bound; Sec. 6's row-column 2-D transform) through the graph-replayed batch:
    every one of the 8192 output ciphertexts decrypts to the oracle's
    closed-form 2-D integer FFT of the same quantized pixels."""
    N1 = N2 = 16
    F, f = 16, 6
    ell = sf.min_ell(N1, N2, F, f, n=1, chi=1)
    assert ell == 992
    sp = sf.param_set("P1", ell)
    p = gsw.Params(sp.n, sp.ell, sp.m, sp.chi)
    keys = sf.keygen(sp, 41)
    pub = torch.from_numpy(keys.public().view(np.int32)).cuda()
    re_, im_ = image_2d(N1, N2, 23)
    batch = sf.Batch(sp, [(N1, N2, F, f)])
    info = batch.info
    assert info["gate_kernel"] == sf.KERNEL_TC and info["noise_ok"] == 1
    cw = sf.ct_words(sp)
    d_in = torch.empty((info["inputs"], cw), dtype=torch.int32, device="cuda")
    sf.encrypt_bits_device(sp, pub, re_, im_, F, f, 7, d_in)
    d_out = torch.zeros((info["outputs"], cw), dtype=torch.int32, device="cuda")
    scratch = torch.empty(max(1, info["scratch_bytes"] // 4), dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    for _ in range(2):   # capture, then replay
        batch.eval(d_in, d_out, scratch, stream)
    batch.check(stream)
    torch.cuda.synchronize()
    cts = d_out.view(info["outputs"], p.Ng, p.n + 1, p.L)
    rows = cts[:, p.ell - 1].cpu().numpy().view(np.uint32)
    ko = gsw.Keys(p, 41)
    got = [gsw.decrypt(ko, _Row(p.ell - 1, rows[c])) for c in range(info["outputs"])]
    xr = [fx.quantize(float(x), F, f) for x in re_]
    xi = [fx.quantize(float(x), F, f) for x in im_]
    yr, yi = fx.fft2_int(xr, xi, N1, N2, F, f)
    want = []
    for k in range(N1 * N2):
        for v in (yr[k], yi[k]):
            want.extend(fx.to_bits(v, F))
    assert got == want
