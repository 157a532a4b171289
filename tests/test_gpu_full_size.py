"""Full-size parity: the default bench workload (64-point FFT of 16-bit 8.8 words at the
noisy leveled parameters, ell = 1056 from the static noise bound) through the evaluator and
launch configuration the bench times (the level-merged program replayed as one CUDA graph,
tensor-core product). The encrypted run is too large for the oracle to evaluate gate by gate
(~3,400 s on 16 cores), so every one of the 2048 output ciphertexts is decrypted with the
oracle's keys and compared with the oracle's closed-form integer FFT of the same quantized
inputs, and the exact noise of sampled outputs is checked against the static bound. Single
gates at ell = 1056 are compared ciphertext for ciphertext in test_gpu_parity. The same
runs for the exclusive-carry circuit variant at its own smallest ell (768)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1611_08769_gb300 as sf  # noqa: E402
from oracle import fixedpoint as fx, gsw  # noqa: E402
from paper_1611_08769_gb300 import build as sfbuild  # noqa: E402
from synthetic import signal_1d  # noqa: E402


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
