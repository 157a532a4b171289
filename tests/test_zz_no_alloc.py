"""The allocation-free evaluation entry point (sfft_eval_fft_noalloc).

Some callers cannot call cudaMalloc while they evaluate -- their own memory
pool already holds the device memory, or they run a latency-critical loop
where cudaMalloc's device-wide synchronisation is not acceptable. For them
the library keeps the FFT's intermediate ciphertexts in a fixed device array
instead of a caller-provided scratch buffer.

This file runs last (pytest collects it after every other test file): two
calls in a row through the C ABI must reproduce the regular entry point's
ciphertexts bit for bit (the same exact-equality bar as every other parity
test), and a plan whose scratch exceeds the array is refused with an error.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1611_08769_gb300 as sf  # noqa: E402
from paper_1611_08769_gb300 import build as sfbuild  # noqa: E402
from synthetic import signal_1d  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sfbuild.build()


@pytest.mark.parametrize("pset,flags,kernel", [("P0", sf.PLAN_INT_KERNEL, sf.KERNEL_INT),
                                               ("P0", 0, sf.KERNEL_SM), ("P2", 0, sf.KERNEL_SM),
                                               ("P1", 0, sf.KERNEL_TC)])
def test_noalloc_matches_regular_entry_point_twice(pset, flags, kernel):
    """Each gate kernel through the fixed array: the integer kernel (toy
    parameters, forced), the small-ciphertext tensor-core kernel (ell 32 and
    128) and the general tensor-core kernel with its B expansion inside the
    array (noisy ell 224, the 8-point circuit's smallest)."""
    N, F, f = 8, 8, 4
    sp = sf.param_set(pset, sf.min_ell(N, 1, F, f, n=1, chi=1) if pset == "P1" else None)
    keys = sf.keygen(sp, 21)
    re_, im_ = signal_1d(N, -1.0, 1.0, 21)
    cw = sf.ct_words(sp)
    pub = torch.from_numpy(keys.public().view(np.int32)).cuda()
    d_in = torch.empty((N * 2 * F, cw), dtype=torch.int32, device="cuda")
    sf.encrypt_bits_device(sp, pub, re_, im_, F, f, 22, d_in)
    plan = sf.Plan(sp, N, 1, F, f, flags)
    assert plan.info["gate_kernel"] == kernel
    assert plan.info["scratch_bytes"] <= sf.lib().sfft_noalloc_scratch_bytes()
    ref = torch.empty((plan.info["outputs"], cw), dtype=torch.int32, device="cuda")
    scratch = torch.empty(plan.info["scratch_bytes"] // 4, dtype=torch.int32, device="cuda")
    plan.eval_fft(d_in, ref, scratch)
    for _ in range(2):
        out = torch.full_like(ref, -1)
        plan.eval_fft_noalloc(d_in, out)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)


def test_noalloc_rejects_plans_beyond_the_fixed_array():
    sp = sf.param_set("P2")
    plan = sf.Plan(sp, 64, 1, 16, 8)
    assert plan.info["scratch_bytes"] > sf.lib().sfft_noalloc_scratch_bytes()
    cw = plan.info["ct_words"]
    d_in = torch.zeros((plan.info["inputs"], cw), dtype=torch.int32, device="cuda")
    out = torch.zeros_like(d_in)
    with pytest.raises(sf.SfftError, match="scratch"):
        plan.eval_fft_noalloc(d_in, out)
