"""Failure detection without a GPU fault: a bounded device wait is made to run
out (the B copy of one K step is withheld, so its barrier never completes);
the kernel stops every role, drains its own MMAs and frees its tensor memory,
the host reads SFFT_ETIMEOUT, and the same context then evaluates the level
correctly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1611_08769_gb300 as sf  # noqa: E402
from paper_1611_08769_gb300 import build as sfbuild  # noqa: E402

SFFT_ETIMEOUT = -4


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sfbuild.build()


def test_withheld_copy_times_out_and_context_recovers():
    sp = sf.param_set("P1", 1056)
    cw = sf.ct_words(sp)
    G = 8
    gen = torch.Generator(device="cuda").manual_seed(3)
    A = torch.randint(-2**31, 2**31 - 1, (G, cw), dtype=torch.int32, device="cuda", generator=gen)
    B = torch.randint(-2**31, 2**31 - 1, (G, cw), dtype=torch.int32, device="cuda", generator=gen)
    code = [sf.pack_code(0, 1, 1, -2)] * G
    flags = [0] * G
    out = torch.zeros((G, cw), dtype=torch.int32, device="cuda")
    with pytest.raises(sf.SfftError) as err:
        sf.gate_level_withheld(sp, A, B, out, code, flags, step=0)
    assert err.value.code == SFFT_ETIMEOUT
    torch.cuda.synchronize()
    # the context is intact: the tensor-core and integer kernels agree
    o_tc = torch.zeros((G, cw), dtype=torch.int32, device="cuda")
    o_int = torch.zeros((G, cw), dtype=torch.int32, device="cuda")
    sf.gate_level(sp, A, B, o_tc, None, code, code, flags, kernel=sf.KERNEL_TC)
    sf.gate_level(sp, A, B, o_int, None, code, code, flags, kernel=sf.KERNEL_INT)
    torch.cuda.synchronize()
    assert torch.equal(o_tc, o_int)
    assert int(o_tc.abs().sum().item()) != 0
