"""The driver's smoke entry point, run as a GPU test so that it cannot drift
from the kernels the plans select."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_smoke_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    __graft_entry__.smoke()
