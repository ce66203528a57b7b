"""The round-trip check the build entry point exposes (__graft_entry__.smoke):
one small FP64 solve through the C ABI against the oracle's dense LU."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_smoke_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.smoke()
