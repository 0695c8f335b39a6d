"""The smoke entry point as a GPU test: one small Algorithm 3 evaluation on the FP64 and the
emulated-FP64 paths against the oracle, one Fisher-BT step on each, and the adjoint gradient."""
import pytest

from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def test_smoke_entry_point():
    require_gpu()
    import __graft_entry__
    __graft_entry__.smoke()
