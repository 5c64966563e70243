"""The device-side bounded waits give up and report TT_STATUS_TIMEOUT.

tt_selftest_wait runs the same bounded mbarrier wait the pipelined kernels
use, with a short limit, on a barrier that never completes: the status word
gets TT_STATUS_TIMEOUT and the kernel returns (the context stays usable).  The
control case, a barrier whose phase completes before the wait, sets nothing.
Nothing asynchronous is in flight in either case, so no fault or hang can
follow from the wait giving up."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2109_00626_gb300 as T  # noqa: E402
from paper_2109_00626_gb300 import _binding as B  # noqa: E402


def _run(complete, limit):
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert T.lib().tt_selftest_wait(int(complete), int(limit), ctypes.c_void_p(st.data_ptr()), None) == 0
    torch.cuda.synchronize()
    return int(st.item())


def test_wait_that_never_completes_reports_timeout():
    for limit in (0, 20000, 2000000):
        assert _run(False, limit) == B.TT_STATUS_TIMEOUT


def test_wait_that_completes_reports_nothing():
    assert _run(True, 20000) == 0


def test_context_usable_after_a_timeout():
    """A contraction right after a wait that gave up runs normally."""

    import oracle as O
    from helpers import norm_scale, to_dev
    from paper_2109_00626_gb300 import inputs as G

    assert _run(False, 1000) == B.TT_STATUS_TIMEOUT
    x, y = G.small_fp64(2)
    op = T.FullContraction(to_dev(x), to_dev(y))
    op()
    torch.cuda.synchronize()
    assert int(op.status.item()) == 0
    assert abs(float(op.out.item()) - O.contract_full(x, y)) <= 1e-12 * norm_scale(x, y)
