"""The batched contraction's no-allocation entry point.

tt_contract_batched_noalloc serves callers that cannot give the library a
device workspace where they contract (a plugin in a framework that owns all
device memory, or a loop that must not allocate once running): its work-queue
counter sits in a static device array inside the library.  Here it is called
through the C ABI twice in a row and compared with tt_contract_batched, which
takes a caller-allocated workspace, within the tolerance the other batched
tests use.  The file is named to run last, and passes alone too.
"""
import numpy as np
import pytest

from helpers import norm_scale, to_dev
from paper_2109_00626_gb300 import inputs as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2109_00626_gb300 as T  # noqa: E402


def _pairs(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for p in range(n):
        order = int(rng.integers(2, 6))
        modes = [int(v) for v in rng.integers(2, 17, size=order)]
        rx = [1] + [int(v) for v in rng.integers(2, 70, size=order - 1)] + [1]
        ry = [1] + [int(v) for v in rng.integers(2, 70, size=order - 1)] + [1]
        x = G.random_tt(rng, modes, rx, np.float32)
        y = G.random_tt(rng, modes, ry, np.float32)
        mask = None if p % 2 == 0 else [1] * (order // 2) + [0] * (order - order // 2)
        out.append((x, y, mask))
    return out


def test_noalloc_matches_workspace_entry_two_calls():
    host = _pairs(40, 77)
    bat = T.BatchedContraction([(to_dev(x), to_dev(y), m) for x, y, m in host])
    bat()
    torch.cuda.synchronize()
    assert int(bat.status.item()) == 0
    ref = bat.out.clone()
    ref_z = [None if z is None else [c.clone() for c in z] for z in bat.z]
    for _ in range(2):
        bat.out.fill_(float("nan"))
        for z in bat.z:
            if z is not None:
                for c in z:
                    c.fill_(float("nan"))
        bat.call_noalloc()
        torch.cuda.synchronize()
        assert int(bat.status.item()) == 0
        for p, (x, y, m) in enumerate(host):
            if m is None:
                tol = 1e-5 * norm_scale(x, y)
                assert abs(float(bat.out[p]) - float(ref[p])) <= tol
            else:
                for c, r in zip(bat.z[p], ref_z[p]):
                    scale = float(r.abs().max()) + 1e-30
                    assert float((c - r).abs().max()) <= 1e-5 * scale
