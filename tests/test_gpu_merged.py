"""GPU parity of the merged (TT-matrix) layout of a partial contraction over
any contracted set, against the oracle's merged cores and the dense Eq. 8."""
import numpy as np
import pytest

import oracle as O
from helpers import norm_scale, to_dev, to_host
from paper_2109_00626_gb300 import inputs as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2109_00626_gb300 as T  # noqa: E402


def _run(x, y, mask):
    op = T.PartialContraction(to_dev(x), to_dev(y), mask, layout="merged")
    op()
    torch.cuda.synchronize()
    return op, to_host(op.z)


def test_merged_small_fp64_modes34():
    x, y = G.small_fp64(0)
    mask = [0, 0, 1, 1]
    op, got = _run(x, y, mask)
    assert int(op.status.item()) == 0
    want, perm = O.partial_merged(x, y, mask)
    assert op.perm == perm
    assert [g.shape for g in got] == [(w.shape[0], w.shape[1] * w.shape[2], w.shape[3]) for w in want]
    scale = norm_scale(x, y)
    for g, w in zip(got, want):
        assert np.abs(g - w.reshape(g.shape)).max() <= 1e-12 * scale
    dense = O.merged_to_dense([g.reshape(w.shape) for g, w in zip(got, want)], perm)
    ref = O.tcp(O.tt_to_dense(x), O.tt_to_dense(y), [2, 3])
    assert np.abs(dense - ref).max() <= 1e-12 * scale


MASKS = [[0, 1, 0, 1, 0], [1, 0, 1, 0, 1], [0, 1, 1, 0, 0], [1, 0, 0, 0, 1], [0, 0, 0, 0, 0], [1, 1, 0, 1, 1],
         [0, 0, 0, 1, 1], [1, 1, 1, 1, 0]]


@pytest.mark.parametrize("mask", MASKS)
def test_merged_any_mask_fp64(mask):
    rng = np.random.default_rng(11 + sum(m << k for k, m in enumerate(mask)))
    modes = [3, 2, 4, 2, 3]
    x = G.random_tt(rng, modes, [1, 2, 5, 3, 2, 1], np.float64)
    y = G.random_tt(rng, modes, [1, 3, 1, 4, 2, 1], np.float64)
    op, got = _run(x, y, mask)
    assert int(op.status.item()) == 0
    want, perm = O.partial_merged(x, y, mask)
    dense = O.merged_to_dense([g.reshape(w.shape) for g, w in zip(got, want)], perm)
    ref = O.tcp(O.tt_to_dense(x), O.tt_to_dense(y), [k for k in range(5) if mask[k]])
    assert np.abs(dense - ref).max() <= 1e-12 * norm_scale(x, y)


def test_merged_secondary_fp32():
    """Order 6, modes 8, ranks 16, a random contracted set of three modes."""
    rng = np.random.default_rng(5)
    x, y = G.pair(5, [8] * 6, G.tt_ranks(6, 16), G.tt_ranks(6, 16), np.float32)
    mask = [0] * 6
    for k in rng.choice(6, 3, replace=False):
        mask[int(k)] = 1
    op, got = _run(x, y, mask)
    assert int(op.status.item()) == 0
    want, _ = O.partial_merged(x, y, mask)
    for g, w in zip(got, want):
        w = w.reshape(g.shape)
        assert np.abs(g - w).max() <= 1e-5 * max(np.abs(w).max(), 1e-30) * 10
