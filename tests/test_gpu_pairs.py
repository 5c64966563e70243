"""GPU parity of tt_contract_pairs: TTs of different orders contracted over
end-block mode pairs (Eq. 8 applied to each pair; Example 1's x_3^2 pairing
when the modes sit at the ends), chain layout, against the oracle's
partial_chain_pairs and the dense Eq. 8 (tcp_pairs).

Tolerances: float64 1e-12 and float32 1e-5 of the per-entry Cauchy-Schwarz
scale ||X[., i_F]|| ||Y[., j_F]|| of Eq. 8's Z (the norms over the contracted
indices); the tf32x3 form 1e-5 as float32.  Copied free cores are compared
bit for bit through the dense result's exactness on the small cases."""
import numpy as np
import pytest

import oracle as O
from helpers import to_dev, to_host
from paper_2109_00626_gb300 import inputs as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2109_00626_gb300 as T  # noqa: E402

CASES = [
    # orders, pairs
    (4, 3, [(0, 0)]),
    (4, 3, [(0, 0), (1, 1)]),
    (3, 5, [(2, 4), (1, 3)]),    # trailing block of X with trailing block of Y
    (5, 3, [(0, 2), (1, 1)]),    # leading block of X against trailing block of Y
    (3, 4, [(2, 0), (1, 1)]),    # trailing block of X against leading block of Y
    (2, 4, [(0, 0), (1, 1)]),    # X fully contracted: Y keeps two free modes
    (4, 2, [(3, 1), (2, 0)]),    # Y fully contracted
    (1, 3, [(0, 2)]),
    (6, 4, [(5, 0), (4, 1), (3, 2)]),
]


def _pair(seed, nx, ny, pairs, dtype, rmax=6, imax=4):
    rng = np.random.default_rng(seed)
    mx = [int(v) for v in rng.integers(2, imax + 1, size=nx)]
    my = [int(v) for v in rng.integers(2, imax + 1, size=ny)]
    for a, b in pairs:
        my[b] = mx[a]
    x = G.random_tt(rng, mx, [1] + [int(v) for v in rng.integers(1, rmax + 1, size=nx - 1)] + [1], dtype)
    y = G.random_tt(rng, my, [1] + [int(v) for v in rng.integers(1, rmax + 1, size=ny - 1)] + [1], dtype)
    return x, y


def _cs_scale(x, y, pairs):
    """||X[., i_F]|| ||Y[., j_F]|| in Eq. 8's axis order."""
    xd = O.tt_to_dense([np.asarray(c, np.float64) for c in x])
    yd = O.tt_to_dense([np.asarray(c, np.float64) for c in y])
    cx = tuple(a for a, _ in pairs)
    cy = tuple(b for _, b in pairs)
    gx = np.sqrt(np.sum(xd * xd, axis=cx)) if cx else np.abs(xd)
    gy = np.sqrt(np.sum(yd * yd, axis=cy)) if cy else np.abs(yd)
    return np.multiply.outer(gx, gy)


@pytest.mark.parametrize("prec,dtype,tol", [("native", np.float64, 1e-12), ("native", np.float32, 1e-5),
                                            ("tf32x3", np.float32, 1e-5)])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_pairs_against_dense(case, prec, dtype, tol):
    nx, ny, pairs = CASES[case]
    x, y = _pair(17 + case, nx, ny, pairs, dtype)
    op = T.PairsContraction(to_dev(x), to_dev(y), pairs, prec=prec)
    op()
    torch.cuda.synchronize()
    assert int(op.status.item()) == 0
    got = to_host(op.z)
    x64 = [np.asarray(c, np.float64) for c in x]
    y64 = [np.asarray(c, np.float64) for c in y]
    want = O.tcp_pairs(O.tt_to_dense(x64), O.tt_to_dense(y64), pairs)
    dense = O.chain_to_dense(got, op.perm)
    assert dense.shape == want.shape
    eps = float(np.max(np.abs(dense - want) / np.maximum(_cs_scale(x64, y64, pairs), 1e-300)))
    print(f"pairs {nx}x{ny} {pairs} {prec} {np.dtype(dtype).name}: cs_eps={eps:.2e}")
    assert eps <= tol
    # same represented tensor as the oracle's chain (whose layout may differ
    # when X has no free mode)
    oc, operm = O.partial_chain_pairs(x64, y64, pairs)
    np.testing.assert_allclose(O.chain_to_dense(oc, operm), want, rtol=1e-10, atol=1e-12)


def test_pairs_example1_shapes_and_rank64():
    """Example 1's x_3^2 with the paired modes at the ends (order 4 against
    order 3, ranks 64, modes 16): X's mode 3 (0-based) against Y's mode 0;
    the chain's cores follow Z^rho and its free cores are copies."""
    rng = np.random.default_rng(3)
    x = G.random_tt(rng, [8, 12, 10, 16], [1, 64, 64, 64, 1], np.float32)
    y = G.random_tt(rng, [16, 14, 6], [1, 64, 64, 1], np.float32)
    pairs = [(3, 0)]
    op = T.PairsContraction(to_dev(x), to_dev(y), pairs)
    op()
    torch.cuda.synchronize()
    assert int(op.status.item()) == 0
    got = to_host(op.z)
    # X walked backwards: its free cores come first in their own order (X
    # reversed twice), then C, then Y's free cores
    assert [g.shape[1] for g in got] == [8, 12, 10, 14, 6]
    np.testing.assert_array_equal(got[0], x[0].astype(np.float64))
    np.testing.assert_array_equal(got[1], x[1].astype(np.float64))
    np.testing.assert_array_equal(got[3], y[1].astype(np.float64))
    np.testing.assert_array_equal(got[4], y[2].astype(np.float64))
    oc, operm = O.partial_chain_pairs(x, y, pairs)
    # C against the oracle's C (same layout here): within 1e-5 of its largest entry
    c_want = oc[2]
    assert np.abs(got[2] - c_want).max() <= 1e-5 * np.abs(c_want).max()


def test_pairs_rejections():
    x, y = _pair(5, 4, 3, [(0, 0)], np.float32)
    xd, yd = to_dev(x), to_dev(y)
    with pytest.raises(T.TTError):
        T.PairsContraction(xd, yd, [(1, 0)])            # not an end block of X
    with pytest.raises(T.TTError):
        T.PairsContraction(xd, yd, [(0, 0), (1, 2)])    # met in different orders
    with pytest.raises(T.TTError):
        T.PairsContraction(xd, yd, [(0, 1)])            # not an end block of Y
