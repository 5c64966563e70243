"""The per-entry Cauchy-Schwarz scales the GPU parity tests divide by
(tests/helpers.py) are upper bounds of the oracle's own values, reached by
rank-1 operands whose contracted factors are parallel."""
import numpy as np

import oracle as O
from helpers import dense_cs_scale, grad_cs_scale
from paper_2109_00626_gb300 import inputs as G


def test_dense_scale_bounds_partial_contraction():
    rng = np.random.default_rng(4)
    x = G.random_tt(rng, [3, 4, 2, 3], [1, 3, 2, 4, 1], np.float64)
    y = G.random_tt(rng, [3, 4, 2, 3], [1, 2, 5, 3, 1], np.float64)
    for contracted in ([0, 1], [2], [1, 3], []):
        z = O.tcp(O.tt_to_dense(x), O.tt_to_dense(y), contracted)
        scale = dense_cs_scale(x, y, contracted)
        assert scale.shape == z.shape
        assert np.all(np.abs(z) <= scale * (1 + 1e-12))


def test_dense_scale_attained_by_parallel_rank1():
    rng = np.random.default_rng(5)
    vs = [rng.standard_normal(4) for _ in range(3)]
    x = [v.reshape(1, -1, 1) for v in vs]
    y = [2.0 * vs[0].reshape(1, -1, 1), -3.0 * vs[1].reshape(1, -1, 1), rng.standard_normal((1, 4, 1))]
    z = O.tcp(O.tt_to_dense(x), O.tt_to_dense(y), [0, 1])
    np.testing.assert_allclose(np.abs(z), dense_cs_scale(x, y, [0, 1]), rtol=1e-12)


def test_grad_scale_bounds_gradients():
    rng = np.random.default_rng(6)
    x = G.random_tt(rng, [3, 4, 2, 3], [1, 3, 2, 4, 1], np.float64)
    y = G.random_tt(rng, [3, 4, 2, 3], [1, 2, 5, 3, 1], np.float64)
    gx, gy = O.grad_full(x, y)
    for g, s in zip(gx + gy, grad_cs_scale(x, y)):
        assert g.shape == s.shape
        assert np.all(np.abs(g) <= s * (1 + 1e-12))
    # attained: Y = X, a rank-1 train (every gradient entry is the CS product)
    r1 = [rng.standard_normal((1, 3, 1)) for _ in range(3)]
    gx, _ = O.grad_full(r1, r1)
    sc = grad_cs_scale(r1, r1)
    for k in range(3):
        i = int(np.argmax(np.abs(r1[k])))
        np.testing.assert_allclose(abs(gx[k][0, i, 0]), sc[k][0, i, 0] * abs(r1[k][0, i, 0]) / np.linalg.norm(r1[k]), rtol=1e-12)
