"""GPU parity of the dense-input path: the TT-SVD (tt_svd, Section II's TT
decomposition with its accuracy guarantee), the dense mode permutation
(tt_dense_permute) and the dense-input contraction of Alg. 2 built from them
(contract_dense_pairs), against the float64 oracle.

What is unique is compared; what has freedom (the gauge of the cores, the
signs of singular vectors) is checked for validity:
- ranks: a tensor of exact TT ranks r (plus, for truncation, noise of 1e-3
  of its norm with eps = 1e-2) gives ranks r; the first unfolding's rank is
  the one the oracle's singular values give for the same threshold;
- the reconstruction error ||X - TT(X)||_F <= eps ||X||_F (+ rounding:
  1e-12 float64, 2e-6 float32, relative to ||X||);
- cores 0 .. N-2 left-orthonormal (sum_{a,i} G[a,i,b] G[a,i,b'] = delta)
  within 1e-12 / 1e-5;
- the permutation bit for bit against numpy;
- the dense-input contraction against Eq. 8 on the dense tensors (oracle
  tcp_pairs) within e_x ||Y~|| + ||X|| e_y (e = the measured reconstruction
  errors) plus rounding (1e-12 / 1e-5 of ||X|| ||Y||), on Example 2's shapes
  (X in R^{20x20x20}, Y of 20^3, 20^3 x 5, 20^3 x 5 x 4; X x_1^1 Y) and on
  interior pairs that need the permutation."""
import numpy as np
import pytest

import oracle as O
from paper_2109_00626_gb300 import inputs as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2109_00626_gb300 as T  # noqa: E402

RTOL = {np.float64: 1e-12, np.float32: 2e-6}
ORTH = {np.float64: 1e-12, np.float32: 1e-5}


def _dense_tt(seed, modes, ranks, dtype):
    rng = np.random.default_rng(seed)
    x = G.random_tt(rng, modes, ranks, np.float64)
    return O.tt_to_dense(x).astype(dtype)


def _decompose(xh, eps, max_rank=0):
    x = torch.from_numpy(np.ascontiguousarray(xh)).cuda()
    cores = T.tt_decompose(x, eps, max_rank)
    torch.cuda.synchronize()
    return [c.cpu().numpy().astype(np.float64) for c in cores]


def _check_valid(xh, cores, eps, dtype, label):
    x64 = np.asarray(xh, dtype=np.float64)
    nrm = np.linalg.norm(x64)
    err = np.linalg.norm(O.tt_to_dense(cores) - x64)
    print(f"{label}: ranks {[c.shape[0] for c in cores] + [1]} err/||x|| = {err / nrm:.2e} (eps {eps:g})")
    assert err <= (eps + RTOL[dtype] * np.sqrt(x64.size)) * nrm
    for k, g in enumerate(cores[:-1]):
        m = g.reshape(-1, g.shape[2])
        gram = m.T @ m
        assert np.abs(gram - np.eye(gram.shape[0])).max() <= ORTH[dtype] * max(1, np.sqrt(m.shape[0])), (label, k)
    return err


EXACT = [
    ([6, 5, 4, 3], [1, 3, 4, 2, 1]),
    ([4, 4, 4, 4, 4], [1, 4, 7, 5, 3, 1]),
    ([20, 20, 20], [1, 6, 9, 1]),
    ([2, 3, 2, 3, 2, 3], [1, 2, 5, 4, 5, 3, 1]),
    ([9], [1, 1]),
    ([1, 7, 1, 5], [1, 1, 3, 3, 1]),
]


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("case", range(len(EXACT)))
def test_exact_ranks_recovered(case, dtype):
    modes, ranks = EXACT[case]
    xh = _dense_tt(31 + case, modes, ranks, dtype)
    eps = 1e-10 if dtype == np.float64 else 1e-5
    cores = _decompose(xh, eps)
    assert [c.shape[0] for c in cores] + [1] == ranks
    _check_valid(xh, cores, eps, dtype, f"exact {modes}")


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_truncation_drops_the_noise(dtype):
    """A rank-(1,5,6,4,1) tensor plus Gaussian noise of 1e-3 of its norm,
    eps = 1e-2: the noise is dropped, the ranks are the structured ones and
    the error stays within the guarantee."""
    modes, ranks = [8, 7, 6, 5], [1, 5, 6, 4, 1]
    x = _dense_tt(5, modes, ranks, np.float64)
    rng = np.random.default_rng(6)
    noise = rng.standard_normal(x.shape)
    x = (x + 1e-3 * np.linalg.norm(x) / np.linalg.norm(noise) * noise).astype(dtype)
    cores = _decompose(x, 1e-2)
    assert [c.shape[0] for c in cores] + [1] == ranks
    _check_valid(x, cores, 1e-2, dtype, "noisy")


@pytest.mark.parametrize("eps", [0.05, 0.3, 0.6])
def test_truncated_gaussian_tensor(eps):
    """A full-rank Gaussian tensor (Example 2's workload, 20 x 20 x 20)
    truncated at eps: the error stays within eps ||X||; the first rank is the
    one the oracle's decomposition taken in the same direction gives (the
    right-to-left oracle on the reversed axes, reversed back), unless a tail
    of the first unfolding's singular values lies within 1e-6 of the
    threshold."""
    rng = np.random.default_rng(77)
    x = rng.standard_normal((20, 20, 20))
    cores = _decompose(x, eps)
    _check_valid(x, cores, eps, np.float64, f"gaussian eps={eps}")
    got = [c.shape[0] for c in cores] + [1]
    want = [c.shape[0] for c in O.reverse_tt(O.tt_svd(np.transpose(x, (2, 1, 0)), eps))] + [1]
    tol = eps * np.linalg.norm(x) / np.sqrt(2)
    sv = np.linalg.svd(x.reshape(20, -1), compute_uv=False)
    tails = np.sqrt(np.cumsum(sv[::-1] ** 2))[::-1]
    if np.min(np.abs(tails - tol)) > 1e-6 * tol:
        assert got[1] == want[1]
    assert max(got) <= 20


def test_max_rank_cap():
    xh = _dense_tt(9, [6, 6, 6, 6], [1, 6, 12, 6, 1], np.float64)
    cores = _decompose(xh, 0.0, max_rank=3)
    assert [c.shape[0] for c in cores] + [1] == [1, 3, 3, 3, 1]
    for g in cores[:-1]:
        m = g.reshape(-1, g.shape[2])
        assert np.abs(m.T @ m - np.eye(3)).max() <= 1e-12


def test_order_one_and_zero_tensor():
    v = np.arange(1.0, 8.0)
    cores = _decompose(v, 0.1)
    assert len(cores) == 1 and cores[0].shape == (1, 7, 1)
    np.testing.assert_array_equal(cores[0].ravel(), v)
    z = np.zeros((3, 4, 5))
    cores = _decompose(z, 0.1)
    assert [c.shape[0] for c in cores] + [1] == [1, 1, 1, 1]
    assert np.abs(O.tt_to_dense(cores)).max() == 0.0


def test_nonfinite_tensor_is_reported():
    x = torch.ones((4, 5, 6), dtype=torch.float64, device="cuda")
    x[1, 2, 3] = float("nan")
    with pytest.raises(ValueError):
        T.tt_decompose(x, 0.1)


@pytest.mark.parametrize("axes", [(2, 0, 1), (1, 2, 0, 3), (3, 2, 1, 0), (0, 1, 2)])
def test_dense_permute_exact(axes):
    rng = np.random.default_rng(len(axes))
    shape = [5, 3, 4, 6][: len(axes)]
    xh = rng.standard_normal(shape)
    x = torch.from_numpy(xh).cuda()
    got = T.dense_permute(x, axes).cpu().numpy()
    np.testing.assert_array_equal(got, np.transpose(xh, axes))
    got32 = T.dense_permute(x.float(), axes).cpu().numpy()
    np.testing.assert_array_equal(got32, np.transpose(xh.astype(np.float32), axes))


def _check_dense_contraction(xh, yh, pairs, eps, dtype, label):
    x = torch.from_numpy(np.ascontiguousarray(xh.astype(dtype))).cuda()
    y = torch.from_numpy(np.ascontiguousarray(yh.astype(dtype))).cuda()
    cores, perm = T.contract_dense_pairs(x, y, pairs, eps)
    torch.cuda.synchronize()
    got = O.chain_to_dense([c.cpu().numpy().astype(np.float64) for c in cores], perm)
    x64, y64 = xh.astype(dtype).astype(np.float64), yh.astype(dtype).astype(np.float64)
    want = O.tcp_pairs(x64, y64, pairs)
    nx, ny = np.linalg.norm(x64), np.linalg.norm(y64)
    # the decompositions the contraction used, measured on the oracle side
    ax = [a for a, _ in pairs] + [k for k in range(x64.ndim) if k not in {a for a, _ in pairs}]
    ay = [b for _, b in pairs] + [k for k in range(y64.ndim) if k not in {b for _, b in pairs}]
    ex = np.linalg.norm(O.tt_to_dense(_decompose(np.transpose(x64, ax).astype(dtype), eps)) - np.transpose(x64, ax))
    ey = np.linalg.norm(O.tt_to_dense(_decompose(np.transpose(y64, ay).astype(dtype), eps)) - np.transpose(y64, ay))
    # each decomposition keeps its own guarantee (the larger unfoldings here take the
    # cluster-wide sweeps)
    slack = RTOL[dtype] * np.sqrt(max(x64.size, y64.size))
    assert ex <= (eps + slack) * nx and ey <= (eps + slack) * ny, (ex / nx, ey / ny)
    bound = ex * (ny + ey) + nx * ey + (1e-12 if dtype == np.float64 else 1e-5) * nx * ny
    err = np.linalg.norm(got - want)
    print(f"{label}: |Z - Z*|_F / (|X||Y|) = {err / (nx * ny):.2e}, bound {bound / (nx * ny):.2e}")
    assert got.shape == want.shape
    assert err <= bound


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("yshape", [(20, 20, 20), (20, 20, 20, 5), (20, 20, 20, 5, 4)])
def test_example2_dense_contraction(yshape, dtype):
    """Example 2's X x_1^1 Y on Gaussian tensors (no truncation: eps = 1e-12
    / 1e-6 keeps the full ranks)."""
    if dtype == np.float64 and len(yshape) == 5:
        pytest.skip("a 400 x 400 Jacobi SVD in float64 is slow on this part's float64 pipe; float32 covers it")
    rng = np.random.default_rng(2 + len(yshape))
    xh = rng.standard_normal((20, 20, 20))
    yh = rng.standard_normal(yshape)
    eps = 1e-12 if dtype == np.float64 else 1e-6
    _check_dense_contraction(xh, yh, [(0, 0)], eps, dtype, f"example2 {yshape} {np.dtype(dtype).name}")


@pytest.mark.parametrize("pairs", [[(1, 2)], [(2, 0)], [(1, 2), (3, 3)], [(0, 1), (2, 0)]])
def test_dense_contraction_interior_pairs(pairs):
    """Pairs that are not leading blocks: the permutation brings them to the
    front first; low-rank operands with noise, truncated at eps = 1e-2."""
    x = _dense_tt(40, [6, 5, 4, 3], [1, 3, 4, 2, 1], np.float64)
    y = _dense_tt(41, [4, 6, 5, 3], [1, 2, 3, 2, 1], np.float64)
    for a, b in pairs:
        assert x.shape[a] == y.shape[b]
    rng = np.random.default_rng(42)
    x = x + 1e-4 * np.linalg.norm(x) * rng.standard_normal(x.shape) / np.sqrt(x.size)
    y = y + 1e-4 * np.linalg.norm(y) * rng.standard_normal(y.shape) / np.sqrt(y.size)
    _check_dense_contraction(x, y, pairs, 1e-2, np.float64, f"interior {pairs}")


def test_large_unfoldings_cluster_sweeps():
    """Unfoldings too large for one CTA's shared memory (20 x 8000, 400 x 400,
    8000 x 20 in float32) are swept across the cluster: exact ranks of a
    low-rank tensor, and a full-rank Gaussian tensor within its guarantee
    with left-orthonormal cores."""
    xh = _dense_tt(60, [20, 20, 20, 5, 4], [1, 12, 40, 15, 4, 1], np.float32)
    cores = _decompose(xh, 1e-5)
    assert [c.shape[0] for c in cores] + [1] == [1, 12, 40, 15, 4, 1]
    _check_valid(xh, cores, 1e-5, np.float32, "low rank 20^3x5x4")
    rng = np.random.default_rng(61)
    g = rng.standard_normal((20, 20, 20, 5, 4)).astype(np.float32)
    cores = _decompose(g, 1e-6)
    assert [c.shape[0] for c in cores] + [1] == [1, 20, 400, 20, 4, 1]
    _check_valid(g, cores, 1e-6, np.float32, "gaussian 20^3x5x4")


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("shape", [(20, 20, 20, 20), (333, 400)])
def test_square_unfoldings_vector_split_sweeps(shape, dtype):
    """Unfoldings with many vectors of moderate length (400 x 400 of a 20^4
    tensor; 333 x 400, an odd count of vectors, so the tournament carries an
    empty one) are swept with the vectors spread over the cluster: a Gaussian
    tensor within its guarantee with left-orthonormal cores, and a low-rank
    one of the same shape at its exact ranks."""
    rng = np.random.default_rng(sum(shape))
    g = rng.standard_normal(shape).astype(dtype)
    eps = 1e-10 if dtype == np.float64 else 1e-6
    cores = _decompose(g, eps)
    _check_valid(g, cores, eps, dtype, f"gaussian {shape} {np.dtype(dtype).name}")
    ranks = [1] + [min(7 + 3 * k, 60) for k in range(len(shape) - 1)] + [1]
    xh = _dense_tt(70 + len(shape), list(shape), ranks, dtype)
    cores = _decompose(xh, eps if dtype == np.float64 else 1e-5)
    assert [c.shape[0] for c in cores] + [1] == ranks
