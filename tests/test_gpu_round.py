"""GPU parity of TT rounding (tt_round: right-orthonormal sweep, then the
TT-SVD's truncation rule from the left) against the float64 oracle
(tt_round) and the definitions it must satisfy.

- X + X (ranks doubled) rounds back to X's ranks at eps ~ 0 and represents
  2X (1e-12 float64, 1e-5 float32 of its largest entry);
- an over-parametrised TT (a rank above what its neighbours allow) comes out
  with the exact ranks;
- on random TTs the error stays within eps ||X||_F (+ rounding), the cores
  but the last are left-orthonormal, and the ranks are the oracle's (same
  singular values) unless a threshold lies within 1e-6 of a tail of them;
- a merged-layout result rounded as a TT of modes I J stays within
  eps ||Z||_F of Eq. 8's Z;
- the max_rank cap."""
import numpy as np
import pytest

import oracle as O
from helpers import to_dev
from paper_2109_00626_gb300 import inputs as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2109_00626_gb300 as T  # noqa: E402

TOL = {np.float64: 1e-12, np.float32: 1e-5}


def _tt_sum(a, b):
    n = len(a)
    out = []
    for k, (ga, gb) in enumerate(zip(a, b)):
        ra, i_dim, ra2 = ga.shape
        rb, _, rb2 = gb.shape
        if k == 0:
            out.append(np.concatenate([ga, gb], axis=2))
        elif k == n - 1:
            out.append(np.concatenate([ga, gb], axis=0))
        else:
            g = np.zeros((ra + rb, i_dim, ra2 + rb2), dtype=ga.dtype)
            g[:ra, :, :ra2] = ga
            g[ra:, :, ra2:] = gb
            out.append(g)
    return out


def _round(cores, eps, max_rank=0):
    out = T.tt_round(to_dev(cores), eps, max_rank)
    torch.cuda.synchronize()
    return [c.cpu().numpy().astype(np.float64) for c in out]


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_round_sum_recovers_ranks(dtype):
    rng = np.random.default_rng(1)
    x = G.random_tt(rng, [4, 3, 5, 3, 4, 2], [1, 3, 4, 6, 4, 2, 1], dtype)
    r = _round(_tt_sum(x, x), 1e-12 if dtype == np.float64 else 1e-5)
    assert [c.shape[0] for c in r] + [1] == [1, 3, 4, 6, 4, 2, 1]
    d = O.tt_to_dense([c.astype(np.float64) for c in x])
    err = np.abs(O.tt_to_dense(r) - 2 * d).max() / np.abs(2 * d).max()
    print(f"X + X {np.dtype(dtype).name}: err {err:.2e}")
    assert err <= TOL[dtype] * 10


def test_round_overparametrised_to_exact_ranks():
    rng = np.random.default_rng(2)
    x = G.random_tt(rng, [2, 3, 2, 2], [1, 2, 30, 4, 1], np.float64)
    r = _round(x, 1e-13)
    # rank 30 after mode 2 is above 2 * 3 and 2 * 2 * ... : at most min(6, 8) = 6, and the neighbours cap it further
    want = [c.shape[0] for c in O.tt_round(x, 1e-13)] + [1]
    assert [c.shape[0] for c in r] + [1] == want
    assert want[2] <= 6
    d = O.tt_to_dense(x)
    assert np.abs(O.tt_to_dense(r) - d).max() <= 1e-12 * np.abs(d).max()


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("eps", [0.02, 0.2, 0.5])
def test_round_random_tt(eps, dtype):
    rng = np.random.default_rng(3)
    y = G.random_tt(rng, [4, 3, 5, 3, 4], [1, 4, 8, 7, 4, 1], dtype)
    y64 = [c.astype(np.float64) for c in y]
    t = _round(y, eps)
    d = O.tt_to_dense(y64)
    err = np.linalg.norm(O.tt_to_dense(t) - d) / np.linalg.norm(d)
    print(f"random {np.dtype(dtype).name} eps={eps}: ranks {[c.shape[0] for c in t] + [1]} err {err:.3e}")
    assert err <= eps + 10 * TOL[dtype]
    for g in t[:-1]:
        m = g.reshape(-1, g.shape[2])
        assert np.abs(m.T @ m - np.eye(m.shape[1])).max() <= 10 * TOL[dtype] * np.sqrt(m.shape[0])
    want = O.tt_round(y64, eps)
    near = False
    tol = eps * np.linalg.norm(d) / 2.0
    for k in range(4):
        sv = np.linalg.svd(d.reshape(int(np.prod(d.shape[: k + 1])), -1), compute_uv=False)
        tails = np.sqrt(np.cumsum(sv[::-1] ** 2))[::-1]
        near |= bool(np.min(np.abs(tails - tol)) <= 1e-6 * tol)
    if not near:
        assert [c.shape[0] for c in t] == [c.shape[0] for c in want]


def test_round_merged_result():
    """The merged layout's cores (ranks R^x R^y = 64) rounded as a TT of
    modes I J: within eps ||Z|| of Eq. 8."""
    x, y = G.pair(4, [3, 4, 3, 4, 3], [1, 8, 8, 8, 8, 1], [1, 8, 8, 8, 8, 1], np.float64)
    mask = [0, 1, 0, 1, 0]
    op = T.PartialContraction(to_dev(x), to_dev(y), mask, layout="merged")
    op()
    torch.cuda.synchronize()
    eps = 1e-3
    rounded = T.round_merged(op.z, eps)
    torch.cuda.synchronize()
    got = O.merged_to_dense([c.cpu().numpy().reshape(c.shape[0], 3, 3, c.shape[2]) for c in rounded], op.perm)
    want = O.tcp(O.tt_to_dense(x), O.tt_to_dense(y), [1, 3])
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    ranks_in = [c.shape[0] for c in op.z] + [1]
    ranks_out = [c.shape[0] for c in rounded] + [1]
    print(f"merged rounding: ranks {ranks_in} -> {ranks_out}, err {err:.2e}")
    assert err <= eps * (1 + 1e-9) + 1e-12
    assert all(a >= b for a, b in zip(ranks_in, ranks_out))


def test_round_max_rank_cap():
    rng = np.random.default_rng(5)
    y = G.random_tt(rng, [5, 5, 5, 5], [1, 5, 9, 5, 1], np.float64)
    t = _round(y, 0.0, max_rank=3)
    assert [c.shape[0] for c in t] + [1] == [1, 3, 3, 3, 1]


def test_round_large_unfoldings_cluster_sweeps():
    """A merged result of ranks 64 and modes 8 x 8 (unfoldings of 4096 x 64,
    swept across the cluster) rounded at eps 1e-4: within eps of Eq. 8, and
    the ranks equal the oracle's rounding unless a threshold is close."""
    x, y = G.pair(6, [8] * 5, G.tt_ranks(5, 8), G.tt_ranks(5, 8), np.float32)
    mask = [0, 1, 0, 1, 0]
    op = T.PartialContraction(to_dev(x), to_dev(y), mask, layout="merged")
    op()
    torch.cuda.synchronize()
    eps = 1e-4
    rounded = T.round_merged(op.z, eps)
    torch.cuda.synchronize()
    got = O.merged_to_dense([c.cpu().numpy().astype(np.float64).reshape(c.shape[0], 8, 8, c.shape[2])
                             for c in rounded], op.perm)
    x64 = [c.astype(np.float64) for c in x]
    y64 = [c.astype(np.float64) for c in y]
    want = O.tcp(O.tt_to_dense(x64), O.tt_to_dense(y64), [1, 3])
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    print(f"merged rank-64 rounding: ranks {[c.shape[0] for c in rounded] + [1]}, err {err:.2e}")
    assert err <= eps + 1e-5
