"""GPU parity of the full and chain-layout partial contractions against the
float64 oracle, element by element, through the C ABI.

Tolerances (normalised error eps = |z - z*| / (||X||_F ||Y||_F)):
  float64 storage: 1e-12      float32 storage: 1e-5
Partial results: every emitted core is compared; copied cores bit-exactly,
the boundary core C entrywise with the Cauchy-Schwarz scale of K.
"""
import numpy as np
import pytest

import oracle as O
from helpers import dense_cs_eps, cs_bound, norm_scale, to_dev, to_host
from paper_2109_00626_gb300 import inputs as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2109_00626_gb300 as T  # noqa: E402

TOL = {np.float64: 1e-12, np.float32: 1e-5}
TDT = {np.float64: torch.float64, np.float32: torch.float32}


def _full(x, y, split=False):
    op = T.FullContraction(to_dev(x), to_dev(y), split=split)
    op()
    torch.cuda.synchronize()
    st = int(op.status.item())
    if split:
        return float(op.out.item()), int(op.log2.item()), st
    return float(op.out.item()), st


def _check_full(x, y, dt):
    z, st = _full(x, y)
    assert st == 0
    want = O.contract_full(x, y)
    eps = abs(z - want) / norm_scale(x, y)
    assert eps <= TOL[dt], (z, want, eps)
    return z, want


def test_full_small_fp64():
    x, y = G.small_fp64(0)
    z, want = _check_full(x, y, np.float64)
    # kappa is modest here, so the plain relative error holds as well
    assert abs(z - want) <= 1e-12 * abs(want) * 1e3


def test_full_order10_r64_fp32():
    x, y = G.order10_r64(0)
    _check_full(x, y, np.float32)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_full_ragged_fp32(seed):
    rng = np.random.default_rng(100 + seed)
    n = [1, 2, 3, 5][seed]
    modes = [int(v) for v in rng.choice([1, 2, 31, 7, 16], size=n)]
    rx = [1] + [int(v) for v in rng.choice([1, 3, 17, 33, 127], size=n - 1)] + [1]
    ry = [1] + [int(v) for v in rng.choice([1, 3, 17, 33, 127], size=n - 1)] + [1]
    x = G.random_tt(rng, modes, rx, np.float32)
    y = G.random_tt(rng, modes, ry, np.float32)
    _check_full(x, y, np.float32)


@pytest.mark.parametrize("r", [1, 3, 17, 33, 64])
def test_full_ragged_fp64(r):
    rng = np.random.default_rng(r)
    modes = [3, 31, 2, 5]
    rx = [1, r, max(1, r // 2), r, 1]
    ry = [1, max(1, r - 1), r, 2, 1]
    x = G.random_tt(rng, modes, rx, np.float64)
    y = G.random_tt(rng, modes, ry, np.float64)
    _check_full(x, y, np.float64)


def test_full_rank1_closed_form_fp64():
    rng = np.random.default_rng(9)
    xs = [rng.standard_normal(16) for _ in range(12)]
    ys = [rng.standard_normal(16) for _ in range(12)]
    want = float(np.prod([np.dot(a, b) for a, b in zip(xs, ys)]))
    z, st = _full(G.rank1_tt(xs), G.rank1_tt(ys))
    assert st == 0 and abs(z - want) <= 1e-12 * abs(want)


def test_full_renormalisation_split_scale():
    """Cores scaled by 2^40 each: z = 2^(40*2N) <X0,Y0> leaves float32's range
    long before the end; the split result (mantissa, log2) must still match."""
    x, y = G.pair(21, [8] * 6, G.tt_ranks(6, 16), G.tt_ranks(6, 16), np.float32)
    xs = [c * np.float32(2.0**40) for c in x]
    ys = [c * np.float32(2.0**40) for c in y]
    m, e, st = _full(xs, ys, split=True)
    assert st == 0
    want = O.contract_full(x, y)
    got = np.ldexp(m, e - 2 * 6 * 40)
    assert abs(got - want) / norm_scale(x, y) <= 1e-5
    # unsplit: 2^480 * z fits in double
    z, st = _full(xs, ys)
    assert st == 0 and abs(np.ldexp(z, -480) - want) / norm_scale(x, y) <= 1e-5


@pytest.mark.parametrize("dt,n", [(np.float32, 2), (np.float32, 3), (np.float32, 10), (np.float32, 11), (np.float64, 7)])
def test_full_both_ends_matches_one_sweep(dt, n):
    """With a workspace the full contraction runs from both ends (two
    clusters meeting in the middle); without one, as a single sweep.  Both
    must agree with the oracle."""
    rng = np.random.default_rng(200 + n)
    modes = [int(v) for v in rng.integers(1, 20, size=n)]
    rmax = 64 if dt == np.float64 else 100
    rx = [1] + [int(v) for v in rng.integers(1, rmax, size=n - 1)] + [1]
    ry = [1] + [int(v) for v in rng.integers(1, rmax, size=n - 1)] + [1]
    x = G.random_tt(rng, modes, rx, dt)
    y = G.random_tt(rng, modes, ry, dt)
    want = O.contract_full(x, y)
    both = T.FullContraction(to_dev(x), to_dev(y))
    one = T.FullContraction(to_dev(x), to_dev(y))
    assert both.ws_bytes > 0
    one.ws_bytes = 0  # no workspace: one sweep
    n0 = T.launch_count()
    both()
    one()
    torch.cuda.synchronize()
    assert int(both.status.item()) == 0 and int(one.status.item()) == 0
    for op in (both, one):
        z = float(op.out.item())
        assert abs(z - want) / norm_scale(x, y) <= TOL[dt], (z, want)
    assert T.launch_count() - n0 == 2


def test_full_overflow_status_without_split():
    x, y = G.pair(22, [4] * 4, G.tt_ranks(4, 4), G.tt_ranks(4, 4), np.float64)
    xs = [c * 2.0**300 for c in x]
    ys = [c * 2.0**300 for c in y]
    z, st = _full(xs, ys)
    assert st & 2 and np.isinf(z)


def test_full_nonfinite_status():
    x, y = G.small_fp64(1)
    x[1] = x[1].copy()
    x[1][0, 0, 0] = np.nan
    z, st = _full(x, y)
    assert st & 1


def _check_chain(x, y, mask, dt):
    xd, yd = to_dev(x), to_dev(y)
    op = T.PartialContraction(xd, yd, mask)
    op()
    torch.cuda.synchronize()
    assert int(op.status.item()) == 0
    got = to_host(op.z)
    want, perm = O.partial_chain(x, y, mask)
    assert perm == op.perm
    assert [g.shape for g in got] == [w.shape for w in want]
    side, s = O.end_block(mask)
    m = len(x) - s
    for p, (g, w) in enumerate(zip(got, want)):
        if p == m - 1:
            # C = boundary core joined with K: scale by |Gx| and the CS bound of K
            kb = cs_bound(x, y, side, s) if s > 0 else np.ones((1, 1))
            gxb = x[s] if side == "lead" else x[m - 1]
            scale = np.abs(gxb).max() * kb.max() * np.sqrt(gxb.shape[0] if side == "lead" else gxb.shape[2])
            assert np.abs(g - w).max() <= TOL[dt] * scale, (np.abs(g - w).max(), scale)
        else:
            np.testing.assert_array_equal(g, w)
    return got, want


def test_partial_small_fp64_dense():
    x, y = G.small_fp64(0)
    mask = [0, 0, 1, 1]
    got, _ = _check_chain(x, y, mask, np.float64)
    dense_want = O.tcp(O.tt_to_dense(x), O.tt_to_dense(y), [2, 3])
    _, perm = O.partial_chain(x, y, mask)
    dense_got = O.chain_to_dense(got, perm)
    assert np.abs(dense_got - dense_want).max() <= 1e-12 * norm_scale(x, y)


def test_partial_order10_leading6_fp32():
    x, y = G.order10_r64(0)
    _check_chain(x, y, [1] * 6 + [0] * 4, np.float32)


@pytest.mark.parametrize("mask", [[1, 0, 0, 0, 0], [0, 0, 0, 1, 1], [1, 1, 1, 1, 0], [0, 1, 1, 1, 1], [0, 0, 0, 0, 0]])
def test_partial_ragged_fp64(mask):
    rng = np.random.default_rng(sum(mask) + 7 * mask[0])
    modes = [3, 2, 31, 2, 5]
    x = G.random_tt(rng, modes, [1, 3, 17, 33, 2, 1], np.float64)
    y = G.random_tt(rng, modes, [1, 5, 1, 9, 4, 1], np.float64)
    got, _ = _check_chain(x, y, mask, np.float64)
    dense_want = O.tcp(O.tt_to_dense(x), O.tt_to_dense(y), [k for k in range(5) if mask[k]])
    _, perm = O.partial_chain(x, y, mask)
    assert np.abs(O.chain_to_dense(got, perm) - dense_want).max() <= 1e-12 * norm_scale(x, y)


def test_partial_split_scale_fp32():
    x, y = G.pair(31, [4] * 6, G.tt_ranks(6, 8), G.tt_ranks(6, 8), np.float32)
    xs = [c * np.float32(2.0**30) for c in x]
    ys = [c * np.float32(2.0**30) for c in y]
    mask = [1, 1, 1, 1, 0, 0]
    op = T.PartialContraction(to_dev(xs), to_dev(ys), mask, split=True)
    op()
    torch.cuda.synchronize()
    assert int(op.status.item()) == 0
    e = int(op.log2.item())
    got = to_host(op.z)
    want, perm = O.partial_chain(x, y, mask)
    # undo: C carries 2^e and the input scaling of 4 X cores (K) and 1 X core (C) and 4 Y cores (K)
    c = got[1] * 2.0 ** (e - 30 * 9)
    # the represented tensor against Eq. 8, within 1e-5 of the per-entry
    # Cauchy-Schwarz scale (the float64 oracle on the unscaled float32 cores)
    x64 = [np.asarray(g, dtype=np.float64) for g in x]
    y64 = [np.asarray(g, dtype=np.float64) for g in y]
    cores = [np.asarray(g, dtype=np.float64) * 2.0**-30 for g in got]
    cores[1] = c
    dense = O.chain_to_dense(cores, perm)
    ref = O.tcp(O.tt_to_dense(x64), O.tt_to_dense(y64), [0, 1, 2, 3])
    eps = dense_cs_eps(dense, ref, x64, y64, [0, 1, 2, 3])
    print(f"split-scale chain: cs_eps={eps:.2e}")
    assert eps <= 1e-5


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("I", [1, 7])
def test_order1_full_and_outer_product(dt, I):
    """Order 1: the full contraction is the inner product of two vectors (the
    last-mode float64 sum alone; no sweep from both ends), and the partial
    contraction over no mode is their outer product as a two-core train."""
    rng = np.random.default_rng(11 + I)
    x = G.random_tt(rng, [I], [1, 1], dt)
    y = G.random_tt(rng, [I], [1, 1], dt)
    z, st = _full(x, y)
    assert st == 0
    want = float(np.dot(x[0].reshape(-1).astype(np.float64), y[0].reshape(-1).astype(np.float64)))
    assert abs(z - want) <= TOL[dt] * norm_scale(x, y)
    got, _ = _check_chain(x, y, [0], dt)
    _, perm = O.partial_chain(x, y, [0])
    dense = O.chain_to_dense(got, perm)
    np.testing.assert_array_equal(dense, np.outer(x[0].reshape(-1).astype(np.float64), y[0].reshape(-1).astype(np.float64)))


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize(
    "rx,scale",
    [([1, 8, 8, 8, 1], 0), ([1, 64, 600, 64, 1], 0), ([1, 1024, 17, 1024, 1], 0), ([1, 16, 16, 16, 1], 40)],
)
def test_full_rank1_y_fold_and_chain(dt, rx, scale):
    """A Y of rank 1 (the sum of a TT's entries is the case y = ones) takes
    the fold-and-chain path: z against the oracle for ranks of X up to 1024
    (vectors longer than a block: several passes per step), a mode of size 1,
    cores scaled by 2^40 each (renormalised on the way), and the split output
    (mantissa, log2) against the folded one."""
    rng = np.random.default_rng(sum(rx) + scale)
    modes = [3, 16, 1, 7]
    x = G.random_tt(rng, modes, rx, dt)
    if scale:
        x = [c * dt(2.0**scale) for c in x]
    y = G.random_tt(rng, modes, [1] * 5, dt)
    z, st = _full(x, y)
    assert st == 0
    want = O.contract_full(x, y)
    eps = abs(z - want) / norm_scale(x, y)
    print(f"rank-1 y {dt.__name__} {rx[1:-1]} 2^{scale}: eps {eps:.2e}")
    assert eps <= TOL[dt], (z, want, eps)
    m, e, st2 = _full(x, y, split=True)
    assert st2 == 0
    assert m * 2.0**e == z


def test_full_rank1_y_sum_of_entries_and_overflow():
    """y = ones: z is the sum of X's entries (dense brute force); scaled past
    the float64 range, the folded output overflows with TT_STATUS_OVERFLOW
    while the split output stays finite."""
    rng = np.random.default_rng(5)
    modes = [4, 3, 5]
    x = G.random_tt(rng, modes, [1, 6, 7, 1], np.float64)
    ones = [np.ones((1, i, 1)) for i in modes]
    z, st = _full(x, ones)
    assert st == 0
    want = O.tt_to_dense(x).sum()
    assert abs(z - want) <= 1e-12 * np.abs(O.tt_to_dense(x)).sum()
    xs = [c * 2.0**400 for c in x]
    z, st = _full(xs, ones)
    assert st & 2 and np.isinf(z)
    m, e, st = _full(xs, ones, split=True)
    assert st == 0 and np.isfinite(m)
    assert abs(m * 2.0 ** (e - 1200) - want) <= 1e-12 * np.abs(O.tt_to_dense(x)).sum()
