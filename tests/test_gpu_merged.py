"""GPU parity of the merged (TT-matrix) layout of a partial contraction over
any contracted set, against the oracle's merged cores and the dense Eq. 8."""
import numpy as np
import pytest

import oracle as O
from helpers import dense_cs_eps, norm_scale, to_dev, to_host
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
    want, perm = O.partial_merged(x, y, mask)
    _f32_check(x, y, mask, got, want, perm)


def _rel_err(got, want):
    return max(np.abs(g - w.reshape(g.shape)).max() / max(np.abs(w).max(), 1e-300) for g, w in zip(got, want))


def _f32_check(x, y, mask, got, want, perm):
    """float32 merged cores: the represented tensor within 1e-5 of the
    per-entry Cauchy-Schwarz scale of Eq. 8's Z (the float64 oracle's dense
    result on the same float32 cores), and every core within 1e-5 of its
    largest entry (the library and the oracle fold the environments into the
    same cores)."""
    x64 = [np.asarray(c, dtype=np.float64) for c in x]
    y64 = [np.asarray(c, dtype=np.float64) for c in y]
    contracted = [k for k in range(len(x)) if mask[k]]
    dense = O.merged_to_dense([g.reshape(w.shape) for g, w in zip(got, want)], perm)
    ref = O.tcp(O.tt_to_dense(x64), O.tt_to_dense(y64), contracted)
    eps = dense_cs_eps(dense, ref, x64, y64, contracted)
    rel = _rel_err(got, want)
    print(f"merged {''.join(map(str, mask))}: cs_eps={eps:.2e} core_rel={rel:.2e}")
    assert eps <= 1e-5 and rel <= 1e-5


@pytest.mark.parametrize("mask", [[int(b) for b in format(v, "06b")] for v in range(64) if bin(v).count("1") == 3])
def test_merged_all_three_of_six_fp32(mask):
    """Every contracted set of three of six modes (modes 8, ranks 16, float32):
    Kronecker cores, interior runs through the transfer matrix, trailing runs
    through the right environment, the left environment folded into core 0."""
    x, y = G.pair(13, [8] * 6, G.tt_ranks(6, 16), G.tt_ranks(6, 16), np.float32)
    op, got = _run(x, y, mask)
    assert int(op.status.item()) == 0
    want, perm = O.partial_merged(x, y, mask)
    assert op.perm == perm
    _f32_check(x, y, mask, got, want, perm)


@pytest.mark.parametrize("mask", [[0, 1, 1, 1, 0, 1, 0], [0, 0, 1, 1, 1, 1, 0], [1, 0, 1, 1, 0, 1, 1], [0, 1, 1, 1, 1, 1, 1]])
def test_merged_long_runs_fp64(mask):
    """Interior runs of up to four modes, ragged ranks (columns not a multiple
    of the vector width), float64."""
    rng = np.random.default_rng(31 + sum(m << k for k, m in enumerate(mask)))
    modes = [3, 2, 3, 2, 3, 2, 3]
    x = G.random_tt(rng, modes, [1, 3, 5, 2, 6, 3, 5, 1], np.float64)
    y = G.random_tt(rng, modes, [1, 2, 3, 7, 2, 5, 3, 1], np.float64)
    op, got = _run(x, y, mask)
    assert int(op.status.item()) == 0
    want, perm = O.partial_merged(x, y, mask)
    dense = O.merged_to_dense([g.reshape(w.shape) for g, w in zip(got, want)], perm)
    ref = O.tcp(O.tt_to_dense(x), O.tt_to_dense(y), [k for k in range(7) if mask[k]])
    assert np.abs(dense - ref).max() <= 1e-12 * norm_scale(x, y)


@pytest.mark.parametrize("dtype,tol", [(np.float32, None), (np.float64, 1e-12)])
def test_merged_rank24_interior_run(dtype, tol):
    """Ranks 24 (the transfer matrix has 576 rows of 576), a two-mode interior
    run after an interior free core, and a free core after it."""
    rng = np.random.default_rng(77)
    modes = [3, 3, 3, 3, 3]
    x = G.random_tt(rng, modes, [1, 24, 24, 24, 24, 1], dtype)
    y = G.random_tt(rng, modes, [1, 24, 24, 24, 24, 1], dtype)
    mask = [1, 0, 1, 1, 0]
    op, got = _run(x, y, mask)
    assert int(op.status.item()) == 0
    want, perm = O.partial_merged(x, y, mask)
    if tol is None:
        _f32_check(x, y, mask, got, want, perm)
    else:
        assert _rel_err(got, want) <= tol


@pytest.mark.parametrize("mask", [[1, 0, 1, 1, 1, 1, 0], [0, 0, 1, 1, 1, 1, 0]])
def test_merged_run_scales_beyond_float32(mask):
    """An interior run whose transfer matrix is of order 2^240 (past the float32
    range) between free cores of order 2^-100 each: the power-of-two scales of
    the transfer matrix and of P carry the result (of order 2^36), where
    Gy P taken at the scale of the inputs would underflow.  The first set puts
    the small cores in the left core (E_L folded in), the second in an
    interior one (P, then the rows)."""
    rng = np.random.default_rng(5)
    modes = [4] * 7
    r = [1, 6, 6, 6, 6, 6, 6, 1]
    x = G.random_tt(rng, modes, r, np.float64)
    y = G.random_tt(rng, modes, r, np.float64)
    for k in (2, 3, 4, 5):
        x[k] = x[k] * 2.0**30
        y[k] = y[k] * 2.0**30
    x[1] = x[1] * 2.0**-100
    y[1] = y[1] * 2.0**-100
    x32 = [c.astype(np.float32) for c in x]
    y32 = [c.astype(np.float32) for c in y]
    op, got = _run(x32, y32, mask)
    assert int(op.status.item()) == 0
    want, perm = O.partial_merged([c.astype(np.float64) for c in x32], [c.astype(np.float64) for c in y32], mask)
    assert all(np.isfinite(g).all() for g in got)
    _f32_check(x32, y32, mask, got, want, perm)


def test_merged_zero_rows_of_transfer():
    """Rows of the transfer matrix that vanish (a zero row of the first run
    core) and a run core that vanishes outright."""
    rng = np.random.default_rng(9)
    modes = [3] * 6
    r = [1, 4, 4, 4, 4, 4, 1]
    x = G.random_tt(rng, modes, r, np.float64)
    y = G.random_tt(rng, modes, r, np.float64)
    x[2][1] = 0.0
    y[2][3] = 0.0
    op, got = _run(x, y, [0, 0, 1, 1, 0, 0])
    assert int(op.status.item()) == 0
    want, _ = O.partial_merged(x, y, [0, 0, 1, 1, 0, 0])
    assert _rel_err(got, want) <= 1e-12
    x[3] = np.zeros_like(x[3])
    op, got = _run(x, y, [0, 0, 1, 1, 0, 0])
    assert int(op.status.item()) == 0
    want, _ = O.partial_merged(x, y, [0, 0, 1, 1, 0, 0])
    assert all(np.abs(g - w.reshape(g.shape)).max() == 0.0 for g, w in zip(got, want))


@pytest.mark.parametrize("mask", [[0, 1, 0, 1, 0], [1, 0, 1, 0, 1], [0, 1, 1, 0, 0], [0, 0, 1, 1, 0], [1, 1, 0, 0, 0]])
def test_merged_unequal_free_modes_fp64(mask):
    """Free modes of X and Y of different sizes (I != J on the free positions;
    equal on S), float64, against the dense Eq. 8."""
    rng = np.random.default_rng(8 + sum(m << k for k, m in enumerate(mask)))
    mx = [3, 2, 4, 2, 3]
    my = [m if mask[k] else m + 2 for k, m in enumerate(mx)]
    x = G.random_tt(rng, mx, [1, 2, 5, 3, 2, 1], np.float64)
    y = G.random_tt(rng, my, [1, 3, 1, 4, 2, 1], np.float64)
    op, got = _run(x, y, mask)
    assert int(op.status.item()) == 0
    want, perm = O.partial_merged(x, y, mask)
    assert [g.shape for g in got] == [(w.shape[0], w.shape[1] * w.shape[2], w.shape[3]) for w in want]
    dense = O.merged_to_dense([g.reshape(w.shape) for g, w in zip(got, want)], perm)
    ref = O.tcp(O.tt_to_dense(x), O.tt_to_dense(y), [k for k in range(5) if mask[k]])
    assert np.abs(dense - ref).max() <= 1e-12 * norm_scale(x, y)


@pytest.mark.parametrize("dtype,tol", [(np.float32, None), (np.float64, 1e-12)])
def test_merged_transfer_slice_chunks(dtype, tol):
    """A run mode of ranks 64 -> 64 with 16 slices: the transfer kernel's slice
    products do not fit shared memory at once and go in chunks (8 slices in
    float32, 4 in float64)."""
    rng = np.random.default_rng(64)
    modes = [3, 3, 16, 3, 3, 3]
    r = [1, 2, 64, 64, 2, 2, 1]
    x = G.random_tt(rng, modes, r, dtype)
    y = G.random_tt(rng, modes, r, dtype)
    mask = [0, 1, 1, 1, 0, 0]
    op, got = _run(x, y, mask)
    assert int(op.status.item()) == 0
    want, perm = O.partial_merged(x, y, mask)
    if tol is None:
        _f32_check(x, y, mask, got, want, perm)
    else:
        assert _rel_err(got, want) <= tol
