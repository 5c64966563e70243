"""GPU parity of the factored partial contraction (tt_contract_factored: any
contracted set S, the runs between free positions as matrices over pair
indices, the free cores as the Kronecker factors of the merged cores)
against the float64 oracle (partial_factored, factored_to_dense).

Run matrices are compared entry by entry within their per-entry
Cauchy-Schwarz scale, |T[(a,b),(c,d)]| <= sqrt(Tx[(a,a),(c,c)] Ty[(b,b),(d,d)])
(Tx, Ty the runs of X with X and of Y with Y): 1e-12 (float64) / 1e-5
(float32).  The represented tensor is compared with the dense Eq. 8 on small
cases within 1e-12 / 1e-5 of its per-entry scale ||X[., i_F]|| ||Y[., j_F]||.
At rank 64 (order 8, modes 16, an interior run of three modes: a 4096 x 4096
transfer matrix) sampled rows are checked against the oracle's sweep from the
basis environment e_a e_b^T, and the end environments in full."""
import numpy as np
import pytest

import oracle as O
from helpers import dense_cs_eps, to_dev
from paper_2109_00626_gb300 import inputs as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2109_00626_gb300 as T  # noqa: E402

TOL = {np.float64: 1e-12, np.float32: 1e-5}


def _gpu_runs(x, y, mask):
    op = T.FactoredContraction(to_dev(x), to_dev(y), mask)
    op()
    torch.cuda.synchronize()
    assert int(op.status.item()) == 0
    runs = []
    for r in op.runs():
        if r is None:
            runs.append(None)
            continue
        tm, lg = r
        runs.append(np.ldexp(tm.cpu().numpy().astype(np.float64), lg.cpu().numpy()[:, None]))
    return op.free_pos, runs


def _run_scale(xc, yc, t, free, n):
    """sqrt(Tx[(a,a),(c,c)] Ty[(b,b),(d,d)]) for every entry ((a,b),(c,d)) of
    run t, with Tx and Ty the same run of X with X and of Y with Y (the only
    run of the self-contraction over the run's modes)."""
    k0 = 0 if t == 0 else free[t - 1] + 1
    k1 = n if t == len(free) else free[t]
    sub = [1 if k0 <= k < k1 else 0 for k in range(n)]
    tx = [r for r in O.partial_factored(xc, xc, sub)[1] if r is not None][0]
    ty = [r for r in O.partial_factored(yc, yc, sub)[1] if r is not None][0]
    ax = xc[k0].shape[0] if t > 0 else 1
    ay = yc[k0].shape[0] if t > 0 else 1
    cx = xc[k1 - 1].shape[2] if t < len(free) else 1
    cy = yc[k1 - 1].shape[2] if t < len(free) else 1
    dx = np.abs(np.array([[tx[a * ax + a, c * cx + c] for c in range(cx)] for a in range(ax)]))
    dy = np.abs(np.array([[ty[b * ay + b, d * cy + d] for d in range(cy)] for b in range(ay)]))
    return np.sqrt(np.einsum("ac,bd->abcd", dx, dy).reshape(ax * ay, cx * cy))


MASKS = [[1, 0, 1, 1, 0], [0, 1, 0, 1, 0], [1, 1, 0, 0, 1], [0, 0, 0, 0, 0], [1, 1, 1, 1, 0], [0, 1, 1, 1, 1],
         [1, 0, 0, 0, 1]]


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("mask", MASKS)
def test_factored_small_against_dense(mask, dtype):
    rng = np.random.default_rng(sum(v << k for k, v in enumerate(mask)) + 50)
    modes = [3, 4, 2, 3, 2]
    x = G.random_tt(rng, modes, [1, 5, 7, 3, 4, 1], dtype)
    y = G.random_tt(rng, modes, [1, 2, 6, 5, 3, 1], dtype)
    free, runs = _gpu_runs(x, y, mask)
    x64 = [c.astype(np.float64) for c in x]
    y64 = [c.astype(np.float64) for c in y]
    want_free, want = O.partial_factored(x64, y64, mask)
    assert free == want_free
    for t, (g, w) in enumerate(zip(runs, want)):
        assert (g is None) == (w is None)
        if g is None:
            continue
        err = np.max(np.abs(g - w) / _run_scale(x64, y64, t, free, 5))
        assert err <= TOL[dtype], (t, err)
    dense = O.factored_to_dense(x64, y64, free, runs)
    contracted = [k for k in range(5) if mask[k]]
    ref = O.tcp(O.tt_to_dense(x64), O.tt_to_dense(y64), contracted)
    if contracted:
        eps = dense_cs_eps(dense, ref, x64, y64, contracted)
    else:
        # nothing contracted: no run, Z is the outer product of the operands
        # (the per-entry scale degenerates to |X[i]| |Y[j]|; compare normwise)
        eps = np.abs(dense - ref).max() / (np.abs(ref).max())
    print(f"factored {''.join(map(str, mask))} {np.dtype(dtype).name}: dense cs eps {eps:.2e}")
    assert eps <= TOL[dtype]


def test_factored_order8_rank16_random_sets():
    """The merged layout's order-8 size (order 8, modes 8, ranks 16, float32)
    over random sets of four modes: every run matrix against the oracle."""
    x, y = G.pair(13, [8] * 8, G.tt_ranks(8, 16), G.tt_ranks(8, 16), np.float32)
    x64 = [c.astype(np.float64) for c in x]
    y64 = [c.astype(np.float64) for c in y]
    rng = np.random.default_rng(8)
    for _ in range(4):
        sset = sorted(rng.choice(8, size=4, replace=False).tolist())
        mask = [1 if k in sset else 0 for k in range(8)]
        free, runs = _gpu_runs(x, y, mask)
        _, want = O.partial_factored(x64, y64, mask)
        for t, (g, w) in enumerate(zip(runs, want)):
            if g is None:
                continue
            err = np.max(np.abs(g - w) / _run_scale(x64, y64, t, free, 8))
            print(f"order8 r16 S={sset} run {t}: {g.shape} err {err:.2e}")
            assert err <= 1e-5


def test_factored_rank64_interior_run():
    """Order 8, modes 16, ranks 64, float32, S = {0, 3, 4, 5}: E_L (1 x 4096),
    a 4096 x 4096 transfer matrix of modes 3-5 (its rows sampled against the
    oracle's sweep from e_a e_b^T), E_R none (mode 7 free)."""
    x, y = G.pair(3, [16] * 8, G.tt_ranks(8, 64), G.tt_ranks(8, 64), np.float32)
    x64 = [c.astype(np.float64) for c in x]
    y64 = [c.astype(np.float64) for c in y]
    mask = [1, 0, 0, 1, 1, 1, 0, 0]
    op = T.FactoredContraction(to_dev(x), to_dev(y), mask)
    op()
    torch.cuda.synchronize()
    assert int(op.status.item()) == 0
    assert op.free_pos == [1, 2, 6, 7]
    runs = op.runs()
    assert runs[0] is not None and runs[1] is None and runs[3] is None and runs[4] is None
    # E_L = the left environment of mode 0
    tm, lg = runs[0]
    el = np.ldexp(tm.cpu().numpy().astype(np.float64), lg.cpu().numpy()[:, None])
    want = O.left_envs(x64[:1], y64[:1])[-1].reshape(1, -1)
    scale = np.sqrt(np.outer(np.diag(O.left_envs(x64[:1], x64[:1])[-1]),
                             np.diag(O.left_envs(y64[:1], y64[:1])[-1]))).reshape(1, -1)
    assert np.max(np.abs(el - want) / scale) <= 1e-5
    tm, lg = runs[2]
    assert tuple(tm.shape) == (4096, 4096)
    lgh = lg.cpu().numpy()
    rows = [0, 1, 63, 64, 2080, 4095]
    for r in rows:
        a, b = divmod(r, 64)
        e = np.zeros((64, 64))
        e[a, b] = 1.0
        ex = np.zeros((64, 64))
        ex[a, a] = 1.0
        ey = np.zeros((64, 64))
        ey[b, b] = 1.0
        for k in (3, 4, 5):
            e = O.absorb_left(e, x64[k], y64[k])
            ex = O.absorb_left(ex, x64[k], x64[k])
            ey = O.absorb_left(ey, y64[k], y64[k])
        got = np.ldexp(tm[r].cpu().numpy().astype(np.float64), int(lgh[r]))
        sc = np.sqrt(np.outer(np.abs(np.diag(ex)), np.abs(np.diag(ey)))).ravel()
        err = np.max(np.abs(got - e.ravel()) / sc)
        print(f"rank64 transfer row {r}: err {err:.2e}")
        assert err <= 1e-5


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_factored_gemm_path_ragged(dtype):
    """Interior runs of 256 and more pair rows take the GEMM path (cuBLAS,
    float64 / float32 arithmetic, rows renormalised per mode); ragged ranks
    and a run of three modes, against the oracle at the dtype's tolerance."""
    rng = np.random.default_rng(21)
    modes = [3, 5, 4, 6, 3, 2]
    x = G.random_tt(rng, modes, [1, 8, 17, 20, 12, 9, 1], dtype)
    y = G.random_tt(rng, modes, [1, 9, 16, 13, 24, 5, 1], dtype)
    x64 = [c.astype(np.float64) for c in x]
    y64 = [c.astype(np.float64) for c in y]
    for mask in ([0, 1, 1, 1, 0, 0], [1, 0, 1, 0, 1, 0], [0, 0, 1, 1, 0, 1]):
        free, runs = _gpu_runs(x, y, mask)
        _, want = O.partial_factored(x64, y64, mask)
        for t, (g, w) in enumerate(zip(runs, want)):
            assert (g is None) == (w is None)
            if g is None:
                continue
            err = np.max(np.abs(g - w) / _run_scale(x64, y64, t, free, 6))
            print(f"gemm path {''.join(map(str, mask))} run {t} {g.shape}: err {err:.2e}")
            assert err <= TOL[dtype]


def test_random_sets_batch_sampled():
    """Pairs of the random-contracted-set batch (order U{4..12}, modes
    U{2..32}, ranks U{4..16}, S a random set of floor(N/2) modes at any
    positions, as timed by the benchmark): every run against the oracle."""
    for p in range(0, 512, 64):
        mask, x, y = G.random_sets_pair(p)
        n = len(x)
        free, runs = _gpu_runs(x, y, mask)
        x64 = [c.astype(np.float64) for c in x]
        y64 = [c.astype(np.float64) for c in y]
        want_free, want = O.partial_factored(x64, y64, mask)
        assert free == want_free
        for t, (g, w) in enumerate(zip(runs, want)):
            assert (g is None) == (w is None)
            if g is None:
                continue
            err = np.max(np.abs(g - w) / _run_scale(x64, y64, t, free, n))
            assert err <= 1e-5, (p, t, err)
