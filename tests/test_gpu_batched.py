"""GPU parity of the batched persistent contraction (one launch over many
uneven pairs) against the float64 oracle, against the single-pair calls, and
between a captured CUDA graph and eager launches."""
import os

import numpy as np
import pytest

import oracle as O
from helpers import cs_bound, norm_scale, to_dev, to_host
from paper_2109_00626_gb300 import inputs as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2109_00626_gb300 as T  # noqa: E402


def _uneven_pairs(n, seed, rmax=48, nmax=6, dtype=np.float32):
    """Uneven batch in the shape of the 4096-pair workload, scaled down so the
    oracle finishes quickly: order U{1..nmax}, modes U{1..20}, ranks U{1..rmax}."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(n):
        order = int(rng.integers(1, nmax + 1))
        modes = [int(v) for v in rng.integers(1, 21, size=order)]
        rx = [1] + [int(v) for v in rng.integers(1, rmax + 1, size=order - 1)] + [1]
        ry = [1] + [int(v) for v in rng.integers(1, rmax + 1, size=order - 1)] + [1]
        x = G.random_tt(rng, modes, rx, dtype)
        y = G.random_tt(rng, modes, ry, dtype)
        mask = None
        if p % 2 == 1 and order >= 2:
            s = int(rng.integers(0, order))
            lead = bool(rng.integers(0, 2))
            mask = [0] * order
            for k in range(s):
                mask[k if lead else order - 1 - k] = 1
        out.append((x, y, mask))
    return out


def _check(pairs, bat, tol):
    for p, (x, y, mask) in enumerate(pairs):
        if mask is None:
            want = O.contract_full(x, y)
            got = float(bat.out[p].item())
            assert abs(got - want) <= tol * norm_scale(x, y), (p, got, want)
        else:
            want, perm = O.partial_chain(x, y, mask)
            got = to_host(bat.z[p])
            assert perm == bat.perm[p]
            side, s = O.end_block(mask)
            m = len(x) - s
            for q, (g, w) in enumerate(zip(got, want)):
                if q == m - 1:
                    kb = cs_bound(x, y, side, s).max() if s > 0 else 1.0
                    gxb = x[s] if side == "lead" else x[m - 1]
                    scale = np.abs(gxb).max() * kb * np.sqrt(gxb.shape[0] if side == "lead" else gxb.shape[2])
                    assert np.abs(g - w).max() <= tol * scale, (p, q)
                else:
                    np.testing.assert_array_equal(g, w)


def test_batched_uneven_fp32():
    pairs = _uneven_pairs(48, 1)
    dev = [(to_dev(x), to_dev(y), m) for x, y, m in pairs]
    bat = T.BatchedContraction(dev)
    bat()
    torch.cuda.synchronize()
    assert int(bat.status.item()) == 0
    _check(pairs, bat, 1e-5)


def test_batched_high_rank_fp32():
    """Pairs that need the 128-rank tile."""
    pairs = _uneven_pairs(6, 2, rmax=128, nmax=3)
    dev = [(to_dev(x), to_dev(y), m) for x, y, m in pairs]
    bat = T.BatchedContraction(dev)
    assert max(bat.tiles()) == 2
    bat()
    torch.cuda.synchronize()
    assert int(bat.status.item()) == 0
    _check(pairs, bat, 1e-5)


def test_batched_fp64():
    pairs = _uneven_pairs(24, 3, rmax=40, dtype=np.float64)
    dev = [(to_dev(x), to_dev(y), m) for x, y, m in pairs]
    bat = T.BatchedContraction(dev)
    bat()
    torch.cuda.synchronize()
    assert int(bat.status.item()) == 0
    _check(pairs, bat, 1e-12)


def test_batched_matches_single_calls_and_graph_replay():
    pairs = _uneven_pairs(32, 4)
    dev = [(to_dev(x), to_dev(y), m) for x, y, m in pairs]
    bat = T.BatchedContraction(dev)
    bat()
    torch.cuda.synchronize()
    eager = bat.out.clone()
    eager_z = [None if z is None else [c.clone() for c in z] for z in bat.z]
    for p, (x, y, m) in enumerate(dev):
        if m is None:
            one = T.FullContraction(x, y)
            one()
            torch.cuda.synchronize()
            a, b = float(one.out.item()), float(eager[p].item())
            assert abs(a - b) <= 1e-5 * norm_scale(pairs[p][0], pairs[p][1])
    g = bat.graph()
    bat.out.zero_()
    for z in bat.z:
        if z is not None:
            for c in z:
                c.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(bat.out, eager)
    for z, ez in zip(bat.z, eager_z):
        if z is not None:
            for c, e in zip(z, ez):
                assert torch.equal(c, e)


def _engine_pairs(dtype, rmax):
    """Shapes that reach every branch of the batched kernel's planner: mode
    sizes above one panel of the float64 last mode, ragged ranks up to the
    cap, both evaluation orders (asymmetric ranks), right-to-left sweeps
    (trailing blocks), an empty contracted set, order-1 pairs."""
    r = lambda v: min(v, rmax)
    shapes = [
        ([70, 3, 45], [1, r(128), 5, 1], [1, 7, r(128), 1], None),
        ([9, 33, 2, 17], [1, r(100), r(127), 3, 1], [1, 4, r(99), r(128), 1], [0, 0, 1, 1]),
        ([5, 6, 7, 8, 9], [1, 3, r(90), 2, r(77), 1], [1, r(64), 1, r(80), 5, 1], [1, 1, 1, 0, 0]),
        ([31, 2, 29], [1, r(65), r(66), 1], [1, r(67), r(68), 1], [0, 0, 0]),
        ([37], [1, 1], [1, 1], None),
        ([4, 130], [1, r(128), 1], [1, r(97), 1], None),
        ([11, 12, 13], [1, 1, 1, 1], [1, r(128), r(128), 1], [1, 0, 0]),
        ([16, 16, 16, 16], [1, r(120), 9, r(121), 1], [1, 2, r(122), 3, 1], [0, 1, 1, 1]),
    ]
    rng = np.random.default_rng(7)
    out = []
    for modes, rx, ry, mask in shapes:
        x = G.random_tt(rng, modes, rx, dtype)
        y = G.random_tt(rng, modes, ry, dtype)
        out.append((x, y, mask))
    return out


@pytest.mark.parametrize("dtype,rmax,tol", [(np.float32, 128, 1e-5), (np.float64, 64, 1e-12)])
def test_batched_engine_shapes(dtype, rmax, tol):
    pairs = _engine_pairs(dtype, rmax)
    dev = [(to_dev(x), to_dev(y), m) for x, y, m in pairs]
    bat = T.BatchedContraction(dev)
    bat()
    torch.cuda.synchronize()
    assert int(bat.status.item()) == 0
    _check(pairs, bat, tol)


def test_batched_rescaling_split_output():
    """Cores scaled by 2^24 each: the float32 environment leaves the float
    range after a few modes unless it is renormalised; the split output
    (mantissa, exponent) must match the float64 oracle."""
    rng = np.random.default_rng(11)
    pairs = []
    for n in (5, 7, 9):
        modes = [int(v) for v in rng.integers(2, 20, size=n)]
        rx = [1] + [int(v) for v in rng.integers(4, 100, size=n - 1)] + [1]
        ry = [1] + [int(v) for v in rng.integers(4, 100, size=n - 1)] + [1]
        x = [c * np.float32(2.0**24) for c in G.random_tt(rng, modes, rx, np.float32)]
        y = [c * np.float32(2.0**24) for c in G.random_tt(rng, modes, ry, np.float32)]
        pairs.append((x, y, None))
    dev = [(to_dev(x), to_dev(y), m) for x, y, m in pairs]
    bat = T.BatchedContraction(dev, split=True)
    bat()
    torch.cuda.synchronize()
    assert int(bat.status.item()) == 0
    for p, (x, y, _) in enumerate(pairs):
        n = len(x)
        xs = [c.astype(np.float64) / 2.0**24 for c in x]
        ys = [c.astype(np.float64) / 2.0**24 for c in y]
        want = O.contract_full(xs, ys)  # z / 2^(48 n)
        m, e = float(bat.out[p].item()), int(bat.log2[p].item())
        got = np.ldexp(m, e - 48 * n)
        assert abs(got - want) <= 1e-5 * norm_scale(xs, ys), (p, got, want)


def test_batched_lpt_and_generator_shapes():
    """A slice of the 4096-pair workload itself (shapes from its generator)."""
    specs = G.batch4096_spec(64)
    assert sum(1 for s in specs if s["kind"] == "full") == 32
    pairs = []
    for p in (0, 1, 2, 3):
        spec, x, y = G.batch_pair(p)
        pairs.append((x, y, None if spec["kind"] == "full" else spec["mask"]))
    dev = [(to_dev(x), to_dev(y), m) for x, y, m in pairs]
    bat = T.BatchedContraction(dev)
    bat()
    torch.cuda.synchronize()
    assert int(bat.status.item()) == 0
    _check(pairs, bat, 1e-5)


def test_autotune_cache(tmp_path, monkeypatch):
    path = str(tmp_path / "tune.txt")
    monkeypatch.setenv("TTC_AUTOTUNE_CACHE", path)
    T.autotune("f32", path)
    lines = open(path).read().split("\n")
    rows = [list(map(int, ln.split())) for ln in lines if ln.strip()]
    assert len(rows) == 20  # 4 rank buckets x 5 mode-size buckets
    for d, rb, ib, cfg in rows:
        assert d == 0 and 0 <= rb < 4 and 0 <= ib < 5 and 0 <= cfg < 12
    pairs = _uneven_pairs(8, 5)
    dev = [(to_dev(x), to_dev(y), m) for x, y, m in pairs]
    bat = T.BatchedContraction(dev)
    bat()
    torch.cuda.synchronize()
    _check(pairs, bat, 1e-5)


@pytest.mark.parametrize("cfg", range(12))
def test_every_tile_configuration(tmp_path, monkeypatch, cfg):
    """Every tile configuration the autotuner can choose (panel-budget level
    and replica cap), forced on every bucket through a cache file, gives the
    oracle's results on uneven pairs of ranks up to 128."""
    path = str(tmp_path / f"cfg{cfg}.txt")
    with open(path, "w") as f:
        for rb in range(4):
            for ib in range(5):
                f.write(f"0 {rb} {ib} {cfg}\n")
    monkeypatch.setenv("TTC_AUTOTUNE_CACHE", path)
    pairs = _uneven_pairs(12, 40 + cfg, rmax=128, nmax=5)
    dev = [(to_dev(x), to_dev(y), m) for x, y, m in pairs]
    bat = T.BatchedContraction(dev)
    assert set(bat.tiles()) == {cfg}
    bat()
    torch.cuda.synchronize()
    assert int(bat.status.item()) == 0
    _check(pairs, bat, 1e-5)


def test_batched_full_size_sampled():
    """The full 4096-pair workload in the launch configuration the benchmark
    times; sampled pairs (the cheapest full and partial ones, plus one of the
    largest) are checked against the oracle one by one."""
    from paper_2109_00626_gb300 import workload as W

    specs, pairs = G.batch4096_device(4096)
    bat = T.BatchedContraction(pairs)
    g = bat.graph()
    g.replay()
    torch.cuda.synchronize()
    assert int(bat.status.item()) == 0
    cost = []
    for s in specs:
        f = W.full_flops(s["modes"], s["ranks_x"], s["ranks_y"]) if s["kind"] == "full" else \
            W.partial_chain_flops(s["modes"], s["ranks_x"], s["ranks_y"], s["mask"])
        cost.append(f)
    full_ids = sorted([p for p in range(4096) if specs[p]["kind"] == "full"], key=lambda p: cost[p])
    part_ids = sorted([p for p in range(4096) if specs[p]["kind"] == "partial"], key=lambda p: cost[p])
    sample = full_ids[:2] + part_ids[:2] + [full_ids[len(full_ids) // 2]]
    for p in sample:
        x = [c.cpu().double().numpy() for c in pairs[p][0]]
        y = [c.cpu().double().numpy() for c in pairs[p][1]]
        mask = pairs[p][2]
        if mask is None:
            want = O.contract_full(x, y)
            got = float(bat.out[p].item())
            assert abs(got - want) <= 1e-5 * norm_scale(x, y), (p, got, want)
        else:
            want, perm = O.partial_chain(x, y, mask)
            got = to_host(bat.z[p])
            side, s = O.end_block(mask)
            m = len(x) - s
            for q, (gq, wq) in enumerate(zip(got, want)):
                if q == m - 1:
                    kb = cs_bound(x, y, side, s).max() if s > 0 else 1.0
                    gxb = x[s] if side == "lead" else x[m - 1]
                    scale = np.abs(gxb).max() * kb * np.sqrt(gxb.shape[0] if side == "lead" else gxb.shape[2])
                    assert np.abs(gq - wq).max() <= 1e-5 * scale, (p, q)
                else:
                    np.testing.assert_array_equal(gq, wq)
    del bat, pairs
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype,scale", [(np.float32, 1.0), (np.float64, 0.5)])
def test_batched_free_core_copies(dtype, scale):
    """Partial pairs whose free cores are copied plainly and transposed: slices
    of more than 4096 elements (a transposed copy cut by rows, ragged last
    cut), right ranks that are and are not a multiple of the 16-byte width,
    cores copied as one run and as runs per row.  Copies must be exact."""
    r = lambda v: max(1, int(v * scale))  # noqa: E731
    shapes = [
        ([3, 70, 41, 9], [1, r(100), r(128), r(77), 1], [1, r(5), r(64), r(33), 1], [1, 0, 0, 0]),
        ([9, 41, 70, 3], [1, r(77), r(128), r(100), 1], [1, r(33), r(64), r(5), 1], [0, 0, 0, 1]),
        ([2, 5, 300, 7, 2], [1, r(4), r(8), r(12), r(3), 1], [1, r(127), r(1), r(13), r(6), 1], [1, 1, 0, 0, 0]),
        ([6, 1, 33, 2], [1, r(128), r(128), r(128), 1], [1, r(128), r(128), r(128), 1], [0, 0, 1, 1]),
    ]
    rng = np.random.default_rng(11)
    pairs = []
    for modes, rx, ry, mask in shapes:
        pairs.append((G.random_tt(rng, modes, rx, dtype), G.random_tt(rng, modes, ry, dtype), mask))
    bat = T.BatchedContraction([(to_dev(x), to_dev(y), m) for x, y, m in pairs])
    bat()
    torch.cuda.synchronize()
    assert int(bat.status.item()) == 0
    _check(pairs, bat, 1e-5 if dtype == np.float32 else 1e-12)
