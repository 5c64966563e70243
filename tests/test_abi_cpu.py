"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every symbol include/ttc.h declares, and rejects bad arguments before it
enqueues anything (fake device pointers are never dereferenced)."""
import ctypes
import os
import re

import pytest

import paper_2109_00626_gb300 as T
from paper_2109_00626_gb300 import _binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2109_00626_gb300 import build

    build.build()
    return T.lib()


def test_header_symbols_exported(L):
    hdr = open(os.path.join(ROOT, "include", "ttc.h")).read()
    declared = set(re.findall(r"\b(tt_[a-z0-9_]+)\s*\(", hdr))
    declared -= {"tt_desc", "tt_batch"}
    assert declared == set(B.EXPORTS), declared ^ set(B.EXPORTS)
    for name in declared:
        assert hasattr(L, name), name


class FakeDesc:
    """tt_desc with non-NULL fake device pointers (host validation only)."""

    def __init__(self, modes, ranks, dtype=B.TT_F32):
        n = len(modes)
        self._modes = (ctypes.c_int32 * n)(*modes)
        self._ranks = (ctypes.c_int32 * (n + 1))(*ranks)
        self._cores = (ctypes.c_void_p * n)(*[0x1000 * (k + 1) for k in range(n)])
        self.desc = B.TTDesc(n, self._modes, self._ranks, self._cores, dtype)

    @property
    def ref(self):
        return ctypes.byref(self.desc)


def _mask(m):
    return (ctypes.c_uint8 * len(m))(*m)


def test_shape_errors(L):
    x = FakeDesc([4, 4, 4], [1, 3, 3, 1])
    y = FakeDesc([4, 5, 4], [1, 2, 2, 1])
    out = ctypes.c_void_p(0x2000)
    assert L.tt_contract_full(x.ref, y.ref, 0, out, None, None, None, 0, None) == -2
    bad = FakeDesc([4, 4], [2, 3, 1])
    assert L.tt_contract_full(bad.ref, bad.ref, 0, out, None, None, None, 0, None) == -2
    z8 = FakeDesc([4, 4, 4], [1, 3, 3, 1], dtype=B.TT_F64)
    assert L.tt_contract_full(x.ref, z8.ref, 0, out, None, None, None, 0, None) == -3
    assert L.tt_contract_full(x.ref, x.ref, 0, None, None, None, None, 0, None) == -1


def test_partial_shape_chain_and_merged(L):
    x = FakeDesc([2, 3, 4, 5], [1, 6, 7, 8, 1])
    y = FakeDesc([2, 3, 4, 5], [1, 9, 10, 11, 1])
    modes, ranks, perm = B.partial_shape(x, y, [1, 1, 0, 0], "chain")
    assert modes == [5, 4, 4, 5] and ranks == [1, 8, 10, 11, 1] and perm == [1, 0, 2, 3]
    modes, ranks, perm = B.partial_shape(x, y, [0, 0, 1, 1], "chain")
    assert modes == [2, 3, 3, 2] and ranks == [1, 6, 10, 9, 1] and perm == [0, 1, 3, 2]
    modes, ranks, perm = B.partial_shape(x, y, [0, 1, 0, 1], "merged")
    assert modes == [4, 16] and ranks == [1, 70, 1] and perm == [0, 2, 1, 3]
    with pytest.raises(B.TTError) as e:
        B.partial_shape(x, y, [0, 1, 1, 0], "chain")
    assert e.value.code == -4
    with pytest.raises(B.TTError) as e:
        B.partial_shape(x, y, [1, 1, 1, 1], "chain")
    assert e.value.code == -1


def test_partial_validation(L):
    x = FakeDesc([2, 3, 4, 5], [1, 6, 7, 8, 1])
    y = FakeDesc([2, 3, 4, 5], [1, 9, 10, 11, 1])
    zbad = FakeDesc([5, 4, 3, 5], [1, 8, 10, 11, 1])
    # the environment stays on chip: a partial contraction needs no workspace
    assert B.workspace_bytes(B.TT_OP_PARTIAL, x, y, [1, 1, 0, 0], "chain") == 0
    # wrong output shape (the third core's mode is 4, not 3)
    rc = L.tt_contract_partial(x.ref, y.ref, _mask([1, 1, 0, 0]), 0, 0, zbad.ref, None, None, None, 0, None)
    assert rc == -2
    # interior contracted block with the chain layout
    modes, ranks, _ = B.partial_shape(x, y, [1, 1, 0, 0], "chain")
    z = FakeDesc(modes, ranks)
    rc = L.tt_contract_partial(x.ref, y.ref, _mask([0, 1, 1, 0]), 0, 0, z.ref, None, None, None, 0, None)
    assert rc == -4
    # output dtype differs from the operands
    z64 = FakeDesc(modes, ranks, dtype=B.TT_F64)
    rc = L.tt_contract_partial(x.ref, y.ref, _mask([1, 1, 0, 0]), 0, 0, z64.ref, None, None, None, 0, None)
    assert rc == -2


def test_error_strings(L):
    for code in range(0, -9, -1):
        assert isinstance(T.error_string(code), str) and T.error_string(code)


def test_partial_shape_degenerate_masks(L):
    """Every mode contracted is a full contraction: the partial call refuses it
    (TT_ERR_ARG); nothing contracted is the outer product, for any order
    including 1 (the chain joins the two trains at rank 1)."""
    x = FakeDesc([2, 3, 4, 5], [1, 6, 7, 8, 1])
    y = FakeDesc([2, 3, 4, 5], [1, 9, 10, 11, 1])
    with pytest.raises(B.TTError):
        B.partial_shape(x, y, [1, 1, 1, 1], "chain")
    modes, ranks, perm = B.partial_shape(x, y, [0, 0, 0, 0], "chain")
    assert modes == [5, 4, 3, 2, 2, 3, 4, 5] and ranks[4] == 1 and sorted(perm) == list(range(8))
    x1, y1 = FakeDesc([5], [1, 1]), FakeDesc([5], [1, 1])
    assert B.partial_shape(x1, y1, [0], "chain") == ([5, 5], [1, 1, 1], [0, 1])
    with pytest.raises(B.TTError):
        B.partial_shape(x1, y1, [1], "chain")


def test_k_entry_points_reject_missing_buffers(L):
    """tt_contract_partial_k needs the backward workspace it fills, and
    tt_contract_backward_k the mask: missing ones are reported before anything
    is enqueued."""
    x = FakeDesc([2, 3, 4, 5], [1, 6, 7, 8, 1])
    y = FakeDesc([2, 3, 4, 5], [1, 9, 10, 11, 1])
    modes, ranks, _ = B.partial_shape(x, y, [1, 1, 0, 0], "chain")
    z = FakeDesc(modes, ranks)
    rc = L.tt_contract_partial_k(x.ref, y.ref, _mask([1, 1, 0, 0]), 0, z.ref, None, None, None, 0, None)
    assert rc == -6  # TT_ERR_WS
    rc = L.tt_contract_backward_k(x.ref, y.ref, None, 0, z.ref, x.ref, y.ref, None, None, 0, None)
    assert rc == -1  # TT_ERR_ARG


def _merged_ws(L, x, y, mask):
    nb = ctypes.c_size_t(0)
    rc = L.tt_workspace_bytes(B.TT_OP_PARTIAL, x.ref, y.ref, _mask(mask), B.LAYOUT["merged"], B.PREC["native"],
                              ctypes.byref(nb))
    return rc, nb.value


def test_merged_workspace_and_caps(L):
    # order 3, S = {1}: the first core has an interior run after it.  Slots
    # (1 + 4 per core), E_L, V, W_0 (I J R^x'R^y' = 24), then for core 0 its
    # transfer matrix (6 x 6) and 6 row scales; core 1 needs nothing: six
    # 256-byte blocks.
    x = FakeDesc([2, 2, 2], [1, 2, 3, 1])
    y = FakeDesc([2, 2, 2], [1, 3, 2, 1])
    assert _merged_ws(L, x, y, [0, 1, 0]) == (0, 6 * 256)
    # no contracted run after any free core: slots, E_L, V only
    assert _merged_ws(L, x, y, [1, 0, 0]) == (0, 3 * 256)
    # an interior run after a later core needs P (R^x I R^y' x the next pair rank)
    x4 = FakeDesc([8] * 6, [1] + [16] * 5 + [1])
    rc, nb = _merged_ws(L, x4, x4, [0, 0, 1, 0, 0, 0])
    assert rc == 0 and nb >= 4 * (16 * 8 * 16 * 256 + 256 * 256) + 8 * 256
    # caps: a merged core over 2^30 entries; a rank above the float64 cap
    big = FakeDesc([3, 3, 3, 3], [1, 128, 128, 128, 1])  # core 1: 128^2 * 9 rows x 128^2 > 2^30
    assert _merged_ws(L, big, big, [0, 1, 0, 0])[0] == -5
    assert _merged_ws(L, big, big, [1, 1, 0, 1])[0] == 0
    d65 = FakeDesc([2, 2, 2], [1, 65, 65, 1], dtype=B.TT_F64)
    assert _merged_ws(L, d65, d65, [0, 1, 0])[0] == -5


def test_merged_rejects_before_enqueue(L):
    """The merged layout checks its output cores and workspace before it touches
    a stream: wrong core count, wrong core shape or dtype, short workspace."""
    x = FakeDesc([3, 2, 4, 2], [1, 2, 5, 3, 1])
    y = FakeDesc([3, 2, 4, 2], [1, 3, 1, 4, 1])
    mask = [0, 1, 0, 1]
    modes, ranks, _ = B.partial_shape(x, y, mask, "merged")
    rc, nb = _merged_ws(L, x, y, mask)
    assert rc == 0 and nb > 0
    ws = ctypes.c_void_p(0x100000)
    z = FakeDesc(modes, ranks)
    assert L.tt_contract_partial(x.ref, y.ref, _mask(mask), 1, 0, z.ref, None, None, ws, nb - 1, None) == -6
    assert L.tt_contract_partial(x.ref, y.ref, _mask(mask), 1, 0, z.ref, None, None, None, nb, None) == -6
    z_short = FakeDesc(modes[:1], ranks[:1] + [1])
    assert L.tt_contract_partial(x.ref, y.ref, _mask(mask), 1, 0, z_short.ref, None, None, ws, nb, None) == -2
    bad = list(ranks)
    bad[1] += 1
    z_bad = FakeDesc(modes, bad)
    assert L.tt_contract_partial(x.ref, y.ref, _mask(mask), 1, 0, z_bad.ref, None, None, ws, nb, None) == -2
    z64 = FakeDesc(modes, ranks, dtype=B.TT_F64)
    assert L.tt_contract_partial(x.ref, y.ref, _mask(mask), 1, 0, z64.ref, None, None, ws, nb, None) == -2


def _batch(xs, ys, masks, zs, prec=0):
    """A tt_batch over FakeDescs; returns it with the arrays it points into."""
    n = len(xs)
    xarr = (B.TTDesc * n)(*[d.desc for d in xs])
    yarr = (B.TTDesc * n)(*[d.desc for d in ys])
    bufs = [(_mask(m) if m is not None else None) for m in masks]
    mp = (ctypes.POINTER(ctypes.c_uint8) * n)(
        *[(ctypes.cast(b, ctypes.POINTER(ctypes.c_uint8)) if b is not None else ctypes.POINTER(ctypes.c_uint8)())
          for b in bufs])
    zarr = None
    if zs is not None:
        zarr = (B.TTDesc * n)(*[(z.desc if z is not None else xs[0].desc) for z in zs])
    batch = B.TTBatch(n, xarr, yarr, mp, zarr, prec)
    return batch, (xarr, yarr, mp, zarr, bufs)


def _plan(L, batch):
    plan = ctypes.c_void_p()
    pb = ctypes.c_size_t(0)
    wb = ctypes.c_size_t(0)
    rc = L.tt_batch_plan(ctypes.byref(batch), ctypes.byref(plan), ctypes.byref(pb), ctypes.byref(wb))
    return rc, plan, pb.value, wb.value


def test_batch_plan_on_the_host(L):
    """tt_batch_plan / tt_batch_pack / tt_plan_info are host-only: a mix of full
    and partial pairs plans, packs into exactly packed_bytes, reports a tile
    configuration per pair; bad pairs are rejected with their codes."""
    specs = [([4, 3, 5], [1, 4, 6, 1], [1, 5, 3, 1], None),
             ([2, 3, 4, 5], [1, 6, 7, 8, 1], [1, 9, 10, 11, 1], [1, 1, 0, 0]),
             ([3, 3, 3, 3, 3], [1, 16, 16, 16, 16, 1], [1, 16, 16, 16, 16, 1], None),
             ([2, 3, 4, 5], [1, 6, 7, 8, 1], [1, 9, 10, 11, 1], [0, 0, 1, 1])]
    xs, ys, masks, zs = [], [], [], []
    for modes, rx, ry, mask in specs:
        x, y = FakeDesc(modes, rx), FakeDesc(modes, ry)
        xs.append(x)
        ys.append(y)
        masks.append(mask)
        if mask is None:
            zs.append(None)
        else:
            zm, zr, _ = B.partial_shape(x, y, mask, "chain")
            zs.append(FakeDesc(zm, zr))
    batch, keep = _batch(xs, ys, masks, zs)
    rc, plan, pb, wb = _plan(L, batch)
    assert rc == 0 and pb > 0 and wb == 256
    try:
        n = ctypes.c_int32(0)
        t = ctypes.c_int32(-1)
        for p in range(len(specs)):
            assert L.tt_plan_info(plan, p, ctypes.byref(n), ctypes.byref(t)) == 0
            assert n.value == len(specs) and t.value == 2  # no tuning cache: full budget, no replica cap
        assert L.tt_plan_info(plan, len(specs), None, ctypes.byref(t)) == -1
        buf = (ctypes.c_uint8 * pb)()
        assert L.tt_batch_pack(plan, buf, pb) == 0
        assert L.tt_batch_pack(plan, buf, pb - 1) == -1
    finally:
        L.tt_plan_free(plan)
    # the partial pairs' free-core copies are packed as jobs: more partial pairs, more bytes
    batch1, keep1 = _batch(xs[:1], ys[:1], masks[:1], zs[:1])
    batch2, keep2 = _batch(xs[:2], ys[:2], masks[:2], zs[:2])
    rc1, p1, pb1, _ = _plan(L, batch1)
    rc2, p2, pb2, _ = _plan(L, batch2)
    assert rc1 == 0 and rc2 == 0 and pb2 > pb1
    L.tt_plan_free(p1)
    L.tt_plan_free(p2)

    def rejects(code, xs_, ys_, masks_, zs_, prec=0):
        b, k = _batch(xs_, ys_, masks_, zs_, prec)
        rc, plan, _, _ = _plan(L, b)
        assert rc == code, (rc, code)
        assert not plan.value  # nothing to free on an error

    x4, y4 = FakeDesc([2, 3, 4, 5], [1, 6, 7, 8, 1]), FakeDesc([2, 3, 4, 5], [1, 9, 10, 11, 1])
    rejects(-4, [x4], [y4], [[0, 1, 1, 0]], [x4])                       # not an end block
    rejects(-1, [x4], [y4], [[1, 1, 0, 0]], None)                       # partial pair, no outputs
    zm, zr, _ = B.partial_shape(x4, y4, [1, 1, 0, 0], "chain")
    zr_bad = list(zr)
    zr_bad[1] += 1
    rejects(-2, [x4], [y4], [[1, 1, 0, 0]], [FakeDesc(zm, zr_bad)])     # output of the wrong shape
    x8 = FakeDesc([4, 3, 5], [1, 4, 6, 1], dtype=B.TT_F64)
    y8 = FakeDesc([4, 3, 5], [1, 5, 3, 1], dtype=B.TT_F64)
    rejects(-3, [xs[0], x8], [ys[0], y8], [None, None], [None, None])   # mixed dtypes
    xb = FakeDesc([4, 3, 5], [1, 4, 6, 1], dtype=B.TT_BF16)
    yb = FakeDesc([4, 3, 5], [1, 5, 3, 1], dtype=B.TT_BF16)
    rejects(-8, [xb], [yb], [None], [None])                              # bfloat16 pairs
    rejects(-8, [xs[0]], [ys[0]], [None], [None], prec=B.PREC["bf16"])  # reduced-precision products
    big = FakeDesc([2, 2, 2], [1, 129, 129, 1])
    rejects(-5, [big], [big], [None], [None])                            # rank above the float32 cap


def test_batched_entries_reject_missing_buffers(L):
    """tt_contract_batched and tt_contract_batched_noalloc return TT_ERR_ARG
    for a NULL plan, packed table or output before any CUDA call, and the
    no-alloc entry plans within the fixed array the header states."""
    hdr = open(os.path.join(ROOT, "include", "ttc.h")).read()
    limit = int(re.search(r"#define TT_NOALLOC_SCRATCH_BYTES (\d+)", hdr).group(1))
    x, y = FakeDesc([4, 3, 5], [1, 4, 6, 1]), FakeDesc([4, 3, 5], [1, 5, 3, 1])
    batch, keep = _batch([x], [y], [None], [None])
    rc, plan, pb, wb = _plan(L, batch)
    assert rc == 0 and 0 < wb <= limit
    try:
        packed, out, st = ctypes.c_void_p(0x3000), ctypes.c_void_p(0x4000), ctypes.c_void_p(0x5000)
        ws = ctypes.c_void_p(0x6000)
        for args in ((None, packed, out), (plan, None, out), (plan, packed, None)):
            assert L.tt_contract_batched_noalloc(*args, None, st, None) == -1
            assert L.tt_contract_batched(*args, None, st, ws, wb, None) == -1
        assert L.tt_contract_batched(plan, packed, out, None, st, None, wb, None) == -6  # no workspace
        assert L.tt_contract_batched(plan, packed, out, None, st, ws, wb - 1, None) == -6  # too small
    finally:
        L.tt_plan_free(plan)


def _pairs_shape(L, x, y, pairs):
    n = x.desc.order + y.desc.order
    xm = (ctypes.c_int32 * len(pairs))(*[a for a, _ in pairs])
    ym = (ctypes.c_int32 * len(pairs))(*[b for _, b in pairs])
    order = ctypes.c_int32(0)
    modes = (ctypes.c_int32 * n)()
    ranks = (ctypes.c_int32 * (n + 1))()
    perm = (ctypes.c_int32 * n)()
    rc = L.tt_pairs_shape(x.ref, y.ref, len(pairs), xm, ym, ctypes.byref(order), modes, ranks, perm)
    o = order.value
    return rc, list(modes[:o]), list(ranks[: o + 1]), list(perm[:o])


def test_pairs_shape_on_the_host(L):
    """tt_pairs_shape: the chain's mode sizes are X's free modes walked back,
    then Y's (Y's walked back when X has none), perm a permutation of Eq. 8's
    axes consistent with the sizes; the oracle's layout where X has free
    modes; rejections before anything is enqueued."""
    import numpy as np

    import oracle as O
    from paper_2109_00626_gb300 import inputs as G

    cases = [([2, 3, 4, 5], [4, 6, 7], [(2, 0)]),   # not an end block of X
             ([2, 3, 4, 5], [5, 6, 7], [(3, 0)]),
             ([2, 3, 4, 5], [6, 5, 4], [(3, 1), (2, 2)]),
             ([3, 4], [3, 4, 5, 6], [(0, 0), (1, 1)]),
             ([5, 4, 3], [3, 4], [(2, 0), (1, 1)])]
    for mx, my, pairs in cases:
        rng = np.random.default_rng(1)
        rx = [1] + [3] * (len(mx) - 1) + [1]
        ry = [1] + [2] * (len(my) - 1) + [1]
        x, y = FakeDesc(mx, rx), FakeDesc(my, ry)
        rc, modes, ranks, perm = _pairs_shape(L, x, y, pairs)
        try:
            oc, operm = O.partial_chain_pairs(G.random_tt(rng, mx, rx, np.float64),
                                              G.random_tt(rng, my, ry, np.float64), pairs)
        except ValueError:
            assert rc == -4, (pairs, rc)  # TT_ERR_LAYOUT
            continue
        assert rc == 0
        fx = [m for k, m in enumerate(mx) if k not in {a for a, _ in pairs}]
        fy = [m for k, m in enumerate(my) if k not in {b for _, b in pairs}]
        eq8 = fx + fy
        assert sorted(perm) == list(range(len(eq8)))
        assert [eq8[pm] for pm in perm] == modes
        assert ranks[0] == 1 and ranks[-1] == 1
        if len(fx) > 0:
            assert modes == [c.shape[1] for c in oc] and perm == operm
            assert ranks[:-1] == [c.shape[0] for c in oc]
    x, y = FakeDesc([2, 3], [1, 2, 1]), FakeDesc([3, 2], [1, 2, 1])
    assert _pairs_shape(L, x, y, [(0, 1), (1, 0)])[0] == -1   # every mode of both: a full contraction
    assert _pairs_shape(L, x, y, [(1, 0), (1, 1)])[0] == -1   # a mode paired twice
    assert _pairs_shape(L, x, FakeDesc([4, 2], [1, 2, 1]), [(1, 0)])[0] == -2  # sizes differ


def test_selftest_wait_arguments(L):
    """The bounded-wait self-test rejects a NULL status and a limit outside
    0 .. 10^9 cycles before launching anything."""
    st = ctypes.c_void_p(0x3000)
    assert L.tt_selftest_wait(0, 1000, None, None) == -1
    assert L.tt_selftest_wait(0, -1, st, None) == -1
    assert L.tt_selftest_wait(0, 10**9 + 1, st, None) == -1


def test_tf32_forms_rejections(L):
    """The tf32 forms take float32 cores with every rank <= 64; the checks
    come back before anything is enqueued."""
    out = ctypes.c_void_p(0x2000)
    st = ctypes.c_void_p(0x3000)
    ok = FakeDesc([4, 4, 4], [1, 64, 8, 1])
    big = FakeDesc([4, 4, 4], [1, 65, 8, 1])
    f64 = FakeDesc([4, 4, 4], [1, 8, 8, 1], dtype=B.TT_F64)
    for prec in ("tf32", "tf32x3"):
        pr = B.PREC[prec]
        assert L.tt_contract_full(big.ref, ok.ref, pr, out, None, st, None, 0, None) == -8
        assert L.tt_contract_full(f64.ref, f64.ref, pr, out, None, st, None, 0, None) == -3
        zm, zr, _ = B.partial_shape(big, ok, [1, 0, 0], "chain")
        z = FakeDesc(zm, zr)
        assert L.tt_contract_partial(big.ref, ok.ref, _mask([1, 0, 0]), 0, pr, z.ref, None, st, None, 0, None) == -8
        # the merged layout has no tf32 form
        assert L.tt_contract_partial(ok.ref, ok.ref, _mask([0, 1, 0]), 1, pr, z.ref, None, st, None, 0, None) == -8
        # workspace query of a full contraction in a tf32 form: the two meeting environments
        rc, nb = _ws(L, B.TT_OP_FULL, ok, ok, prec=prec)
        assert rc == 0 and nb > 0
    assert L.tt_contract_full(ok.ref, ok.ref, 7, out, None, st, None, 0, None) == -8  # unknown form


def _ws(L, op, x, y, mask=None, layout="chain", prec="native"):
    nb = ctypes.c_size_t(0)
    m = _mask(mask) if mask is not None else None
    rc = L.tt_workspace_bytes(op, x.ref, y.ref, m, B.LAYOUT[layout], B.PREC[prec], ctypes.byref(nb))
    return rc, nb.value


def test_svd_workspace_and_rejections(L):
    """tt_svd_workspace: the largest ranks a TT-SVD can return (the shorter
    side of each unfolding, capped by max_rank) for Example 2's shapes and
    the limits; tt_svd and tt_dense_permute reject bad arguments before they
    enqueue (fake device pointers, never dereferenced)."""
    assert T.svd_workspace([20, 20, 20], B.TT_F64)[0] == [1, 20, 20, 1]
    assert T.svd_workspace([20, 20, 20, 5], B.TT_F32)[0] == [1, 20, 100, 5, 1]
    assert T.svd_workspace([20, 20, 20, 5, 4], B.TT_F32)[0] == [1, 20, 400, 20, 4, 1]
    assert T.svd_workspace([20, 20, 20, 5, 4], B.TT_F32, max_rank=8)[0] == [1, 8, 8, 8, 4, 1]
    assert T.svd_workspace([7], B.TT_F64)[0] == [1, 1]
    cap, ws = T.svd_workspace([3, 5, 2], B.TT_F64)
    assert cap == [1, 3, 2, 1]
    # two copies of the tensor, the 3 x 3 rotations, singular values and order
    assert ws == 2 * 256 + 256 + 256 + 256
    cap = (ctypes.c_int32 * 8)()
    ws = ctypes.c_size_t(0)
    md = (ctypes.c_int32 * 2)(600, 600)
    assert L.tt_svd_workspace(2, md, B.TT_F32, 0, cap, ctypes.byref(ws)) == -5   # 600 x 600 unfolding
    assert L.tt_svd_workspace(2, md, B.TT_F32, 100, cap, ctypes.byref(ws)) == -5  # the cap does not shrink the SVD
    assert L.tt_svd_workspace(2, md, B.TT_BF16, 0, cap, ctypes.byref(ws)) == -3
    md0 = (ctypes.c_int32 * 2)(4, 0)
    assert L.tt_svd_workspace(2, md0, B.TT_F32, 0, cap, ctypes.byref(ws)) == -2
    assert L.tt_svd_workspace(0, md0, B.TT_F32, 0, cap, ctypes.byref(ws)) == -1
    md = (ctypes.c_int32 * 3)(4, 5, 6)
    cores = (ctypes.c_void_p * 3)(0x1000, 0x2000, 0x3000)
    fake = ctypes.c_void_p(0x4000)
    need = T.svd_workspace([4, 5, 6], B.TT_F32)[1]
    assert L.tt_svd(None, 3, md, B.TT_F32, 1e-3, 0, cores, fake, fake, fake, need, None) == -1
    assert L.tt_svd(fake, 3, md, B.TT_F32, -1.0, 0, cores, fake, fake, fake, need, None) == -1
    assert L.tt_svd(fake, 3, md, B.TT_F32, float("nan"), 0, cores, fake, fake, fake, need, None) == -1
    assert L.tt_svd(fake, 3, md, B.TT_F32, 1e-3, 0, cores, fake, fake, fake, need - 1, None) == -6
    nul = (ctypes.c_void_p * 3)(0x1000, None, 0x3000)
    assert L.tt_svd(fake, 3, md, B.TT_F32, 1e-3, 0, nul, fake, fake, fake, need, None) == -1
    ax = (ctypes.c_int32 * 3)(2, 0, 2)
    assert L.tt_dense_permute(fake, 3, md, ax, B.TT_F32, ctypes.c_void_p(0x5000), None) == -1
    ax = (ctypes.c_int32 * 3)(2, 0, 3)
    assert L.tt_dense_permute(fake, 3, md, ax, B.TT_F32, ctypes.c_void_p(0x5000), None) == -1
    ax = (ctypes.c_int32 * 3)(2, 0, 1)
    assert L.tt_dense_permute(fake, 3, md, ax, B.TT_F32, fake, None) == -1  # in place
    assert L.tt_dense_permute(fake, 3, md, ax, B.TT_BF16, ctypes.c_void_p(0x5000), None) == -3


def test_factored_shape_on_the_host(L):
    """tt_factored_shape: free positions, run shapes over pair indices (an
    empty run is 0 x 0), arena offsets; rejections before anything is
    enqueued."""
    x = FakeDesc([3, 4, 5, 4, 3], [1, 2, 3, 4, 2, 1])
    y = FakeDesc([3, 4, 5, 4, 3], [1, 3, 2, 2, 3, 1])
    f = B.TTFactored()
    assert L.tt_factored_shape(x.ref, y.ref, _mask([1, 0, 1, 1, 0]), ctypes.byref(f)) == 0
    assert f.n_free == 2 and list(f.free_pos[:2]) == [1, 4]
    # T_0: 1 x (2*3); T_1: modes 2..3, (3*2) x (2*3); T_2: none (mode 4 is free and last)
    assert (f.rows[0], f.cols[0]) == (1, 6)
    assert (f.rows[1], f.cols[1]) == (6, 6)
    assert (f.rows[2], f.cols[2]) == (0, 0)
    assert f.off_t[0] == 0 and f.off_log2[0] == 256 and f.off_t[1] == 512 and f.off_log2[1] == 768
    assert f.bytes == 1024
    assert L.tt_factored_shape(x.ref, y.ref, _mask([0, 1, 1, 1, 1]), ctypes.byref(f)) == 0
    assert (f.rows[0], f.rows[1], f.cols[1]) == (0, 2 * 3, 1)
    assert L.tt_factored_shape(x.ref, y.ref, _mask([1, 1, 1, 1, 1]), ctypes.byref(f)) == -1
    y_bad = FakeDesc([3, 4, 6, 4, 3], [1, 3, 2, 2, 3, 1])
    assert L.tt_factored_shape(x.ref, y_bad.ref, _mask([1, 0, 1, 1, 0]), ctypes.byref(f)) == -2
    big = FakeDesc([3, 4, 5, 4, 3], [1, 200, 3, 4, 2, 1])
    assert L.tt_factored_shape(big.ref, y.ref, _mask([1, 0, 1, 1, 0]), ctypes.byref(f)) == -5
    # the contraction checks its shape against the operands and S
    assert L.tt_factored_shape(x.ref, y.ref, _mask([1, 0, 1, 1, 0]), ctypes.byref(f)) == 0
    out = ctypes.c_void_p(0x10000)
    st = ctypes.c_void_p(0x20000)
    assert f.ws_bytes == 0  # runs of fewer than 256 pair rows need no workspace
    assert L.tt_contract_factored(x.ref, y.ref, _mask([1, 1, 0, 1, 0]), ctypes.byref(f), out, st, None, 0, None) == -2
    assert L.tt_contract_factored(x.ref, y.ref, _mask([1, 0, 1, 1, 0]), ctypes.byref(f), None, st, None, 0, None) == -1
    # a rank-64 interior run goes through the GEMM path and needs its workspace
    x64 = FakeDesc([16] * 5, [1, 64, 64, 64, 64, 1])
    assert L.tt_factored_shape(x64.ref, x64.ref, _mask([0, 1, 1, 0, 0]), ctypes.byref(f)) == 0
    assert (f.rows[1], f.cols[1]) == (4096, 4096)
    # two environment buffers of 4096 x 4096 floats and a chunk of 2^26 floats of the intermediate
    assert f.ws_bytes == 2 * 4096 * 4096 * 4 + (1 << 26) * 4
    assert L.tt_contract_factored(x64.ref, x64.ref, _mask([0, 1, 1, 0, 0]), ctypes.byref(f), out, st, None, 0,
                                  None) == -6


def test_round_workspace_and_rejections(L):
    """tt_round_workspace and tt_round's argument checks (host only)."""
    x = FakeDesc([4, 3, 5], [1, 3, 4, 1])
    ws = ctypes.c_size_t(0)
    assert L.tt_round_workspace(x.ref, 0, ctypes.byref(ws)) == 0 and ws.value > 0
    assert L.tt_round_workspace(x.ref, -1, ctypes.byref(ws)) == -1
    xb = FakeDesc([4, 3, 5], [1, 3, 4, 1], dtype=B.TT_BF16)
    assert L.tt_round_workspace(xb.ref, 0, ctypes.byref(ws)) == -3
    big = FakeDesc([4, 600, 4], [1, 600, 600, 1])
    assert L.tt_round_workspace(big.ref, 0, ctypes.byref(ws)) == -5
    L.tt_round_workspace(x.ref, 0, ctypes.byref(ws))
    outs = (ctypes.c_void_p * 3)(0x1000, 0x2000, 0x3000)
    fake = ctypes.c_void_p(0x4000)
    assert L.tt_round(x.ref, 0.1, 0, outs, fake, fake, fake, ws.value - 1, None) == -6
    assert L.tt_round(x.ref, -0.1, 0, outs, fake, fake, fake, ws.value, None) == -1
    assert L.tt_round(x.ref, 0.1, 0, outs, None, fake, fake, ws.value, None) == -1
    nul = (ctypes.c_void_p * 3)(0x1000, None, 0x3000)
    assert L.tt_round(x.ref, 0.1, 0, nul, fake, fake, fake, ws.value, None) == -1


def test_workspace_queries_and_their_limits(L):
    """tt_workspace_bytes per operation, and the conditions the header states
    for each path (host only)."""
    x = FakeDesc([16] * 10, [1] + [64] * 9 + [1])
    rc, nb = _ws(L, B.TT_OP_FULL, x, x)
    assert rc == 0 and nb > 0                        # the two-sided sweep's meeting environments
    one = FakeDesc([5], [1, 1])
    assert _ws(L, B.TT_OP_FULL, one, one) == (0, 0)  # order 1: one sweep, nothing to meet
    # a Y of rank 1 (the sum of x's entries): room for x's cores folded with y
    ones = FakeDesc([16] * 10, [1] * 11)
    rc, nb = _ws(L, B.TT_OP_FULL, x, ones)
    assert rc == 0 and nb >= 4 * (64 + 8 * 64 * 64 + 64)
    assert _ws(L, B.TT_OP_PARTIAL, x, x, [1] * 6 + [0] * 4) == (0, 0)  # chain: K stays on chip
    # tensor-core forms: bfloat16 storage, or float32 storage with bf16 / bf16x3 products
    xb = FakeDesc([32] * 4, [1, 256, 128, 256, 1], dtype=B.TT_BF16)
    yb = FakeDesc([32] * 4, [1, 64, 192, 256, 1], dtype=B.TT_BF16)
    rc, nb = _ws(L, B.TT_OP_FULL, xb, yb)
    assert rc == 0 and nb > 0
    x32 = FakeDesc([32] * 4, [1, 128, 128, 128, 1])
    y32 = FakeDesc([32] * 4, [1, 128, 64, 128, 1])
    r3, n3 = _ws(L, B.TT_OP_FULL, x32, y32, prec="bf16x3")
    r1, n1 = _ws(L, B.TT_OP_FULL, x32, y32, prec="bf16")
    assert r3 == 0 and r1 == 0 and n3 > n1 > 0      # the split form keeps hi and lo copies
    assert _ws(L, B.TT_OP_FULL, FakeDesc([32] * 4, [1, 64, 64, 64, 1], dtype=B.TT_BF16), yb)[0] == -8
    assert _ws(L, B.TT_OP_FULL, xb, FakeDesc([32] * 4, [1, 96, 64, 64, 1], dtype=B.TT_BF16))[0] == -8
    assert _ws(L, B.TT_OP_FULL, FakeDesc([32] * 2, [1, 128, 1], dtype=B.TT_BF16),
               FakeDesc([32] * 2, [1, 128, 1], dtype=B.TT_BF16))[0] == -8
    x64 = FakeDesc([32] * 4, [1, 128, 128, 128, 1], dtype=B.TT_F64)
    assert _ws(L, B.TT_OP_FULL, x64, x64, prec="bf16")[0] == -3  # bf16 products need float32 storage
    # backward: the adjoint's rank cap, lifted when Y has rank 1 everywhere (the vector adjoint)
    xs = FakeDesc([4] * 5, [1, 3, 3, 3, 3, 1])
    rc, nb = _ws(L, B.TT_OP_BACKWARD, xs, xs)
    assert rc == 0 and nb > 0
    rc, nb = _ws(L, B.TT_OP_BACKWARD, xs, xs, [1, 1, 0, 0, 0])
    assert rc == 0 and nb > 0
    wide = FakeDesc([4] * 3, [1, 33, 33, 1], dtype=B.TT_F64)
    ones = FakeDesc([4] * 3, [1, 1, 1, 1], dtype=B.TT_F64)
    assert _ws(L, B.TT_OP_BACKWARD, wide, wide)[0] == -5
    rc, nb = _ws(L, B.TT_OP_BACKWARD, wide, ones)
    assert rc == 0 and nb > 0
    # the order-12 rank-64 gradient step: every left and right environment of
    # the 8-mode block and leg-swapped copies of its 16 cores fit (float32)
    x12 = FakeDesc([16] * 12, [1] + [64] * 11 + [1])
    rc, nb = _ws(L, B.TT_OP_BACKWARD, x12, x12, [1] * 8 + [0] * 4)
    env, core = 64 * 64 * 4, 64 * 16 * 64 * 4
    assert rc == 0 and nb >= 2 * 8 * env + 2 * 7 * core + 2 * 16 * 64 * 4  # the first cores have rank 1 on the left


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """With no built library the binding raises; there is no other code path
    to fall back to."""
    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B, "LIB_PATH", str(tmp_path / "libttc.so"))
    with pytest.raises(RuntimeError, match="not built"):
        B.lib()
