"""GPU parity of the tf32 tensor-core sweep (tcgen05.mma kind::tf32; precision
forms TT_P_TF32X3 and TT_P_TF32 on float32 cores with ranks <= 64) against the
float64 oracle.

Full contractions: |z - z*| <= the rounding-error model's bound for the form
(oracle/error_model.tf32_bound: 8 predicted standard deviations of the random
part plus twice the coherent shrinkage of the tensor-core accumulators),
one-sided (the last mode summed in float64 on the CUDA cores) and from both
ends (every mode on the tensor cores, the halves joined in float64).  The
split form is also held to the float32 contract: eps = |z - z*| / (||X|| ||Y||)
<= 1e-5.
Chain-layout partial contractions: the copied free cores bit for bit; the
joined core C within the per-entry Cauchy-Schwarz scale of the oracle's
(|Gx| max times the largest sqrt(Gram_x[a, a] Gram_y[b, b]) of K times
sqrt(rank)): 1e-5 for tf32x3, 8 * 2^-11 * sqrt(2 s) for tf32 (two tf32
roundings per contracted mode, s modes); small cases against the dense Eq. 8
within the per-entry scale ||X[., i_F]|| ||Y[., j_F]|| (with nothing
contracted, C entry by entry: one tf32 rounding, 2^-11, or 2^-20 for the
split).
The measured errors are printed (pytest -s).
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from helpers import cs_bound, dense_cs_eps, norm_scale, to_dev, to_host
from oracle import error_model as M
from paper_2109_00626_gb300 import inputs as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2109_00626_gb300 as T  # noqa: E402
from paper_2109_00626_gb300 import _binding as B  # noqa: E402

PRECS = ["tf32x3", "tf32"]


def _full(x, y, prec, two_sided):
    """z through tt_contract_full: with the workspace (both ends) or without
    it (one sweep)."""
    op = T.FullContraction(to_dev(x), to_dev(y), prec=prec, split=True)
    if two_sided:
        op()
        torch.cuda.synchronize()
        return np.ldexp(float(op.out.item()), int(op.log2.item())), int(op.status.item())
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    lg = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = T.lib().tt_contract_full(ctypes.byref(op.xd.desc), ctypes.byref(op.yd.desc), B.PREC[prec],
                                  ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(lg.data_ptr()),
                                  ctypes.c_void_p(st.data_ptr()), None, 0, None)
    assert rc == 0
    torch.cuda.synchronize()
    return np.ldexp(float(out.item()), int(lg.item())), int(st.item())


def _check_full(x, y, prec, two_sided, label):
    x64 = [np.asarray(c, dtype=np.float64) for c in x]
    y64 = [np.asarray(c, dtype=np.float64) for c in y]
    z, st = _full(x, y, prec, two_sided)
    assert st == 0
    want = O.contract_full(x64, y64)
    bound = M.tf32_bound(x64, y64, prec, want, two_sided)
    eps = abs(z - want) / norm_scale(x64, y64)
    print(f"{label} {prec} two_sided={two_sided}: rel={abs(z - want) / abs(want):.2e} eps={eps:.2e} "
          f"err/bound={abs(z - want) / bound:.3f}")
    assert abs(z - want) <= bound
    if prec == "tf32x3":
        assert eps <= 1e-5
    return z, want


SMALL = [
    # modes, ranks x, ranks y (ragged ranks, ranks 1, a mode of size 1)
    ([4, 5, 3], [1, 32, 16, 1], [1, 8, 24, 1]),
    ([6, 3, 7, 2, 5], [1, 7, 64, 33, 5, 1], [1, 64, 2, 64, 9, 1]),
    ([3, 1, 17, 2], [1, 3, 3, 1, 1], [1, 1, 5, 64, 1]),
    ([40, 2], [1, 64, 1], [1, 64, 1]),
]


@pytest.mark.parametrize("two_sided", [False, True])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", range(len(SMALL)))
def test_full_small(case, prec, two_sided):
    modes, rx, ry = SMALL[case]
    rng = np.random.default_rng(100 + case)
    x = G.random_tt(rng, modes, rx, np.float32)
    y = G.random_tt(rng, modes, ry, np.float32)
    _check_full(x, y, prec, two_sided, f"small {modes}")


@pytest.mark.parametrize("prec", PRECS)
def test_full_order1(prec):
    rng = np.random.default_rng(5)
    x = G.random_tt(rng, [9], [1, 1], np.float32)
    y = G.random_tt(rng, [9], [1, 1], np.float32)
    _check_full(x, y, prec, False, "order 1")


@pytest.mark.parametrize("two_sided", [False, True])
@pytest.mark.parametrize("prec", PRECS)
def test_full_order10_rank64(prec, two_sided):
    """The order-10, mode-16, rank-64 pair of the benchmark, and <X, X>."""
    x, y = G.order10_r64(0)
    _check_full(x, y, prec, two_sided, "order10")
    z, want = _check_full(x, x, prec, two_sided, "order10 <X,X>")
    if prec == "tf32x3":
        assert abs(z - want) <= 2e-5 * want  # kappa = 1: the plain relative error


def test_full_scaled_cores_split_scale():
    """Cores scaled by 2^40 and 2^-40 alternately: the power-of-two
    renormalisation keeps the environments in range; z returned as mantissa
    and exponent."""
    x, y = G.pair(21, [6] * 8, G.tt_ranks(8, 48), G.tt_ranks(8, 32), np.float32)
    f = [2.0**40 if k % 2 == 0 else 2.0**-30 for k in range(8)]
    xs = [(c * np.float32(s)).astype(np.float32) for c, s in zip(x, f)]
    want = O.contract_full([c.astype(np.float64) for c in x], [c.astype(np.float64) for c in y])
    for two_sided in (False, True):
        z, st = _full(xs, y, "tf32x3", two_sided)
        assert st == 0
        got = z * 2.0 ** -sum(40 if k % 2 == 0 else -30 for k in range(8))
        print(f"scaled cores two_sided={two_sided}: rel={abs(got - want) / abs(want):.2e}")
        bound = M.tf32_bound([c.astype(np.float64) for c in x], [c.astype(np.float64) for c in y], "tf32x3", want,
                             two_sided)
        assert abs(got - want) <= bound


def _partial(x, y, mask, prec):
    op = T.PartialContraction(to_dev(x), to_dev(y), mask, prec=prec)
    op()
    torch.cuda.synchronize()
    return op, to_host(op.z)


def _c_tol(prec, s):
    return 1e-5 if prec == "tf32x3" else 8 * 2.0**-11 * np.sqrt(2 * max(s, 1))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("mask", [[1] * 6 + [0] * 4, [0] * 4 + [1] * 6, [1] + [0] * 9, [0] * 9 + [1], [0] * 10])
def test_partial_chain_order10(prec, mask):
    """Chain layout over leading and trailing blocks of the order-10 pair:
    copies bit for bit, C within its Cauchy-Schwarz scale."""
    x, y = G.order10_r64(0)
    op, got = _partial(x, y, mask, prec)
    assert int(op.status.item()) == 0
    want, perm = O.partial_chain(x, y, mask)
    assert op.perm == perm
    side, s = O.end_block(mask)
    m = len(x) - s
    for p, (g, w) in enumerate(zip(got, want)):
        if p == m - 1:
            kb = cs_bound(x, y, side, s) if s > 0 else np.ones((1, 1))
            gxb = x[s] if side == "lead" else x[m - 1]
            scale = np.abs(gxb).max() * kb.max() * np.sqrt(gxb.shape[0] if side == "lead" else gxb.shape[2])
            err = np.abs(g - w).max() / scale
            print(f"partial {''.join(map(str, mask))} {prec}: C err/scale={err:.2e} "
                  f"rel to max={np.abs(g - w).max() / np.abs(w).max():.2e}")
            assert err <= _c_tol(prec, s)
        else:
            np.testing.assert_array_equal(g, w)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("mask", [[1, 1, 0, 0, 0], [0, 0, 1, 1, 1], [1, 0, 0, 0, 0], [0, 0, 0, 0, 0], [1, 1, 1, 1, 0]])
def test_partial_chain_small_dense(prec, mask):
    """Small ragged pairs against the dense Eq. 8."""
    rng = np.random.default_rng(7 + sum(v << k for k, v in enumerate(mask)))
    modes = [3, 4, 2, 3, 2]
    x = G.random_tt(rng, modes, [1, 5, 12, 7, 3, 1], np.float32)
    y = G.random_tt(rng, modes, [1, 2, 9, 4, 6, 1], np.float32)
    op, got = _partial(x, y, mask, prec)
    assert int(op.status.item()) == 0
    _, perm = O.partial_chain(x, y, mask)
    x64 = [c.astype(np.float64) for c in x]
    y64 = [c.astype(np.float64) for c in y]
    contracted = [k for k in range(5) if mask[k]]
    if not contracted:
        # nothing contracted: C is the boundary core of X times K = [1], one
        # tf32 rounding (nearest) of each entry, or hi + lo with lo truncated
        want, _ = O.partial_chain(x64, y64, mask)
        c, w = got[len(x) - 1], want[len(x) - 1]
        rel = float(np.max(np.abs(c - w) / np.maximum(np.abs(w), 1e-300)))
        print(f"partial small {''.join(map(str, mask))} {prec}: C entrywise rel={rel:.2e}")
        assert rel <= (2.0**-11 if prec == "tf32" else 2.0**-20)
        return
    dense = O.chain_to_dense(got, perm)
    ref = O.tcp(O.tt_to_dense(x64), O.tt_to_dense(y64), contracted)
    eps = dense_cs_eps(dense, ref, x64, y64, contracted)
    print(f"partial small {''.join(map(str, mask))} {prec}: cs_eps={eps:.2e}")
    assert eps <= _c_tol(prec, len(contracted))


def test_tf32x3_agrees_with_native_float32():
    """The split form and the CUDA-core float32 sweep give the same result to
    within the float32 contract on the benchmark pair."""
    x, y = G.order10_r64(3)
    zt, _ = _full(x, y, "tf32x3", True)
    zn, _ = _full(x, y, "native", True)
    assert abs(zt - zn) <= 1e-5 * norm_scale(x, y)
