"""GPU checks of the tensor-core (tcgen05) full contraction in its three
precision forms, against the float64 oracle.

Bound: |z - z*| <= 8 sigma + 2 |b| |z*|, with sigma the standard deviation of
the error that oracle/error_model.py predicts for these operands from the
roundings the form makes (first-order model, each rounding an independent
relative perturbation) and b its predicted coherent bias (the tensor cores'
float32 accumulation rounds toward zero: half an ulp per accumulation step,
shrinking z).  Both parts are pinned against literal simulations of the
roundings in tests/test_error_model.py.
  bfloat16 products (cores stored or rounded to bfloat16), oracle on the
  bfloat16-rounded cores: E and each T_i rounded to bfloat16 at every interior
  mode (unit roundoff 2^-8), sums in float32;
  split bfloat16 x3 on float32 cores, oracle on the float32 cores: E, T_i and
  the interior cores held as hi + lo pieces (representation error ~2^-16
  relative), lo*lo dropped from every product, sums in float32.
sigma is data dependent: for a random pair at order 16 / rank 256 it is about
1 % of |z| for bfloat16 (kappa ~ 1e12) and about 4e-5 of |z| for x3; for
<X, X> (kappa = 1) 4e-4 and 6e-7 of |z|, with b = -2e-5 and -6e-5.  One
dropped mode slice moves z by several per cent.  The measured error over the
bound is printed (pytest -s).
"""
import numpy as np
import pytest

import oracle as O
from helpers import norm_scale, to_dev
from oracle import error_model as M
from paper_2109_00626_gb300 import inputs as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2109_00626_gb300 as T  # noqa: E402


def _bf16(cores):
    return [G.to_bf16_f32(c) for c in cores]


def _run(xd, yd, prec, split=False):
    op = T.FullContraction(xd, yd, prec=prec, split=split)
    op()
    torch.cuda.synchronize()
    st = int(op.status.item())
    if split:
        return float(op.out.item()), int(op.log2.item()), st
    return float(op.out.item()), st


SMALL = [
    # modes, ranks x, ranks y
    ([5, 8, 3, 6], [1, 128, 256, 128, 1], [1, 64, 192, 128, 1]),
    ([4, 16, 2], [1, 256, 128, 1], [1, 256, 64, 1]),
    ([7, 1, 32, 9, 3], [1, 128, 128, 256, 128, 1], [1, 128, 64, 256, 192, 1]),
]


@pytest.mark.parametrize("modes,rx,ry", SMALL)
def test_bf16_storage_native(modes, rx, ry):
    rng = np.random.default_rng(len(modes) * 7 + modes[0])
    x = _bf16(G.random_tt(rng, modes, rx, np.float32))
    y = _bf16(G.random_tt(rng, modes, ry, np.float32))
    z, st = _run(to_dev(x, torch.bfloat16), to_dev(y, torch.bfloat16), "native")
    assert st == 0
    want = O.contract_full(x, y)
    bound = M.tc_bound(x, y, "bf16", want)
    print(f"bf16 native {modes}: eps={abs(z - want) / norm_scale(x, y):.3e} err/bound={abs(z - want) / bound:.3f}")
    assert abs(z - want) <= bound


@pytest.mark.parametrize("modes,rx,ry", SMALL)
def test_bf16x3_on_fp32(modes, rx, ry):
    rng = np.random.default_rng(len(modes) * 11 + modes[0])
    x = G.random_tt(rng, modes, rx, np.float32)
    y = G.random_tt(rng, modes, ry, np.float32)
    z, st = _run(to_dev(x), to_dev(y), "bf16x3")
    assert st == 0
    want = O.contract_full(x, y)
    bound = M.tc_bound(x, y, "bf16x3", want)
    print(f"bf16x3 {modes}: eps={abs(z - want) / norm_scale(x, y):.3e} err/bound={abs(z - want) / bound:.3f}")
    assert abs(z - want) <= bound


def test_bf16_rounding_of_fp32_matches_bf16_storage():
    rng = np.random.default_rng(3)
    modes, rx, ry = SMALL[0]
    x = G.random_tt(rng, modes, rx, np.float32)
    y = G.random_tt(rng, modes, ry, np.float32)
    z1, s1 = _run(to_dev(x), to_dev(y), "bf16")
    z2, s2 = _run(to_dev(x, torch.bfloat16), to_dev(y, torch.bfloat16), "native")
    assert s1 == 0 and s2 == 0 and z1 == z2


def test_order16_r256_lognormal_both_forms():
    """Order 16, modes 32, ranks 256, log-normal core scales: bfloat16 cores
    with float32 sums, and the split-bfloat16 x3 variant on the float32 cores."""
    x, y = G.order16_r256(0)
    scale32 = norm_scale(x, y)
    want32 = O.contract_full(x, y)
    z3, e3, st = _run(to_dev(x), to_dev(y), "bf16x3", split=True)
    assert st == 0
    eps3 = abs(np.ldexp(z3, e3) - want32) / scale32
    xb, yb = _bf16(x), _bf16(y)
    want16 = O.contract_full(xb, yb)
    zb, eb, st = _run(to_dev(xb, torch.bfloat16), to_dev(yb, torch.bfloat16), "native", split=True)
    assert st == 0
    eps16 = abs(np.ldexp(zb, eb) - want16) / norm_scale(xb, yb)
    eps16_e2e = abs(np.ldexp(zb, eb) - want32) / scale32
    z16, zx3 = np.ldexp(zb, eb), np.ldexp(z3, e3)
    print(f"order16 r256: bf16 eps={eps16:.3e} (vs fp32 cores {eps16_e2e:.3e}); bf16x3 eps={eps3:.3e}; "
          f"z* fp32={want32:.6e} bf16={want16:.6e} got bf16={z16:.6e} x3={zx3:.6e} kappa={scale32 / abs(want32):.2e}")
    b16 = M.tc_bound(xb, yb, "bf16", want16)
    b3 = M.tc_bound(x, y, "bf16x3", want32)
    print(f"  err/bound: bf16 {abs(z16 - want16) / b16:.3f} (bound/|z*| {b16 / abs(want16):.2e}), "
          f"x3 {abs(zx3 - want32) / b3:.3f} (bound/|z*| {b3 / abs(want32):.2e})")
    assert abs(z16 - want16) <= b16
    assert abs(zx3 - want32) <= b3
    assert b3 <= 1e-3 * abs(want32)  # the x3 bound is a small fraction of |z*|


@pytest.mark.parametrize("prec", ["native", "bf16x3"])
def test_order16_r256_norm_invariant(prec):
    """<X, X> = ||X||_F^2 (condition number 1) at the full order-16, rank-256
    size: the plain relative error is meaningful here."""
    x, _ = G.order16_r256(1)
    if prec == "native":
        xb = _bf16(x)
        want = O.contract_full(xb, xb)
        z, e, st = _run(to_dev(xb, torch.bfloat16), to_dev(xb, torch.bfloat16), "native", split=True)
        bound = M.tc_bound(xb, xb, "bf16", want)
    else:
        want = O.contract_full(x, x)
        z, e, st = _run(to_dev(x), to_dev(x), "bf16x3", split=True)
        bound = M.tc_bound(x, x, "bf16x3", want)
    assert st == 0
    err = abs(np.ldexp(z, e) - want)
    print(f"order16 r256 <X,X> {prec}: rel={err / want:.3e} err/bound={err / bound:.3f} bound/z={bound / want:.2e}")
    assert err <= bound
    assert bound <= 5e-3 * want  # far below the few per cent one dropped slice costs
