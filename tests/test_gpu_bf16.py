"""GPU checks of the tensor-core (tcgen05) full contraction in its three
precision forms, against the float64 oracle.

Error measure: eps = |z - z*| / (||X||_F ||Y||_F).
  bfloat16 products (cores stored or rounded to bfloat16), oracle on the
  bfloat16-rounded cores:      eps <= 2N * 2^-8   (rounding of E and T to
                               bfloat16 at every mode, unit roundoff 2^-9,
                               two roundings per mode)
  split bfloat16 x3 on float32 cores, oracle on the float32 cores:
                               eps <= 2N * 2^-15  (the dropped lo*lo term and
                               the second rounding are below 2^-16 relative)
The measured errors are printed (pytest -s) and stay well inside.
"""
import numpy as np
import pytest

import oracle as O
from helpers import norm_scale, to_dev
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
    eps = abs(z - want) / norm_scale(x, y)
    print(f"bf16 native {modes}: eps={eps:.3e}")
    assert eps <= 2 * len(modes) * 2.0**-8


@pytest.mark.parametrize("modes,rx,ry", SMALL)
def test_bf16x3_on_fp32(modes, rx, ry):
    rng = np.random.default_rng(len(modes) * 11 + modes[0])
    x = G.random_tt(rng, modes, rx, np.float32)
    y = G.random_tt(rng, modes, ry, np.float32)
    z, st = _run(to_dev(x), to_dev(y), "bf16x3")
    assert st == 0
    want = O.contract_full(x, y)
    eps = abs(z - want) / norm_scale(x, y)
    print(f"bf16x3 {modes}: eps={eps:.3e}")
    assert eps <= 2 * len(modes) * 2.0**-15


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
    # the results are not trivially small: they agree with the oracle to a fraction of |z*|
    assert abs(zx3 - want32) <= 1e-3 * abs(want32)
    assert eps16 <= 2 * 16 * 2.0**-8
    assert eps3 <= 2 * 16 * 2.0**-15


@pytest.mark.parametrize("prec", ["native", "bf16x3"])
def test_order16_r256_norm_invariant(prec):
    """<X, X> = ||X||_F^2 (condition number 1) at the full order-16, rank-256
    size: the plain relative error is meaningful here."""
    x, _ = G.order16_r256(1)
    if prec == "native":
        xb = _bf16(x)
        want = O.contract_full(xb, xb)
        z, e, st = _run(to_dev(xb, torch.bfloat16), to_dev(xb, torch.bfloat16), "native", split=True)
        bound = 2 * 16 * 2.0**-8
    else:
        want = O.contract_full(x, x)
        z, e, st = _run(to_dev(x), to_dev(x), "bf16x3", split=True)
        bound = 2 * 16 * 2.0**-15
    assert st == 0
    rel = abs(np.ldexp(z, e) - want) / want
    print(f"order16 r256 <X,X> {prec}: rel={rel:.3e} z={np.ldexp(z, e):.6e} want={want:.6e}")
    assert rel <= bound
