"""GPU parity of the hand-written adjoint (tt_contract_backward) against the
oracle's gradients, against central finite differences of the GPU forward in
float64, and through torch.autograd (TTFull / TTPartial)."""
import numpy as np
import pytest

import oracle as O
from helpers import grad_cs_eps, grad_cs_scale, to_dev, to_host
from paper_2109_00626_gb300 import inputs as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2109_00626_gb300 as T  # noqa: E402


def _rel(got, want):
    """max |got - want| over all cores / max |want| over all cores."""
    num = max(float(np.abs(g - w).max()) for g, w in zip(got, want))
    den = max(float(np.abs(w).max()) for w in want)
    return num / den


# float32 gradients: within 1e-5 of the largest oracle gradient (every core of
# both operands); the full-contraction gradients also within 1e-5 of their
# per-entry Cauchy-Schwarz scale.  float64: 1e-12.
F32_TOL = 1e-5


def test_full_grad_fd_fp64():
    """Finite-difference size: order 5, mode 4, ranks 3, float64.  z is linear
    in every core, so central differences of the GPU forward are exact up to
    rounding for any step; h = 1."""
    x, y = G.pair(5, [4] * 5, G.tt_ranks(5, 3), G.tt_ranks(5, 3), np.float64)
    xd, yd = to_dev(x), to_dev(y)
    cot = torch.tensor([1.0], dtype=torch.float64, device="cuda")
    gx, gy, st = T.backward(xd, yd, None, cot=cot)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    gxh, gyh = to_host(gx), to_host(gy)
    wx, wy = O.grad_full(x, y)
    assert _rel(gxh + gyh, wx + wy) <= 1e-12

    def z_of(xc, yc):
        op = T.FullContraction(xc, yc)
        op()
        return float(op.out.item())

    for k in range(5):
        for side in (0, 1):
            cores = xd if side == 0 else yd
            grad = gxh[k] if side == 0 else gyh[k]
            fd = np.zeros_like(grad)
            base = cores[k].clone()
            for idx in np.ndindex(*grad.shape):
                for sgn in (+1, -1):
                    cores[k] = base.clone()
                    cores[k][idx] += sgn * 1.0
                    val = z_of(xd, yd)
                    fd[idx] += sgn * val / 2.0
            cores[k] = base
            assert np.abs(fd - grad).max() <= 1e-12 * max(1.0, np.abs(grad).max())


def test_full_grad_cotangent_scaling_and_euler():
    x, y = G.pair(6, [6, 3, 5, 4], [1, 5, 7, 3, 1], [1, 2, 9, 4, 1], np.float64)
    xd, yd = to_dev(x), to_dev(y)
    cot = torch.tensor([-2.5], dtype=torch.float64, device="cuda")
    gx, gy, _ = T.backward(xd, yd, None, cot=cot)
    torch.cuda.synchronize()
    z = O.contract_full(x, y)
    for g, c in zip(to_host(gx) + to_host(gy), x + y):
        # Euler: <G_k, dz/dG_k> = z for every core
        assert abs(np.sum(g * c) / -2.5 - z) <= 1e-12 * max(1.0, abs(z))


@pytest.mark.parametrize("stride", [1, 2, 3, 10])
def test_full_grad_order10_fp32_checkpoint_strides(stride):
    """The order-10 gradients for every value of the checkpoint-stride
    argument (accepted and ignored: every environment is kept)."""
    x, y = G.order10_r64(0)
    xd, yd = to_dev(x), to_dev(y)
    cot = torch.tensor([1.0], dtype=torch.float64, device="cuda")
    gx, gy, st = T.backward(xd, yd, None, cot=cot, ckpt_stride=stride)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    wx, wy = O.grad_full(x, y)
    got = to_host(gx) + to_host(gy)
    rel, cs = _rel(got, wx + wy), grad_cs_eps(got, wx + wy, grad_cs_scale(x, y))
    print(f"order10 grads stride {stride}: rel={rel:.2e} cs_eps={cs:.2e}")
    assert rel <= F32_TOL and cs <= F32_TOL


def _sum_cotangents(zc):
    """Cotangents of the output cores for loss = sum of all entries of Z."""
    ones = [np.ones((1, c.shape[1], 1)) for c in zc]
    dz, _ = O.grad_full(zc, ones)
    return dz


@pytest.mark.parametrize("mask", [[1, 1, 1, 0, 0], [0, 0, 1, 1, 1], [1, 0, 0, 0, 0], [0, 0, 0, 0, 0]])
def test_partial_grad_fp64(mask):
    rng = np.random.default_rng(sum(mask) * 3 + mask[0])
    modes = [3, 4, 2, 3, 2]
    x = G.random_tt(rng, modes, [1, 2, 3, 4, 2, 1], np.float64)
    y = G.random_tt(rng, modes, [1, 3, 2, 2, 3, 1], np.float64)
    zc, _ = O.partial_chain(x, y, mask)
    dz = [rng.standard_normal(c.shape) for c in zc]
    gx, gy, st = T.backward(to_dev(x), to_dev(y), mask, dz=to_dev(dz))
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    wx, wy = O.grad_partial_chain(x, y, mask, dz)
    assert _rel(to_host(gx) + to_host(gy), wx + wy) <= 1e-12


def test_partial_grad_order12_sum_fp32():
    """Loss = sum of the partial contraction over modes 1-8 of the order-12,
    mode 16, rank 64 pair; gradients for all 24 cores."""
    x, y = G.order12_r64(0)
    mask = [1] * 8 + [0] * 4
    zc, _ = O.partial_chain(x, y, mask)
    dz = _sum_cotangents(zc)
    gx, gy, st = T.backward(to_dev(x), to_dev(y), mask, dz=to_dev(dz, torch.float32))
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    wx, wy = O.grad_partial_chain(x, y, mask, dz)
    rel = _rel(to_host(gx) + to_host(gy), wx + wy)
    print(f"order12 partial grads: rel={rel:.2e}")
    assert rel <= F32_TOL


def test_autograd_sum_of_partial_fp32():
    """torch.autograd through TTPartial and TTFull: loss = sum(Z)."""
    x, y = G.order12_r64(1)
    mask = [1] * 8 + [0] * 4
    xd = [c.requires_grad_(True) for c in to_dev(x)]
    yd = [c.requires_grad_(True) for c in to_dev(y)]
    zc = T.tt_partial(xd, yd, mask)
    loss = T.tt_sum(zc)
    loss.backward()
    zo, _ = O.partial_chain(x, y, mask)
    ones = [np.ones((1, c.shape[1], 1)) for c in zo]
    want_loss = O.contract_full(zo, ones)
    assert abs(float(loss.detach()) - want_loss) <= 1e-5 * max(1.0, abs(want_loss))
    dz = _sum_cotangents(zo)
    wx, wy = O.grad_partial_chain(x, y, mask, dz)
    got = [c.grad.detach().cpu().double().numpy() for c in xd + yd]
    rel = _rel(got, wx + wy)
    print(f"autograd order12: rel={rel:.2e}")
    assert rel <= F32_TOL


def test_autograd_gradcheck_full_fp64():
    x, y = G.pair(8, [3, 2, 3], [1, 2, 2, 1], [1, 3, 2, 1], np.float64)
    xd = [c.requires_grad_(True) for c in to_dev(x)]
    yd = [c.requires_grad_(True) for c in to_dev(y)]
    assert torch.autograd.gradcheck(lambda *c: T.tt_full(list(c[:3]), list(c[3:])), (*xd, *yd), eps=1e-6, atol=1e-9)


@pytest.mark.parametrize("lead", [True, False])
def test_partial_grad_uneven_ranks_fp32(lead):
    """Chain-layout gradients with ranks up to 64 that are not multiples of the
    16-byte width, mode sizes 3..9, both end blocks: the boundary core and dK
    (dK blocks, cp.async pipeline) within tolerance, and every free core's
    gradient -- a plain or leg-swapped copy of its cotangent -- exactly."""
    rng = np.random.default_rng(41 if lead else 43)
    modes = [5, 7, 3, 9, 4, 6]
    x = G.random_tt(rng, modes, [1, 64, 63, 37, 64, 50, 1], np.float32)
    y = G.random_tt(rng, modes, [1, 61, 64, 33, 64, 48, 1], np.float32)
    mask = [1, 1, 1, 0, 0, 0] if lead else [0, 0, 0, 1, 1, 1]
    zc, _ = O.partial_chain(x, y, mask)
    dz = [rng.standard_normal(c.shape).astype(np.float32) for c in zc]
    gx, gy, st = T.backward(to_dev(x), to_dev(y), mask, dz=to_dev(dz))
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    wx, wy = O.grad_partial_chain(x, y, mask, [d.astype(np.float64) for d in dz])
    gxh, gyh = to_host(gx), to_host(gy)
    rel = _rel(gxh + gyh, wx + wy)
    print(f"chain grads: rel={rel:.2e}")
    assert rel <= F32_TOL
    n, s = len(modes), 3
    free_x = range(s + 1, n) if lead else range(0, n - s - 1)  # the boundary core is X's s (lead) / n-s-1 (trail)
    free_y = range(s, n) if lead else range(0, n - s)
    for k in free_x:
        np.testing.assert_array_equal(gxh[k].astype(np.float64), wx[k])
    for k in free_y:
        np.testing.assert_array_equal(gyh[k].astype(np.float64), wy[k])


@pytest.mark.parametrize("dt,lead", [(np.float32, True), (np.float32, False), (np.float64, True), (np.float64, False)])
def test_partial_k_kept_for_backward(dt, lead):
    """tt_contract_partial_k writes the same output cores as the plain partial
    contraction and fills a backward workspace (K; for a leading block also
    every left environment, stored by the forward sweep); the backward pass
    that starts from it gives the oracle's gradients, like the one that
    recomputes everything."""
    rng = np.random.default_rng(51 if lead else 53)
    modes = [5, 7, 3, 9, 4, 6, 3, 2, 4]
    r = 64 if dt == np.float32 else 32
    rx = [1, 16, r - 1, 20, r, 8, r, 5, 9, 1]
    ry = [1, 12, r, 17, r - 3, 9, 11, r, 3, 1]
    x = G.random_tt(rng, modes, rx, dt)
    y = G.random_tt(rng, modes, ry, dt)
    mask = [1] * 7 + [0] * 2 if lead else [0] * 2 + [1] * 7  # seven contracted modes
    xd, yd = to_dev(x), to_dev(y)
    ref = T.PartialContraction(xd, yd, mask)
    ref()
    z = [torch.empty_like(c) for c in ref.z]
    fws, st = T.partial_k(xd, yd, mask, z)
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and int(ref.status.item()) == 0
    tol = 1e-5 if dt == np.float32 else 1e-12
    for a, b in zip(to_host(z), to_host(ref.z)):
        assert np.abs(a - b).max() <= tol * max(1.0, float(np.abs(b).max()))
    zo, _ = O.partial_chain(x, y, mask)
    dz = [rng.standard_normal(c.shape).astype(dt) for c in zo]
    dzd = to_dev(dz)
    wx, wy = O.grad_partial_chain(x, y, mask, [d.astype(np.float64) for d in dz])
    for kept in (None, fws):
        gx, gy, st = T.backward(xd, yd, mask, dz=dzd, fwd_ws=kept)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        rel = _rel(to_host(gx) + to_host(gy), wx + wy)
        print(f"{dt.__name__} grads: rel={rel:.2e}")
        assert rel <= (F32_TOL if dt == np.float32 else 1e-12)


@pytest.mark.parametrize(
    "dt,rx,scale",
    [
        (np.float32, [1, 33, 61, 56, 34, 1], 0),
        (np.float32, [1, 530, 40, 600, 7, 1], 0),
        (np.float64, [1, 23, 30, 1, 28, 1], 0),
        (np.float32, [1, 24, 24, 27, 41, 1], 20),
    ],
)
def test_full_grad_rank1_y(dt, rx, scale):
    """Full contraction with every rank of Y equal to 1 (the sum of a TT's
    entries is the case y = ones): the vector adjoint against the oracle's
    gradients, for ranks of X above the matrix path's cap (the environment
    columns then run in chunks), a mode of size 1, a cotangent, and cores
    scaled by 2^20 each (the vectors are renormalised on the way)."""
    rng = np.random.default_rng(sum(rx) + scale)
    modes = [3, 16, 1, 7, 5]
    x = G.random_tt(rng, modes, rx, dt)
    if scale:
        x = [c * dt(2.0**scale) for c in x]
    y = G.random_tt(rng, modes, [1] * 6, dt)
    cot = torch.tensor([-1.5], dtype=torch.float64, device="cuda")
    gx, gy, st = T.backward(to_dev(x), to_dev(y), None, cot=cot)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    wx, wy = O.grad_full(x, y, cot=-1.5)
    rx_, ry_ = _rel(to_host(gx), wx), _rel(to_host(gy), wy)
    print(f"{dt.__name__} grads: rel x {rx_:.2e} y {ry_:.2e}")
    assert rx_ <= (F32_TOL if dt == np.float32 else 1e-12)
    assert ry_ <= (F32_TOL if dt == np.float32 else 1e-12)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("modes,rx", [([5], [1, 1]), ([4, 6], [1, 9, 1]), ([1, 1], [1, 3, 1])])
def test_full_grad_rank1_y_short_trains(dt, modes, rx):
    """The vector adjoint on trains of order 1 and 2 (the left or right vector
    is the unit start for every core) and on modes of size 1."""
    rng = np.random.default_rng(len(modes) * 10 + rx[1])
    x = G.random_tt(rng, modes, rx, dt)
    y = G.random_tt(rng, modes, [1] * (len(modes) + 1), dt)
    cot = torch.tensor([0.75], dtype=torch.float64, device="cuda")
    gx, gy, st = T.backward(to_dev(x), to_dev(y), None, cot=cot)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    wx, wy = O.grad_full(x, y, cot=0.75)
    tol = F32_TOL if dt == np.float32 else 1e-12
    rx_, ry_ = _rel(to_host(gx), wx), _rel(to_host(gy), wy)
    print(f"{dt.__name__} grads: rel x {rx_:.2e} y {ry_:.2e}")
    assert rx_ <= tol and ry_ <= tol
