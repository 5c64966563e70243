"""Pins of the rounding-error model (oracle/error_model.py) on the CPU.

The model predicts the standard deviation of z - z* for a sweep whose
quantities are rounded at stated places.  Here the rounding process it
describes is carried out literally in numpy (float64 arithmetic with explicit
rounding to 8 significant bits at exactly those places) over many seeded
draws, and the spread of the simulated errors is compared with the
prediction, one kind of rounding at a time.  The model is then used as the
GPU tests use it: at the order-16, mode-32, rank-256 size, a sweep that drops
one mode slice, or reads the environment transposed, lands far outside the
bound, while the predicted spread stays far below |z|.
"""
import numpy as np
import pytest

import oracle as O
from oracle import error_model as M
from paper_2109_00626_gb300 import inputs as G


def _round_bits(x, bits):
    """Round to `bits` significant bits, nearest, ties to even (float64 in and out)."""
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 2.0**bits) / 2.0**bits, e)


def _split(x, bits):
    hi = _round_bits(x, bits)
    return hi, _round_bits(x - hi, bits)


def _sim_sweep(xc, yc, mode):
    """<X, Y> by the sweep with the roundings of `mode`:
      "e"   L_k rounded at the interior modes
      "t"   T_i rounded at the interior modes
      "x3"  E, T_i and the interior cores held as hi + lo (8 bits each), each
            product formed as hi*hi + hi*lo + lo*hi (lo*lo dropped)."""
    n = len(xc)
    e = np.ones((1, 1))
    for k in range(n):
        interior = 0 < k < n - 1
        gx, gy = xc[k], yc[k]
        out = np.zeros((gx.shape[2], gy.shape[2]))
        if mode == "x3" and interior:
            eh, el = _split(e, 8)
            for i in range(gx.shape[1]):
                ah, al = _split(gx[:, i, :], 8)
                bh, bl = _split(gy[:, i, :], 8)
                t = eh @ bh + eh @ bl + el @ bh
                th, tl = _split(t, 8)
                out += ah.T @ th + ah.T @ tl + al.T @ th
        else:
            ein = _round_bits(e, 8) if (mode == "e" and interior) else e
            for i in range(gx.shape[1]):
                t = ein @ gy[:, i, :]
                if mode == "t" and interior:
                    t = _round_bits(t, 8)
                out += gx[:, i, :].T @ t
        e = out
    return float(e[0, 0])


def _ratios(mode, rounds, n_draws=120):
    out = []
    for s in range(n_draws):
        rng = np.random.default_rng(1000 + s)
        x = G.random_tt(rng, [4, 3, 5, 4, 3], [1, 12, 16, 16, 12, 1], np.float64)
        y = G.random_tt(rng, [4, 3, 5, 4, 3], [1, 16, 12, 16, 16, 1], np.float64)
        z = O.contract_full(x, y)
        sig = M.sweep_error_sigma(x, y, rounds, modes=[1, 2, 3])
        out.append((_sim_sweep(x, y, mode) - z) / sig)
    return np.array(out)


@pytest.mark.parametrize("mode,kind", [("e", "e"), ("t", "t")])
def test_model_predicts_rounding_of_one_kind(mode, kind):
    """Only E (or only T) rounded to bfloat16: the simulated errors, divided
    by the predicted standard deviation, have a root mean square near 1."""
    r = _ratios(mode, {kind: M.rn_std(M.U_BF16)})
    rms = float(np.sqrt(np.mean(r**2)))
    assert 0.7 <= rms <= 1.4, rms
    assert np.abs(r).max() <= 5.0


def test_model_predicts_split_x3():
    """The split form (hi + lo pieces of E, T and the cores; lo*lo dropped)."""
    s = M.rn_std(M.U_BF16) ** 2
    r = _ratios("x3", {"e": s, "t": s, "core": s, "prod": s})
    rms = float(np.sqrt(np.mean(r**2)))
    assert 0.5 <= rms <= 1.5, rms
    assert np.abs(r).max() <= 5.0


def test_model_missing_a_term_is_caught():
    """A model that forgot the T roundings predicts far too little for a sweep
    that rounds both E and T (the pin above bites on each term)."""
    rng = np.random.default_rng(7)
    x = G.random_tt(rng, [4, 3, 5, 4, 3], [1, 12, 16, 16, 12, 1], np.float64)
    y = G.random_tt(rng, [4, 3, 5, 4, 3], [1, 16, 12, 16, 16, 1], np.float64)
    s = M.rn_std(M.U_BF16)
    both = M.sweep_error_sigma(x, y, {"e": s, "t": s}, modes=[1, 2, 3])
    only_e = M.sweep_error_sigma(x, y, {"e": s}, modes=[1, 2, 3])
    assert both > 1.3 * only_e


def test_rn_std_of_bfloat16_rounding():
    """The relative standard deviation of one rounding to 8 bits, measured on
    log-uniform samples, matches rn_std(2^-8)."""
    rng = np.random.default_rng(3)
    v = np.exp(rng.uniform(-20, 20, size=200000)) * rng.choice([-1, 1], size=200000)
    rel = (_round_bits(v, 8) - v) / v
    assert abs(np.std(rel) / M.rn_std(M.U_BF16) - 1) < 0.02


def _rz32(v):
    """float64 -> the float32 value next to it toward zero."""
    f = np.asarray(v, dtype=np.float64).astype(np.float32)
    over = np.abs(f.astype(np.float64)) > np.abs(v)
    f[over] = np.nextafter(f[over], np.float32(0))
    return f.astype(np.float64)


def _gemm_rz(a, b, step=16):
    """a @ b accumulated over the inner index in steps of 16 exact products,
    each step added to a float32 accumulator rounding toward zero."""
    d = np.zeros((a.shape[0], b.shape[1]))
    for k0 in range(0, a.shape[1], step):
        d = _rz32(d + a[:, k0:k0 + step] @ b[k0:k0 + step])
    return d


def _sim_sweep_rz(xc, yc, cluster):
    """<X, Y> with the interior modes' two GEMMs accumulated toward zero in
    float32 (P over the slices of one CTA in one accumulator; the CTAs' P's
    added exactly), the end modes exact."""
    n = len(xc)
    e = np.ones((1, 1))
    for k in range(n):
        gx, gy = xc[k], yc[k]
        if 0 < k < n - 1:
            out = np.zeros((gx.shape[2], gy.shape[2]))
            for c in range(cluster):
                p = np.zeros_like(out)
                for i in range(c, gx.shape[1], cluster):
                    t = _gemm_rz(e, gy[:, i, :])
                    for k0 in range(0, gx.shape[0], 16):
                        p = _rz32(p + gx[k0:k0 + 16, i, :].T @ t[k0:k0 + 16])
                out += p
            e = out
        else:
            e = O.absorb_left(e, gx, gy)
    return float(e[0, 0])


def test_model_predicts_round_toward_zero_bias():
    """Accumulation toward zero shrinks <X, X> by the predicted relative bias
    (mean over seeds within a factor of two; every seed shrinks)."""
    rel = []
    for s in range(12):
        rng = np.random.default_rng(300 + s)
        x = G.random_tt(rng, [4] * 6, [1, 32, 48, 32, 48, 32, 1], np.float64)
        z = O.contract_full(x, x)
        rel.append((_sim_sweep_rz(x, x, cluster=2) - z) / z)
    # the model's count: GEMM 1 ceil(R^y / 16) steps, GEMM 2 ceil(R^x / 16) steps x 2 slices per CTA
    pred = -sum(M.acc_bias_rel(-(-x[k].shape[0] // 16)) + M.acc_bias_rel(-(-x[k].shape[0] // 16) * 2)
                for k in range(1, 5))
    assert all(r < 0 for r in rel), rel
    assert 0.5 <= np.mean(rel) / pred <= 2.0, (np.mean(rel), pred)


def test_tc_bias_counts_roundings():
    """tc_bias: three products per step for the split form, one otherwise;
    only interior modes; slices per CTA = ceil(I / cluster)."""
    x = [np.zeros((1, 4, 64)), np.zeros((64, 32, 128)), np.zeros((128, 32, 64)), np.zeros((64, 4, 1))]
    y = [np.zeros((1, 4, 32)), np.zeros((32, 32, 256)), np.zeros((256, 32, 16)), np.zeros((16, 4, 1))]
    # mode 1: T over 32/16 = 2 steps, P over 64/16 = 4 steps x 2 slices; mode 2: T 16 steps, P 8 x 2
    n_r = (2 + 4 * 2) + (16 + 8 * 2)
    assert M.tc_bias(x, y, "bf16") == -0.5 * n_r * M.U_F32
    assert M.tc_bias(x, y, "bf16x3") == -1.5 * n_r * M.U_F32


def _trunc_bits(x, bits):
    """Round toward zero to `bits` significant bits."""
    m, e = np.frexp(x)
    return np.ldexp(np.trunc(m * 2.0**bits) / 2.0**bits, e)


def _tf32_repr(x, x3):
    """The value the tf32 sweep multiplies: tf32(x), or hi + (lo with its low
    bits dropped) for the split form."""
    hi = _round_bits(x, 11)
    return hi + _trunc_bits(x - hi, 11) if x3 else hi


def _sim_sweep_tf32(xc, yc, x3, modes):
    """<X, Y> with E, each T_i and the core slices of `modes` replaced by their
    tf32 representation (float64 arithmetic otherwise)."""
    e = np.ones((1, 1))
    for k, (gx, gy) in enumerate(zip(xc, yc)):
        out = np.zeros((gx.shape[2], gy.shape[2]))
        if k in modes:
            er = _tf32_repr(e, x3)
            for i in range(gx.shape[1]):
                t = _tf32_repr(er @ _tf32_repr(gy[:, i, :], x3), x3)
                out += _tf32_repr(gx[:, i, :], x3).T @ t
        else:
            for i in range(gx.shape[1]):
                out += gx[:, i, :].T @ e @ gy[:, i, :]
        e = out
    return float(e[0, 0])


@pytest.mark.parametrize("prec", ["tf32", "tf32x3"])
def test_model_predicts_tf32_forms(prec):
    """The tf32 forms' random part (tf32_rounds without accumulation) against
    a literal simulation of their representations, over 120 seeds."""
    r = []
    rounds = dict(M.tf32_rounds(prec))
    rounds.pop("acc")
    for s in range(120):
        rng = np.random.default_rng(2000 + s)
        x = G.random_tt(rng, [4, 3, 5, 4, 3], [1, 12, 16, 16, 12, 1], np.float64)
        y = G.random_tt(rng, [4, 3, 5, 4, 3], [1, 16, 12, 16, 16, 1], np.float64)
        z = O.contract_full(x, y)
        sig = M.sweep_error_sigma(x, y, rounds, modes=[0, 1, 2, 3])
        r.append((_sim_sweep_tf32(x, y, prec == "tf32x3", [0, 1, 2, 3]) - z) / sig)
    rms = float(np.sqrt(np.mean(np.square(r))))
    assert 0.5 <= rms <= 1.5, rms
    assert np.abs(r).max() <= 5.0


def _absorb_drop_slice(e, gx, gy, drop=5):
    out = np.zeros((gx.shape[2], gy.shape[2]))
    for i in range(gx.shape[1]):
        if i != drop:
            out += gx[:, i, :].T @ e @ gy[:, i, :]
    return out


def _absorb_transposed(e, gx, gy):
    if e.shape[0] != e.shape[1]:
        return O.absorb_left(e, gx, gy)
    out = np.zeros((gx.shape[2], gy.shape[2]))
    for i in range(gx.shape[1]):
        out += gx[:, i, :].T @ e.T @ gy[:, i, :]
    return out


def _sweep_with(xc, yc, absorb, k_bad):
    e = np.ones((1, 1))
    for k, (gx, gy) in enumerate(zip(xc, yc)):
        e = absorb(e, gx, gy) if k == k_bad else O.absorb_left(e, gx, gy)
    return float(e[0, 0])


@pytest.mark.slow
def test_bounds_reject_slips_at_order16_rank256():
    """At the order-16 / mode-32 / rank-256 workload the GPU tests' bounds
    (8 predicted standard deviations plus twice the coherent bias) catch one dropped mode slice, or the
    environment read transposed, in one interior mode:
      <X, X> on the bfloat16 cores, bfloat16 form (a symmetric environment:
      only the dropped slice is a slip there);
      the random pair X, Y on the float32 cores, split x3 form, and on the
      bfloat16 cores, bfloat16 form."""
    x, y = G.order16_r256(1)
    xb = [G.to_bf16_f32(c).astype(np.float64) for c in x]
    z = O.contract_full(xb, xb)
    bound = M.tc_bound(xb, xb, "bf16", z)
    assert bound < 5e-3 * abs(z)
    assert abs(_sweep_with(xb, xb, _absorb_drop_slice, 7) - z) > 5 * bound
    x, y = G.order16_r256(0)
    for prec, xs, ys in (("bf16x3", [c.astype(np.float64) for c in x], [c.astype(np.float64) for c in y]),
                         ("bf16", [G.to_bf16_f32(c).astype(np.float64) for c in x],
                          [G.to_bf16_f32(c).astype(np.float64) for c in y])):
        z = O.contract_full(xs, ys)
        bound = M.tc_bound(xs, ys, prec, z)
        for absorb in (_absorb_drop_slice, _absorb_transposed):
            dz = abs(_sweep_with(xs, ys, absorb, 7) - z)
            assert dz > (5 if prec == "bf16x3" else 1) * bound, (prec, absorb.__name__, dz / bound)
