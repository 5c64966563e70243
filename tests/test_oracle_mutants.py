"""Planted slips in the oracle (on the CPU) must be caught by the pins.

Each mutant patches one oracle function with a plausible mistake; the test
then evaluates the independent check used in test_oracle_pins.py and asserts
that it now fails.  This shows that the pins constrain every part they cover.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from oracle import tt_oracle as T
from paper_2109_00626_gb300 import inputs as G


def _dense_by_entries(cores):
    shape = tuple(g.shape[1] for g in cores)
    out = np.empty(shape)
    for idx in itertools.product(*[range(s) for s in shape]):
        m = np.ones((1, 1))
        for g, i in zip(cores, idx):
            m = m @ g[:, i, :]
        out[idx] = m[0, 0]
    return out


def _absorb_drop_first_slice(e, gx, gy):
    out = np.zeros((gx.shape[2], gy.shape[2]))
    for i in range(1, gx.shape[1]):
        out += gx[:, i, :].T @ e @ gy[:, i, :]
    return out


def _absorb_transposed_env(e, gx, gy):
    out = np.zeros((gx.shape[2], gy.shape[2]))
    for i in range(gx.shape[1]):
        out += gx[:, i, :].T @ e.T @ gy[:, i, :]
    return out


def _absorb_sign(e, gx, gy):
    out = np.zeros((gx.shape[2], gy.shape[2]))
    for i in range(gx.shape[1]):
        out += (-1) ** i * (gx[:, i, :].T @ e @ gy[:, i, :])
    return out


@pytest.mark.parametrize("mutant", [_absorb_drop_first_slice, _absorb_transposed_env, _absorb_sign])
def test_full_pin_catches_absorb_mutants(mutant, monkeypatch):
    x, y = G.pair(11, [3, 4, 3], [1, 3, 3, 1], [1, 3, 3, 1], np.float64)
    ref = math.fsum((_dense_by_entries(x) * _dense_by_entries(y)).ravel())
    assert abs(O.contract_full(x, y) - ref) < 1e-14
    monkeypatch.setattr(T, "absorb_left", mutant)
    assert abs(T.contract_full(x, y) - ref) > 1e-6


def test_chain_pin_catches_unswapped_legs(monkeypatch):
    x, y = G.pair(12, [2, 3, 2, 3], [1, 2, 2, 2, 1], [1, 2, 2, 2, 1], np.float64)
    want = O.tcp(_dense_by_entries(x), _dense_by_entries(y), [0])
    monkeypatch.setattr(T, "_swap_rank_legs", lambda g: np.ascontiguousarray(g))
    try:
        cores, perm = T.partial_chain(x, y, [1, 0, 0, 0])
        got = T.chain_to_dense(cores, perm)
        assert got.shape != want.shape or np.abs(got - want).max() > 1e-6
    except ValueError:
        pass  # leg sizes no longer join: caught as well


def test_chain_pin_catches_wrong_perm(monkeypatch):
    x, y = G.pair(13, [2, 3, 4, 2], [1, 2, 3, 2, 1], [1, 3, 2, 2, 1], np.float64)
    want = O.tcp(_dense_by_entries(x), _dense_by_entries(y), [0, 1])
    cores, perm = O.partial_chain(x, y, [1, 1, 0, 0])
    np.testing.assert_allclose(O.chain_to_dense(cores, perm), want, atol=1e-14)
    bad = list(perm)
    bad[0], bad[1] = bad[1], bad[0]
    got = O.chain_to_dense(cores, bad)
    assert got.shape != want.shape or np.abs(got - want).max() > 1e-6


def test_grad_pin_catches_shifted_env(monkeypatch):
    x, y = G.pair(14, [3, 3, 3], [1, 2, 2, 1], [1, 2, 2, 1], np.float64)
    z = O.contract_full(x, y)

    def bad_grad_sweep(xc, yc, start=None, end=None):
        le = T.left_envs(xc, yc, start)
        fe = T.right_envs(xc, yc, end)
        gx = []
        for k, (a, b) in enumerate(zip(xc, yc)):
            d = np.zeros_like(a)
            f = fe[min(k + 2, len(fe) - 1)]
            for i in range(a.shape[1]):
                if f.shape[0] != a.shape[2]:
                    f = fe[k + 1] * 1.5
                d[:, i, :] = le[k] @ b[:, i, :] @ f.T
            gx.append(d)
        return gx, [np.zeros_like(b) for b in yc]

    monkeypatch.setattr(T, "grad_sweep", bad_grad_sweep)
    gx, _ = T.grad_full(x, y)
    # Euler's identity <G_k, dz/dG_k> = z fails for at least one core
    assert max(abs(np.sum(g * c) - z) for g, c in zip(gx, x)) > 1e-6


# ---- compensated accumulation ----

def _dot2_no_error_sum(x, y):
    x, y = np.broadcast_arrays(np.asarray(x, dtype=np.float64), np.asarray(y, dtype=np.float64))
    p = x[..., 0] * y[..., 0]
    for k in range(1, x.shape[-1]):
        p = p + x[..., k] * y[..., k]
    return p, np.zeros_like(p)


def _absorb_dd_drop_lo(ehi, elo, gx, gy):
    return _ORIG_ABSORB_DD(ehi, np.zeros_like(elo), gx, gy)


def _two_product_no_error(a, b):
    return a * b, np.zeros_like(a * b)


_ORIG_ABSORB_DD = T.absorb_left_dd


def _cancelling_pair():
    rng = np.random.default_rng(21)
    x = G.random_tt(rng, [3, 2, 3], [1, 2, 3, 1], np.float64)
    w = [c.copy() for c in x]
    w[0] = w[0] * -(1 + 2.0**-30)
    # Y = X + X'' as a TT sum: first cores side by side, interior block-diagonal, last stacked
    y = [np.concatenate([x[0], w[0]], axis=2)]
    g = np.zeros((4, 2, 6))
    g[:2, :, :3] = x[1]
    g[2:, :, 3:] = w[1]
    y.append(g)
    y.append(np.concatenate([x[2], w[2]], axis=0))
    return x, y


@pytest.mark.parametrize("name,mutant", [("dot2_dd", _dot2_no_error_sum), ("absorb_left_dd", _absorb_dd_drop_lo),
                                         ("two_product", _two_product_no_error)])
def test_cancellation_pin_catches_compensation_mutants(name, mutant, monkeypatch):
    x, y = _cancelling_pair()
    # reference from the unmutated compensated sweep; its own pin (exact rationals) is in test_oracle_pins
    ref = O.contract_full_dd(x, y)
    monkeypatch.setattr(T, name, mutant)
    assert abs(T.contract_full_dd(x, y) - ref) > 1e3 * 2.0**-53 * abs(ref)


def _reverse_without_swap(cores):
    return [np.asarray(g, dtype=np.float64).copy() for g in reversed(cores)]


def _svd_keep_one_too_few(x, eps=0.0):
    cores = _ORIG_TT_SVD(x, eps)
    # drop the last rank-1 direction of the first bond
    if cores[0].shape[2] > 1:
        cores[0] = cores[0][:, :, :-1]
        cores[1] = cores[1][:-1]
    return cores


_ORIG_TT_SVD = T.tt_svd


def test_pairs_pin_catches_reversal_without_leg_swap(monkeypatch):
    x, y = G.pair(14, [2, 3, 2], [1, 2, 3, 1], [1, 2, 2, 1], np.float64)
    y5 = G.random_tt(np.random.default_rng(5), [3, 2, 2, 3, 2], [1, 2, 3, 2, 2, 1], np.float64)
    pairs = [(0, 4), (1, 3)]  # X's leading block against Y's trailing block (Y reversed)
    want = O.tcp_pairs(O.tt_to_dense(x), O.tt_to_dense(y5), pairs)
    cores, perm = O.partial_chain_pairs(x, y5, pairs)
    assert np.abs(O.chain_to_dense(cores, perm) - want).max() < 1e-13
    monkeypatch.setattr(T, "reverse_tt", _reverse_without_swap)
    try:
        cores, perm = T.partial_chain_pairs(x, y5, pairs)
        caught = np.abs(T.chain_to_dense(cores, perm) - want).max() > 1e-6
    except (ValueError, AssertionError):
        caught = True  # the unswapped ranks no longer chain
    assert caught


def test_tt_svd_pin_catches_a_dropped_direction(monkeypatch):
    rng = np.random.default_rng(9)
    x = rng.standard_normal((4, 5, 3))
    assert np.abs(O.tt_to_dense(O.tt_svd(x)) - x).max() < 1e-12
    monkeypatch.setattr(T, "tt_svd", _svd_keep_one_too_few)
    assert np.abs(T.tt_to_dense(T.tt_svd(x)) - x).max() > 1e-3


def _transfer_pairs_swapped(gx, gy):
    """The pair index taken as b R^x + a on the right only."""
    rx, _, rx2 = gx.shape
    ry, _, ry2 = gy.shape
    return np.einsum("aiu,biv->abvu", gx, gy).reshape(rx * ry, rx2 * ry2)


def _transfer_drop_last_slice(gx, gy):
    rx, _, rx2 = gx.shape
    ry, _, ry2 = gy.shape
    return np.einsum("aiu,biv->abuv", gx[:, :-1], gy[:, :-1]).reshape(rx * ry, rx2 * ry2)


@pytest.mark.parametrize("mutant", [_transfer_pairs_swapped, _transfer_drop_last_slice])
def test_factored_pin_catches_transfer_mutants(mutant, monkeypatch):
    x, y = G.pair(15, [2, 3, 2, 3, 2], [1, 2, 3, 2, 2, 1], [1, 3, 2, 2, 2, 1], np.float64)
    mask = [0, 1, 1, 0, 1]
    want = O.tcp(O.tt_to_dense(x), O.tt_to_dense(y), [1, 2, 4])
    f, runs = O.partial_factored(x, y, mask)
    assert np.abs(O.factored_to_dense(x, y, f, runs) - want).max() < 1e-13
    monkeypatch.setattr(T, "transfer_matrix", mutant)
    f, runs = T.partial_factored(x, y, mask)
    assert np.abs(T.factored_to_dense(x, y, f, runs) - want).max() > 1e-6


def _round_without_orthogonalising(cores, eps=0.0):
    """Truncation from the left without the right-orthonormal sweep first."""
    cores = [np.array(c, dtype=np.float64) for c in cores]
    n = len(cores)
    nrm = math.sqrt(T.contract_full(cores, cores))
    tol = eps * nrm / np.sqrt(n - 1)
    for k in range(n - 1):
        r0, i_dim, r1 = cores[k].shape
        u, sv, vt = np.linalg.svd(cores[k].reshape(r0 * i_dim, r1), full_matrices=False)
        dropped = np.sqrt(np.cumsum(sv[::-1] ** 2))[::-1]
        keep = len(sv)
        while keep > 1 and dropped[keep - 1] <= tol:
            keep -= 1
        cores[k] = u[:, :keep].reshape(r0, i_dim, keep)
        cores[k + 1] = np.einsum("ab,bic->aic", sv[:keep, None] * vt[:keep], cores[k + 1])
    return cores


def test_round_pin_catches_missing_orthogonalisation(monkeypatch):
    """Without the right-orthonormal sweep the kept ranks are not the TT-SVD's
    (and the error bound can break): the rank pin sees it."""
    rng = np.random.default_rng(31)
    y = G.random_tt(rng, [4, 3, 5, 3, 4], [1, 4, 8, 7, 4, 1], np.float64)
    for c in y:
        c *= rng.uniform(0.2, 5.0)
    dy = O.tt_to_dense(y)
    eps = 0.2
    want = [c.shape[0] for c in O.reverse_tt(O.tt_svd(np.transpose(dy, (4, 3, 2, 1, 0)), eps))]
    assert [c.shape[0] for c in O.tt_round(y, eps)] == want
    monkeypatch.setattr(T, "tt_round", _round_without_orthogonalising)
    t = T.tt_round(y, eps)
    err = np.linalg.norm(T.tt_to_dense(t) - dy) / np.linalg.norm(dy)
    assert [c.shape[0] for c in t] != want or err > eps
