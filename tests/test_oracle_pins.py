"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test checks an oracle function against an independent statement of the
same quantity: brute force over explicit index loops, closed forms (rank-1 and
CP-structured TTs), invariants (norm, gauge, zero padding, symmetry,
linearity) and exact finite differences.  A plausible slip in the oracle (a
dropped term, a transposed operand, a wrong leg order) fails at least one of
them; ``test_oracle_mutants.py`` plants such slips and checks that.
"""
import itertools
from fractions import Fraction
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2109_00626_gb300 import inputs as G

HERE = os.path.dirname(os.path.abspath(__file__))


def _tt_entry(cores, idx):
    """X[i_1..i_N] = G1[:,i1,:] G2[:,i2,:] ... GN[:,iN,:] (the TT value, Eq. 9)."""
    m = np.ones((1, 1))
    for g, i in zip(cores, idx):
        m = m @ np.asarray(g, dtype=np.float64)[:, i, :]
    return m[0, 0]


def _dense_by_entries(cores):
    shape = tuple(g.shape[1] for g in cores)
    out = np.empty(shape)
    for idx in itertools.product(*[range(s) for s in shape]):
        out[idx] = _tt_entry(cores, idx)
    return out


def _rand_tt(rng, modes, ranks):
    return G.random_tt(rng, modes, ranks, np.float64)


SMALL_SHAPES = [
    ([8, 8, 8, 8], [1, 4, 4, 4, 1], [1, 4, 4, 4, 1]),
    ([3], [1, 1], [1, 1]),
    ([2, 5], [1, 3, 1], [1, 2, 1]),
    ([1, 4, 3], [1, 2, 3, 1], [1, 1, 4, 1]),
    ([3, 2, 4, 2, 3], [1, 2, 5, 3, 2, 1], [1, 3, 1, 4, 2, 1]),
]


@pytest.mark.parametrize("modes,rx,ry", SMALL_SHAPES)
def test_dense_reconstruction_entrywise(modes, rx, ry, rng):
    x = _rand_tt(rng, modes, rx)
    np.testing.assert_allclose(O.tt_to_dense(x), _dense_by_entries(x), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("modes,rx,ry", SMALL_SHAPES)
def test_full_contraction_brute_force(modes, rx, ry, rng):
    x = _rand_tt(rng, modes, rx)
    y = _rand_tt(rng, modes, ry)
    zx = _dense_by_entries(x)
    zy = _dense_by_entries(y)
    ref = math.fsum((zx * zy).ravel())
    z = O.contract_full(x, y)
    assert abs(z - ref) <= 1e-13 * np.linalg.norm(zx) * np.linalg.norm(zy)


def test_small_fp64_workload_brute_force():
    x, y = G.small_fp64(0)
    zx, zy = _dense_by_entries(x), _dense_by_entries(y)
    ref = math.fsum((zx * zy).ravel())
    assert abs(O.contract_full(x, y) - ref) <= 1e-14
    # partial over modes 3,4 (1-based): explicit loop over the contracted indices
    want = np.zeros((8, 8, 8, 8))
    for i3 in range(8):
        for i4 in range(8):
            want += np.einsum("ab,cd->abcd", zx[:, :, i3, i4], zy[:, :, i3, i4])
    cores, perm = O.partial_chain(x, y, [0, 0, 1, 1])
    assert [c.shape for c in cores] == [(1, 8, 4), (4, 8, 4), (4, 8, 4), (4, 8, 1)]
    np.testing.assert_allclose(O.chain_to_dense(cores, perm), want, rtol=0, atol=1e-15)


def test_tcp_against_loops(rng):
    x = rng.standard_normal((3, 4, 2))
    y = rng.standard_normal((3, 5, 2))
    z = O.tcp(x, y, [0, 2])
    want = np.zeros((4, 5))
    for a in range(4):
        for b in range(5):
            want[a, b] = sum(x[i, a, k] * y[i, b, k] for i in range(3) for k in range(2))
    np.testing.assert_allclose(z, want, rtol=1e-14, atol=1e-14)
    # Eq. 8 with different orders: X (2,3,4) x_2^1 Y (3,5) -> (2,4,5)
    x = rng.standard_normal((2, 3, 4))
    y = rng.standard_normal((3, 5))
    z = O.tcp_nm(x, y, 1, 0)
    want = np.zeros((2, 4, 5))
    for a, c, d in itertools.product(range(2), range(4), range(5)):
        want[a, c, d] = sum(x[a, i, c] * y[i, d] for i in range(3))
    np.testing.assert_allclose(z, want, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("n,i_dim", [(1, 5), (4, 8), (10, 16), (16, 32)])
def test_rank1_closed_form(n, i_dim, rng):
    xs = [rng.standard_normal(i_dim) for _ in range(n)]
    ys = [rng.standard_normal(i_dim) for _ in range(n)]
    want = math.prod(float(np.dot(a, b)) for a, b in zip(xs, ys))
    z = O.contract_full(G.rank1_tt(xs), G.rank1_tt(ys))
    assert abs(z - want) <= 1e-13 * abs(want)


def test_rank1_partial_closed_form(rng):
    n, i_dim = 5, 3
    xs = [rng.standard_normal(i_dim) for _ in range(n)]
    ys = [rng.standard_normal(i_dim) for _ in range(n)]
    for mask in ([1, 1, 0, 0, 0], [0, 0, 0, 1, 1], [0, 1, 0, 1, 0]):
        c = math.prod(float(np.dot(xs[k], ys[k])) for k in range(n) if mask[k])
        vecs = [xs[k] for k in range(n) if not mask[k]] + [ys[k] for k in range(n) if not mask[k]]
        want = c
        for v in vecs:
            want = np.multiply.outer(want, v)
        if O.end_block(mask) is not None:
            cores, perm = O.partial_chain(G.rank1_tt(xs), G.rank1_tt(ys), mask)
            np.testing.assert_allclose(O.chain_to_dense(cores, perm), want, rtol=1e-13, atol=1e-15)
        cores, perm = O.partial_merged(G.rank1_tt(xs), G.rank1_tt(ys), mask)
        np.testing.assert_allclose(O.merged_to_dense(cores, perm), want, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("n,i_dim,rx,ry", [(10, 16, 64, 64), (4, 32, 128, 96), (6, 8, 5, 7)])
def test_cp_structured_closed_form(n, i_dim, rx, ry, rng):
    ux = [rng.standard_normal((rx, i_dim)) / np.sqrt(i_dim) for _ in range(n)]
    uy = [rng.standard_normal((ry, i_dim)) / np.sqrt(i_dim) for _ in range(n)]
    # z = sum_{r,s} prod_k <u_k^r, v_k^s>
    want = np.ones((rx, ry))
    for k in range(n):
        want = want * (ux[k] @ uy[k].T)
    want_z = math.fsum(want.ravel())
    z = O.contract_full(G.cp_tt(ux), G.cp_tt(uy))
    scale = math.fsum(np.abs(want).ravel())
    assert abs(z - want_z) <= 1e-13 * scale


def _left_orthonormalise(cores):
    """QR sweep: every core but the last becomes left-orthonormal; X is unchanged."""
    cores = [np.array(c, dtype=np.float64) for c in cores]
    for k in range(len(cores) - 1):
        r0, i_dim, r1 = cores[k].shape
        q, r = np.linalg.qr(cores[k].reshape(r0 * i_dim, r1))
        cores[k] = q.reshape(r0, i_dim, q.shape[1])
        cores[k + 1] = np.tensordot(r, cores[k + 1], axes=([1], [0]))
    return cores


def test_norm_invariant_small(rng):
    x = _rand_tt(rng, [3, 4, 2, 5], [1, 3, 4, 2, 1])
    d = _dense_by_entries(x)
    assert abs(O.contract_full(x, x) - math.fsum((d * d).ravel())) <= 1e-14 * np.sum(d * d)


def test_norm_invariant_large():
    x, _ = G.order10_r64(0, np.float64)
    q = _left_orthonormalise(x)
    want = float(np.sum(q[-1] ** 2))
    assert abs(O.contract_full(x, x) - want) <= 1e-12 * want
    assert abs(O.contract_full(q, q) - want) <= 1e-12 * want


def test_example1_single_leading_mode(rng):
    """Example 1: with the contracted mode first, K = A_x^T A_y is one matrix product."""
    x = _rand_tt(rng, [6, 3, 4, 2], [1, 5, 2, 3, 1])
    y = _rand_tt(rng, [6, 3, 4, 2], [1, 4, 3, 2, 1])
    ax = x[0][0]  # (I_1, R_1)
    ay = y[0][0]
    k = O.left_envs(x[:1], y[:1])[-1]
    np.testing.assert_allclose(k, ax.T @ ay, rtol=1e-14, atol=1e-15)
    # and the chain built on it reproduces Eq. 8 for S = {1}
    cores, perm = O.partial_chain(x, y, [1, 0, 0, 0])
    want = O.tcp(_dense_by_entries(x), _dense_by_entries(y), [0])
    np.testing.assert_allclose(O.chain_to_dense(cores, perm), want, rtol=1e-12, atol=1e-14)


CHAIN_MASKS = [
    [1, 0, 0, 0, 0],
    [1, 1, 0, 0, 0],
    [1, 1, 1, 1, 0],
    [0, 0, 0, 0, 1],
    [0, 0, 1, 1, 1],
    [0, 1, 1, 1, 1],
    [0, 0, 0, 0, 0],
]


@pytest.mark.parametrize("mask", CHAIN_MASKS)
def test_partial_chain_vs_dense(mask, rng):
    modes = [3, 2, 4, 2, 3]
    x = _rand_tt(rng, modes, [1, 2, 5, 3, 2, 1])
    y = _rand_tt(rng, modes, [1, 3, 1, 4, 2, 1])
    cores, perm = O.partial_chain(x, y, mask)
    zx, zy = _dense_by_entries(x), _dense_by_entries(y)
    s = [k for k in range(5) if mask[k]]
    want = O.tcp(zx, zy, s)
    got = O.chain_to_dense(cores, perm)
    assert got.shape == want.shape
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14)
    # chain ranks join: consecutive legs agree, ends are 1
    assert cores[0].shape[0] == 1 and cores[-1].shape[2] == 1
    for a, b in zip(cores[:-1], cores[1:]):
        assert a.shape[2] == b.shape[0]


@pytest.mark.parametrize("mask", [[0, 1, 0, 1, 0], [1, 0, 1, 0, 1], [0, 1, 1, 0, 0], [1, 0, 0, 0, 1], [0, 0, 0, 0, 0], [1, 1, 0, 1, 1]])
def test_partial_merged_vs_dense(mask, rng):
    modes = [3, 2, 4, 2, 3]
    x = _rand_tt(rng, modes, [1, 2, 5, 3, 2, 1])
    y = _rand_tt(rng, modes, [1, 3, 1, 4, 2, 1])
    cores, perm = O.partial_merged(x, y, mask)
    zx, zy = _dense_by_entries(x), _dense_by_entries(y)
    want = O.tcp(zx, zy, [k for k in range(5) if mask[k]])
    np.testing.assert_allclose(O.merged_to_dense(cores, perm), want, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("mask", [[0, 1, 0, 1, 0], [1, 0, 1, 0, 1], [0, 0, 1, 1, 0], [1, 1, 0, 0, 0]])
def test_partial_merged_unequal_free_modes_vs_dense(mask, rng):
    """Free modes of X and Y of different sizes (equal on S)."""
    mx = [3, 2, 4, 2, 3]
    my = [m if mask[k] else m + 2 for k, m in enumerate(mx)]
    x = _rand_tt(rng, mx, [1, 2, 5, 3, 2, 1])
    y = _rand_tt(rng, my, [1, 3, 1, 4, 2, 1])
    cores, perm = O.partial_merged(x, y, mask)
    want = O.tcp(_dense_by_entries(x), _dense_by_entries(y), [k for k in range(5) if mask[k]])
    np.testing.assert_allclose(O.merged_to_dense(cores, perm), want, rtol=1e-12, atol=1e-14)


def test_chain_rejects_interior_and_all():
    x, y = G.small_fp64(0)
    with pytest.raises(ValueError):
        O.partial_chain(x, y, [0, 1, 1, 0])
    with pytest.raises(ValueError):
        O.partial_chain(x, y, [1, 1, 1, 1])
    with pytest.raises(ValueError):
        O.partial_merged(x, y, [1, 1, 1, 1])


def test_gauge_and_padding_invariance(rng):
    x, y = G.small_fp64(3)
    z = O.contract_full(x, y)
    q, _ = np.linalg.qr(rng.standard_normal((4, 4)))
    xg = [c.copy() for c in x]
    xg[1] = np.tensordot(xg[1], q, axes=([2], [0]))
    xg[2] = np.tensordot(q.T, xg[2], axes=([1], [0]))
    assert abs(O.contract_full(xg, y) - z) <= 1e-15
    # zero padding of bond 2 (4 -> 7)
    xp = [c.copy() for c in x]
    xp[1] = np.concatenate([xp[1], np.zeros((4, 8, 3))], axis=2)
    xp[2] = np.concatenate([xp[2], np.zeros((3, 8, 4))], axis=0)
    assert abs(O.contract_full(xp, y) - z) <= 1e-16
    cores, perm = O.partial_chain(xp, y, [0, 0, 1, 1])
    c0, p0 = O.partial_chain(x, y, [0, 0, 1, 1])
    np.testing.assert_allclose(O.chain_to_dense(cores, perm), O.chain_to_dense(c0, p0), atol=1e-16)


def test_symmetry_and_linearity(rng):
    x, y = G.small_fp64(5)
    z = O.contract_full(x, y)
    assert abs(O.contract_full(y, x) - z) <= 1e-17
    for k in range(4):
        xs = [c.copy() for c in x]
        xs[k] = xs[k] * -2.5
        assert abs(O.contract_full(xs, y) + 2.5 * z) <= 1e-16
    # swapping operands of a partial swaps the free blocks
    c1, p1 = O.partial_chain(x, y, [0, 0, 1, 1])
    c2, p2 = O.partial_chain(y, x, [0, 0, 1, 1])
    z1 = O.chain_to_dense(c1, p1)
    z2 = O.chain_to_dense(c2, p2)
    np.testing.assert_allclose(z1, np.transpose(z2, (2, 3, 0, 1)), atol=1e-16)


def _fd_grad(fun, cores, k, h=1.0):
    """Central differences; exact for functions linear in core k."""
    g = np.zeros_like(cores[k])
    for idx in np.ndindex(*cores[k].shape):
        cp = [c.copy() for c in cores]
        cm = [c.copy() for c in cores]
        cp[k][idx] += h
        cm[k][idx] -= h
        g[idx] = (fun(cp) - fun(cm)) / (2 * h)
    return g


def test_grad_full_fd_and_euler():
    # adjoint check size: order 5, mode 4, ranks 3, float64
    x, y = G.pair(7, [4] * 5, G.tt_ranks(5, 3), G.tt_ranks(5, 3), np.float64)
    z = O.contract_full(x, y)
    gx, gy = O.grad_full(x, y)
    for k in range(5):
        fx = _fd_grad(lambda c: O.contract_full(c, y), x, k)
        fy = _fd_grad(lambda c: O.contract_full(x, c), y, k)
        np.testing.assert_allclose(gx[k], fx, rtol=1e-10, atol=1e-14)
        np.testing.assert_allclose(gy[k], fy, rtol=1e-10, atol=1e-14)
        # Euler: z is linear in each core, so <G_k, dz/dG_k> = z
        assert abs(np.sum(gx[k] * x[k]) - z) <= 1e-14
        assert abs(np.sum(gy[k] * y[k]) - z) <= 1e-14


def test_grad_full_unit_cores(rng):
    """dz/dGx_k[a,i,a'] = <Y, X with core k replaced by the unit tensor e_{a,i,a'}>."""
    x = _rand_tt(rng, [2, 3, 2], [1, 2, 3, 1])
    y = _rand_tt(rng, [2, 3, 2], [1, 3, 2, 1])
    zy = _dense_by_entries(y)
    gx, _ = O.grad_full(x, y, cot=1.0)
    for k in range(3):
        want = np.zeros_like(x[k])
        for idx in np.ndindex(*x[k].shape):
            xe = [c.copy() for c in x]
            xe[k] = np.zeros_like(x[k])
            xe[k][idx] = 1.0
            want[idx] = np.sum(_dense_by_entries(xe) * zy)
        np.testing.assert_allclose(gx[k], want, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("mask", [[1, 1, 1, 0, 0], [0, 0, 1, 1, 1], [1, 0, 0, 0, 0], [0, 0, 0, 0, 1]])
def test_grad_partial_chain_fd(mask, rng):
    modes = [3, 2, 3, 2, 2]
    x = _rand_tt(rng, modes, [1, 2, 3, 3, 2, 1])
    y = _rand_tt(rng, modes, [1, 3, 2, 2, 3, 1])
    cores, perm = O.partial_chain(x, y, mask)
    w = rng.standard_normal(O.chain_to_dense(cores, perm).shape)

    def loss_of_z(zc):
        return float(np.sum(O.chain_to_dense(zc, perm) * w))

    def loss(xc, yc):
        zc, _ = O.partial_chain(xc, yc, mask)
        return loss_of_z(zc)

    dz = [_fd_grad(loss_of_z, cores, p) for p in range(len(cores))]
    gx, gy = O.grad_partial_chain(x, y, mask, dz)
    for k in range(5):
        fx = _fd_grad(lambda c: loss(c, y), x, k)
        fy = _fd_grad(lambda c: loss(x, c), y, k)
        np.testing.assert_allclose(gx[k], fx, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(gy[k], fy, rtol=1e-9, atol=1e-12)


def test_tt_svd_exact_and_truncated(rng):
    x = rng.standard_normal((4, 5, 3, 6))
    cores = O.tt_svd(x, 0.0)
    np.testing.assert_allclose(O.tt_to_dense(cores), x, rtol=0, atol=1e-12)
    # untruncated ranks are min(prod of left dims, prod of right dims)
    assert [c.shape[0] for c in cores] == [1, 4, 18, 6]
    # the accuracy guarantee: ||X - TT(X)||_F <= eps ||X||_F
    for eps in (0.05, 0.3, 0.7):
        t = O.tt_svd(x, eps)
        err = np.linalg.norm(O.tt_to_dense(t) - x)
        assert err <= eps * np.linalg.norm(x) * (1 + 1e-12)
    # truncation really happens: a larger eps never gives larger ranks
    r_small = [c.shape[2] for c in O.tt_svd(x, 0.05)]
    r_large = [c.shape[2] for c in O.tt_svd(x, 0.7)]
    assert all(a >= b for a, b in zip(r_small, r_large)) and r_small != r_large
    # a TT of known low rank is found exactly, with its ranks
    low = _rand_tt(rng, [5, 6, 7], [1, 2, 3, 1])
    t = O.tt_svd(O.tt_to_dense(low), 1e-10)
    assert [c.shape[2] for c in t] == [2, 3, 1]
    np.testing.assert_allclose(O.tt_to_dense(t), O.tt_to_dense(low), rtol=0, atol=1e-12)
    # order 1 and a mode of size 1
    v = rng.standard_normal(7)
    np.testing.assert_allclose(O.tt_to_dense(O.tt_svd(v)), v, rtol=0, atol=0)
    w = rng.standard_normal((3, 1, 4))
    np.testing.assert_allclose(O.tt_to_dense(O.tt_svd(w)), w, rtol=0, atol=1e-13)


def test_tt_svd_taken_left_to_right(rng):
    """The decomposition taken from the left (the order the GPU kernel uses)
    is the oracle's right-to-left one on the reversed axes, reversed back:
    it reconstructs the tensor within eps ||X||, its first rank is the one
    the SVD of the first unfolding I_1 x rest gives for the threshold
    eps ||X|| / sqrt(N - 1), and its cores 0 .. N-2 are left-orthonormal."""
    x = rng.standard_normal((6, 5, 4, 3))
    n = x.ndim
    for eps in (0.0, 0.1, 0.4):
        t = O.reverse_tt(O.tt_svd(np.transpose(x, tuple(range(n - 1, -1, -1))), eps))
        assert np.linalg.norm(O.tt_to_dense(t) - x) <= eps * np.linalg.norm(x) * (1 + 1e-12) + 1e-12
        sv = np.linalg.svd(x.reshape(6, -1), compute_uv=False)
        tol = eps * np.linalg.norm(x) / np.sqrt(n - 1)
        tails = np.sqrt(np.cumsum(sv[::-1] ** 2))[::-1]  # tails[r] = ||sv[r:]||
        r1 = next((r for r in range(1, len(sv)) if tails[r] <= tol), len(sv))
        assert t[0].shape[2] == r1
        for g in t[:-1]:
            m = g.reshape(-1, g.shape[2])
            np.testing.assert_allclose(m.T @ m, np.eye(m.shape[1]), rtol=0, atol=1e-12)


def test_reverse_tt_reverses_modes(rng):
    x = _rand_tt(rng, [3, 4, 2, 5], [1, 2, 3, 4, 1])
    d = O.tt_to_dense(x)
    np.testing.assert_allclose(O.tt_to_dense(O.reverse_tt(x)), np.transpose(d, (3, 2, 1, 0)), rtol=0, atol=1e-14)


def test_tcp_pairs_by_index_loops(rng):
    x = rng.standard_normal((2, 3, 4))
    y = rng.standard_normal((4, 5, 2))
    got = O.tcp_pairs(x, y, [(2, 0), (0, 2)])  # free: x mode 1, y mode 1
    want = np.zeros((3, 5))
    for i1 in range(3):
        for j1 in range(5):
            for a in range(2):
                for b in range(4):
                    want[i1, j1] += x[a, i1, b] * y[b, j1, a]
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(O.tcp_pairs(x, y, [(2, 0)]), O.tcp_nm(x, y, 2, 0), rtol=0, atol=0)


PAIR_CASES = [
    # orders, pairs
    (4, 3, [(0, 0)]),
    (4, 3, [(0, 0), (1, 1)]),
    (3, 5, [(2, 4), (1, 3)]),        # trailing block of X with trailing block of Y
    (5, 3, [(0, 2), (1, 1)]),        # leading block of X against trailing block of Y
    (3, 4, [(2, 0), (1, 1)]),        # trailing block of X against leading block of Y
    (2, 4, [(0, 0), (1, 1)]),        # X fully contracted: Y keeps two free modes
    (4, 2, [(3, 1), (2, 0)]),        # Y fully contracted
    (1, 3, [(0, 2)]),
]


@pytest.mark.parametrize("nx,ny,pairs", PAIR_CASES)
def test_partial_chain_pairs_against_dense(rng, nx, ny, pairs):
    """Different orders and end-block pairings: the chain TT (un-permuted by
    perm) equals Eq. 8 on the dense tensors."""
    mx = [int(v) for v in rng.integers(2, 4, size=nx)]
    my = [int(v) for v in rng.integers(2, 4, size=ny)]
    for a, b in pairs:
        my[b] = mx[a]
    x = _rand_tt(rng, mx, [1] + [int(v) for v in rng.integers(1, 4, size=nx - 1)] + [1])
    y = _rand_tt(rng, my, [1] + [int(v) for v in rng.integers(1, 4, size=ny - 1)] + [1])
    cores, perm = O.partial_chain_pairs(x, y, pairs)
    assert sorted(perm) == list(range(nx + ny - 2 * len(pairs)))
    want = O.tcp_pairs(O.tt_to_dense(x), O.tt_to_dense(y), pairs)
    np.testing.assert_allclose(O.chain_to_dense(cores, perm), want, rtol=1e-12, atol=1e-12)


def test_partial_chain_pairs_rejects_non_end_blocks(rng):
    x = _rand_tt(rng, [2, 2, 2, 2], [1, 2, 2, 2, 1])
    y = _rand_tt(rng, [2, 2, 2], [1, 2, 2, 1])
    for pairs in ([(1, 0)], [(0, 0), (1, 2)], [(0, 1), (1, 0)], [(0, 0), (1, 1), (2, 2), (3, 0)]):
        with pytest.raises(ValueError):
            O.partial_chain_pairs(x, y, pairs)
    with pytest.raises(ValueError):
        O.partial_chain_pairs(x[:3], y, [(0, 0), (1, 1), (2, 2)])


def test_partial_chain_pairs_same_order_equals_partial_chain(rng):
    x = _rand_tt(rng, [3, 2, 4, 3], [1, 2, 3, 2, 1])
    y = _rand_tt(rng, [3, 2, 4, 3], [1, 3, 2, 2, 1])
    for mask, pairs in (([1, 1, 0, 0], [(0, 0), (1, 1)]), ([0, 0, 1, 1], [(3, 3), (2, 2)])):
        c1, p1 = O.partial_chain(x, y, mask)
        c2, p2 = O.partial_chain_pairs(x, y, pairs)
        np.testing.assert_allclose(O.chain_to_dense(c1, p1), O.chain_to_dense(c2, p2), rtol=1e-13, atol=1e-13)


def _ttcp_dense(x, y, n, m, eps=0.0):
    """Dense operands: move the paired modes to the front, decompose both
    with tt_svd, contract the TTs over their first modes, and return Z in
    Eq. 8 order together with the chain cores (Z^rho)."""
    xt = O.tt_svd(np.moveaxis(x, n, 0), eps)
    yt = O.tt_svd(np.moveaxis(y, m, 0), eps)
    cores, perm = O.partial_chain_pairs(xt, yt, [(0, 0)])
    # perm refers to the moved operands' free modes, which keep their order
    return O.chain_to_dense(cores, perm), cores


def test_example1_dense_operands_of_different_order(rng):
    """Example 1: X (order 4) x_3^2 Y (order 3); Z^rho is I4 x I2 x I1 x J1 x J3."""
    x = rng.standard_normal((2, 3, 4, 5))
    y = rng.standard_normal((6, 4, 3))
    z, cores = _ttcp_dense(x, y, 2, 1)
    np.testing.assert_allclose(z, O.tcp_nm(x, y, 2, 1), rtol=1e-10, atol=1e-11)
    assert tuple(c.shape[1] for c in cores) == (5, 3, 2, 6, 3)
    assert z.shape == (2, 3, 5, 6, 3)


def test_example2_first_modes_dense_operands(rng):
    """Example 2's contraction X x_1^1 Y on Gaussian tensors (reduced sizes),
    exact TTs and eps-truncated ones (error within the truncation bound)."""
    for dims in ((6, 6, 6), (6, 6, 6, 3), (5, 5, 5, 3, 2)):
        x = rng.standard_normal(dims)
        y = rng.standard_normal(dims)
        want = O.tcp_nm(x, y, 0, 0)
        z, _ = _ttcp_dense(x, y, 0, 0)
        np.testing.assert_allclose(z, want, rtol=1e-9, atol=1e-10)
        eps = 0.2
        zt, _ = _ttcp_dense(x, y, 0, 0, eps)
        # ||Z - Z~|| <= ||X - X~|| ||Y|| + ||X~|| ||Y - Y~|| <= (2 eps + eps^2) ||X|| ||Y||
        bound = (2 * eps + eps**2) * np.linalg.norm(x) * np.linalg.norm(y)
        assert np.linalg.norm(zt - want) <= bound


def test_paper_operation_counts():
    gold = json.load(open(os.path.join(HERE, "golden", "complexity.json")))
    assert math.log10(O.tcp_ops(10, 5)) == gold["tcp_order5_i10_ops_order_of_magnitude"]
    assert float(O.tcp_ops(1000, 5)) == gold["tcp_order5_i1000_ops"]
    assert O.ttcp_ops(1000, 5) == gold["ttcp_i1000_r5_ops"]
    assert O.ttcp_ops(1000, 2) == gold["ttcp_i1000_r2_ops"]
    assert math.floor(math.log10(O.tcp_ops(1000, 5) / O.ttcp_ops(1000, 5))) == gold["reduction_i1000_n5_r5_log10_approx"]


def test_generator_norm_expectation():
    """The input recipe sigma = 1/sqrt(I R_right) gives E||X||_F^2 = 1."""
    vals = []
    for s in range(400):
        x = G.random_tt(np.random.default_rng(s), [4, 4, 4], [1, 3, 3, 1])
        vals.append(O.contract_full(x, x))
    assert abs(np.mean(vals) - 1.0) < 0.1


# ---- compensated accumulation (reference values under cancellation) ----

U64 = 2.0**-53


def _fr(v):
    return Fraction(float(v))


def _exact_full(x, y):
    """<X, Y> in exact rational arithmetic from the TT entries (Eq. 9)."""
    shape = tuple(g.shape[1] for g in x)
    total = Fraction(0)
    for idx in itertools.product(*[range(s) for s in shape]):
        vx = [[Fraction(1)]]
        vy = [[Fraction(1)]]
        for gx, gy, i in zip(x, y, idx):
            sx = [[_fr(gx[a, i, b]) for b in range(gx.shape[2])] for a in range(gx.shape[0])]
            sy = [[_fr(gy[a, i, b]) for b in range(gy.shape[2])] for a in range(gy.shape[0])]
            vx = [[sum(vx[0][a] * sx[a][b] for a in range(len(sx))) for b in range(len(sx[0]))]]
            vy = [[sum(vy[0][a] * sy[a][b] for a in range(len(sy))) for b in range(len(sy[0]))]]
        total += vx[0][0] * vy[0][0]
    return total


def _tt_sum(a, b):
    """The TT of the entrywise sum A + B (ranks added: first cores side by side,
    interior cores block-diagonal, last cores stacked)."""
    n = len(a)
    out = []
    for k, (ga, gb) in enumerate(zip(a, b)):
        ra0, i_dim, ra1 = ga.shape
        rb0, _, rb1 = gb.shape
        r0 = 1 if k == 0 else ra0 + rb0
        r1 = 1 if k == n - 1 else ra1 + rb1
        g = np.zeros((r0, i_dim, r1))
        oa0, ob0 = 0, (0 if k == 0 else ra0)
        oa1, ob1 = 0, (0 if k == n - 1 else ra1)
        g[oa0:oa0 + ra0, :, oa1:oa1 + ra1] = ga
        g[ob0:ob0 + rb0, :, ob1:ob1 + rb1] = gb
        out.append(g)
    return out


def test_error_free_transformations_are_exact(rng):
    a = rng.standard_normal(300) * 2.0 ** rng.integers(-60, 61, 300)
    b = rng.standard_normal(300) * 2.0 ** rng.integers(-60, 61, 300)
    s, e = O.two_sum(a, b)
    p, f = O.two_product(a, b)
    for k in range(300):
        assert _fr(s[k]) + _fr(e[k]) == _fr(a[k]) + _fr(b[k])
        assert _fr(p[k]) + _fr(f[k]) == _fr(a[k]) * _fr(b[k])
        assert s[k] == a[k] + b[k] and p[k] == a[k] * b[k]


@pytest.mark.parametrize("n", [1, 2, 7, 64])
def test_dot2_within_its_bound(n, rng):
    """|hi + lo - x.y| <= 2 gamma_n^2 sum |x_k y_k| against exact rationals, on
    plain vectors and on vectors whose products cancel to a small remainder
    (where a plain float64 dot product errs by about u sum |x_k y_k|)."""
    x = rng.standard_normal(n)
    y = rng.standard_normal(n)
    cases = [(x, y), (np.concatenate([x, x, [1e-3]]), np.concatenate([y, -y, [1.0]]))]
    for u, v in cases:
        m = len(u)
        exact = sum((_fr(a) * _fr(b) for a, b in zip(u, v)), Fraction(0))
        hi, lo = O.dot2_dd(u, v)
        gamma = m * U64 / (1 - m * U64)
        bound = 2 * gamma**2 * float(np.sum(np.abs(u * v)))
        assert abs(float(_fr(hi) + _fr(lo) - exact)) <= bound
        assert hi == float(hi + lo)  # a normalised pair


def test_contract_full_dd_exact_to_rounding(rng):
    for modes, rx, ry in [([3, 2, 3], [1, 2, 3, 1], [1, 3, 2, 1]), ([2, 2, 2, 2], [1, 2, 2, 2, 1], [1, 2, 3, 2, 1])]:
        x = _rand_tt(rng, modes, rx)
        y = _rand_tt(rng, modes, ry)
        exact = _exact_full(x, y)
        assert abs(O.contract_full_dd(x, y) - float(exact)) <= U64 * abs(float(exact))


def test_contract_full_dd_under_cancellation(rng):
    """Y = X + X'' where X'' is X with its first core scaled by -(1 + 2^-30): Y's
    entries cancel to about 2^-30 of its parts, and the plain sweep loses about
    30 bits; the compensated sweep stays within one rounding of the exact value."""
    x = _rand_tt(rng, [3, 2, 3], [1, 2, 3, 1])
    w = [c.copy() for c in x]
    w[0] = w[0] * -(1 + 2.0**-30)
    y = _tt_sum(x, w)
    exact = float(_exact_full(x, y))
    assert abs(O.contract_full_dd(x, y) - exact) <= 2 * U64 * abs(exact)
    assert abs(O.contract_full(x, y) - exact) > 1e3 * U64 * abs(exact)  # the case does need compensation


@pytest.mark.parametrize("mask", [[1, 0, 1, 1, 0], [0, 1, 0, 1, 0], [1, 1, 0, 0, 1], [0, 0, 0, 0, 0],
                                  [1, 1, 1, 1, 0], [0, 1, 1, 1, 1], [1, 0, 0, 0, 1]])
def test_factored_form_against_brute_force(mask):
    """The factored form multiplied out equals Eq. 8 computed entry by entry
    on the dense tensors, for interior, end, alternating and empty sets; and
    it agrees with the merged layout's cores (the same Z)."""
    rng = np.random.default_rng(sum(v << k for k, v in enumerate(mask)) + 3)
    x = _rand_tt(rng, [3, 2, 3, 2, 2], [1, 2, 3, 2, 2, 1])
    y = _rand_tt(rng, [3, 2, 3, 2, 2], [1, 3, 2, 2, 3, 1])
    dx, dy = O.tt_to_dense(x), O.tt_to_dense(y)
    sset = [k for k in range(5) if mask[k]]
    free = [k for k in range(5) if not mask[k]]
    want = np.zeros([dx.shape[k] for k in free] + [dy.shape[k] for k in free])
    for idx in itertools.product(*[range(dx.shape[k]) for k in free]):
        for jdx in itertools.product(*[range(dy.shape[k]) for k in free]):
            tot = 0.0
            for sdx in itertools.product(*[range(dx.shape[k]) for k in sset]):
                ix, iy = [0] * 5, [0] * 5
                for k, v in zip(free, idx):
                    ix[k] = v
                for k, v in zip(free, jdx):
                    iy[k] = v
                for k, v in zip(sset, sdx):
                    ix[k] = iy[k] = v
                tot += dx[tuple(ix)] * dy[tuple(iy)]
            want[idx + jdx] = tot
    f, runs = O.partial_factored(x, y, mask)
    assert f == free and len(runs) == len(free) + 1
    np.testing.assert_allclose(O.factored_to_dense(x, y, f, runs), want, rtol=0, atol=1e-13)
    cores, perm = O.partial_merged(x, y, mask)
    np.testing.assert_allclose(O.merged_to_dense(cores, perm), want, rtol=0, atol=1e-13)


def test_transfer_matrix_entries_and_runs(rng):
    """A mode's transfer matrix entry by entry (sum over the shared index of
    one X entry times one Y entry, pair index a R^y + b); a run's matrix is
    the product, so row (a, b) is the run swept from e_a e_b^T; the left and
    right environments are its end rows and columns."""
    gx = rng.standard_normal((2, 3, 4))
    gy = rng.standard_normal((3, 3, 2))
    t = O.transfer_matrix(gx, gy)
    for a, b, u, v in itertools.product(range(2), range(3), range(4), range(2)):
        assert abs(t[a * 3 + b, u * 2 + v] - sum(gx[a, i, u] * gy[b, i, v] for i in range(3))) < 1e-14
    x = _rand_tt(rng, [2, 3, 2, 3], [1, 2, 3, 2, 1])
    y = _rand_tt(rng, [2, 3, 2, 3], [1, 3, 2, 2, 1])
    f, runs = O.partial_factored(x, y, [0, 1, 1, 0])
    e = np.zeros((2, 3))
    e[1, 2] = 1.0
    row = O.absorb_left(O.absorb_left(e, x[1], y[1]), x[2], y[2]).ravel()
    np.testing.assert_allclose(runs[1][1 * 3 + 2], row, rtol=0, atol=1e-14)
    assert runs[0] is None and runs[2] is None
    f, runs = O.partial_factored(x, y, [1, 0, 1, 1])
    np.testing.assert_allclose(runs[0].ravel(), O.left_envs(x[:1], y[:1])[-1].ravel(), rtol=0, atol=1e-14)
    assert len(runs) == 2
    np.testing.assert_allclose(runs[1].ravel(), O.right_envs(x[2:], y[2:])[0].ravel(), rtol=0, atol=1e-14)


def _tt_sum(a, b):
    """The TT of A + B: block-diagonal interior cores (ranks add)."""
    n = len(a)
    out = []
    for k, (ga, gb) in enumerate(zip(a, b)):
        ra, i_dim, ra2 = ga.shape
        rb, _, rb2 = gb.shape
        if n == 1:
            out.append(ga + gb)
        elif k == 0:
            out.append(np.concatenate([ga, gb], axis=2))
        elif k == n - 1:
            out.append(np.concatenate([ga, gb], axis=0))
        else:
            g = np.zeros((ra + rb, i_dim, ra2 + rb2))
            g[:ra, :, :ra2] = ga
            g[ra:, :, ra2:] = gb
            out.append(g)
    return out


def test_tt_round_recovers_ranks_and_bounds_the_error(rng):
    """Rounding X + X (ranks doubled, the tensor 2X of the original ranks)
    recovers the original ranks with eps ~ 0 and the same tensor; on a random
    TT the error stays within eps ||X||_F; the cores come out left-orthonormal
    except the last; and the ranks equal those of the TT-SVD of the dense
    tensor taken left to right at the same eps (the same singular values),
    unless a threshold lies within 1e-6 of a tail of them."""
    x = _rand_tt(rng, [4, 3, 5, 3, 4], [1, 3, 4, 4, 2, 1])
    d = O.tt_to_dense(x)
    r = O.tt_round(_tt_sum(x, x), 1e-12)
    assert [c.shape[0] for c in r] + [1] == [1, 3, 4, 4, 2, 1]
    np.testing.assert_allclose(O.tt_to_dense(r), 2 * d, rtol=0, atol=1e-12 * np.abs(d).max())
    y = _rand_tt(rng, [4, 3, 5, 3, 4], [1, 4, 8, 7, 4, 1])
    dy = O.tt_to_dense(y)
    for eps in (0.02, 0.2, 0.5):
        t = O.tt_round(y, eps)
        assert np.linalg.norm(O.tt_to_dense(t) - dy) <= eps * np.linalg.norm(dy) * (1 + 1e-12)
        for g in t[:-1]:
            m = g.reshape(-1, g.shape[2])
            np.testing.assert_allclose(m.T @ m, np.eye(m.shape[1]), rtol=0, atol=1e-12)
        ltr = O.reverse_tt(O.tt_svd(np.transpose(dy, (4, 3, 2, 1, 0)), eps))
        near = False
        tol = eps * np.linalg.norm(dy) / 2.0
        for k in range(4):
            sv = np.linalg.svd(dy.reshape(int(np.prod(dy.shape[: k + 1])), -1), compute_uv=False)
            tails = np.sqrt(np.cumsum(sv[::-1] ** 2))[::-1]
            near |= bool(np.min(np.abs(tails - tol)) <= 1e-6 * tol)
        if not near:
            assert [c.shape[0] for c in t] == [c.shape[0] for c in ltr]
