"""CPU oracle for tensor-train contraction (Kisil et al., arXiv 2109.00626).

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct float64
reference that the CUDA library is checked against.  Only the test-suite, the
smoke check and the benchmark's CPU-baseline leg may import it; the library
itself never calls it and has no CPU fallback.

Every function works on plain numpy float64 arrays and cites the passage of the
paper it restates.  Library primitives (matmul, einsum, svd) serve as single
steps; nothing is blocked, fused or reordered beyond the definitions.

Conventions
-----------
* A TT of order N is a list of cores, core k shaped (R_k, I_k, R_{k+1}) with
  R_0 = R_N = 1 (0-based bond index; the paper's G^(k) in R^{R_{k-1} x I_k x R_k},
  Def. 7 / Eq. 9 and the rank conditions of Example 1).  Row-major storage:
  the right rank is fastest.  (The paper's little-endian unfolding of Eq. 2 is
  not used; all reshapes here are row-major, stated where they occur.)
* Contracted set S: position k of X is contracted with position k of Y.  The
  paper contracts one mode pair (Eq. 8); several pairs are contracted one
  after the other, which gives the same result in any order because the sums
  are over distinct indices.
* Output mode order of a partial contraction follows Eq. 8: the free modes of
  X ascending, then the free modes of Y ascending.  A layout whose modes come
  in another order carries ``perm`` with Z_rho = Z.transpose(perm), i.e. axis p
  of the emitted TT is axis perm[p] of Eq. 8's Z (the re-ordering of Step 6 of
  Algorithm 2, kept as a relabelling in line with Remark 2).

Functions
---------
tt_to_dense            Eq. 9
tcp / tcp_nm           Eq. 8 (set of same-position pairs / one (n, m) pair)
absorb_left            one contracted mode folded into the left environment
                       (Example 1's K = A_x^T A_y generalised, Algorithm 2 step 4)
absorb_right           the mirror image, right environment
contract_full          all modes contracted -> scalar (Fig. 1b's full contraction)
two_sum / two_product / dot2_dd / absorb_left_dd / contract_full_dd
                       the same sweep with compensated (double-double)
                       accumulation, for reference values under cancellation
partial_chain          end-block S -> chain TT (Algorithm 2 steps 4-6)
partial_merged         any S -> TT-matrix of merged cores
chain_to_dense / merged_to_dense   dense reconstruction + un-permutation
transfer_matrix / partial_factored / factored_to_dense
                       any S in factored form: the contracted runs as
                       matrices over pair indices, the free cores as the
                       Kronecker factors of the merged cores (Eq. 8)
grad_sweep / grad_full / grad_partial_chain   gradients by the L/F formulas
tt_svd                 a TT of a dense tensor within eps ||X||_F (Section II)
tt_round               a TT re-expressed with truncated ranks within eps ||X||_F
reverse_tt             the same TT with its modes in reverse order
tcp_pairs              Eq. 8 over several (n, m) pairs, operands of any orders
partial_chain_pairs    end-block pairs of TTs of different orders -> chain TT
tcp_ops / ttcp_ops     the operation counts of Section IV and Remark 3

Parity status: every function here is pinned by a test in tests/ that does not
re-use its formula (brute force, closed forms, invariants or finite
differences); none is "parity unpinned".
"""
from __future__ import annotations

import string

import numpy as np

__all__ = [
    "tt_to_dense",
    "tcp",
    "tcp_nm",
    "absorb_left",
    "absorb_right",
    "left_envs",
    "right_envs",
    "contract_full",
    "two_sum",
    "two_product",
    "dot2_dd",
    "absorb_left_dd",
    "contract_full_dd",
    "end_block",
    "partial_chain",
    "partial_merged",
    "chain_to_dense",
    "merged_to_dense",
    "transfer_matrix",
    "partial_factored",
    "factored_to_dense",
    "tt_round",
    "grad_sweep",
    "grad_full",
    "grad_partial_chain",
    "tt_svd",
    "reverse_tt",
    "tcp_pairs",
    "partial_chain_pairs",
    "tcp_ops",
    "ttcp_ops",
]


def _f64(cores):
    return [np.asarray(c, dtype=np.float64) for c in cores]


# --------------------------------------------------------------------------
# Dense semantics
# --------------------------------------------------------------------------
def tt_to_dense(cores):
    """Eq. 9: X = G^(1) x_2^1 G^(2) x_3^1 ... x_3^1 G^(N).

    Each step contracts the last (rank) mode of the running tensor with the
    first (rank) mode of the next core, one TCP of Eq. 8 at a time.
    """
    cores = _f64(cores)
    z = cores[0].reshape(cores[0].shape[1], cores[0].shape[2])  # R_0 = 1
    for g in cores[1:]:
        z = np.tensordot(z, g, axes=([z.ndim - 1], [0]))
    return z.reshape(z.shape[:-1])  # R_N = 1


def tcp(x, y, contracted):
    """Eq. 8 for several same-position pairs: Z = sum over i_S of X[..] Y[..].

    ``contracted`` lists 0-based positions k; position k of X is summed
    against position k of Y.  Result axes: free modes of X ascending, then
    free modes of Y ascending (Eq. 8's ordering).
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = x.ndim
    assert y.ndim == n
    letters = string.ascii_letters
    xs = [letters[k] for k in range(n)]
    ys = [letters[k] if k in contracted else letters[n + k] for k in range(n)]
    out = [xs[k] for k in range(n) if k not in contracted] + [ys[k] for k in range(n) if k not in contracted]
    return np.einsum("".join(xs) + "," + "".join(ys) + "->" + "".join(out), x, y)


def tcp_nm(x, y, n, m):
    """Eq. 8 literally: the (n, m)-contraction of tensors of any orders (0-based n, m)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    assert x.shape[n] == y.shape[m]
    letters = string.ascii_letters
    xs = [letters[k] for k in range(x.ndim)]
    ys = [letters[x.ndim + k] for k in range(y.ndim)]
    ys[m] = xs[n]
    out = [xs[k] for k in range(x.ndim) if k != n] + [ys[k] for k in range(y.ndim) if k != m]
    return np.einsum("".join(xs) + "," + "".join(ys) + "->" + "".join(out), x, y)


# --------------------------------------------------------------------------
# Environment sweep (Algorithm 2 step 4, generalised to many modes)
# --------------------------------------------------------------------------
def absorb_left(e, gx, gy):
    """E'[a',b'] = sum_{a,b,i} E[a,b] Gx[a,i,a'] Gy[b,i,b'].

    With E = [[1]] and one mode this is Example 1's K = A_x^T A_y.  Written as
    a sum over the mode index i of Gx[:,i,:]^T E Gy[:,i,:].
    """
    gx = np.asarray(gx, dtype=np.float64)
    gy = np.asarray(gy, dtype=np.float64)
    assert gx.shape[1] == gy.shape[1]
    out = np.zeros((gx.shape[2], gy.shape[2]))
    for i in range(gx.shape[1]):
        out += gx[:, i, :].T @ e @ gy[:, i, :]
    return out


def absorb_right(f, gx, gy):
    """F[a,b] = sum_{a',b',i} Gx[a,i,a'] F'[a',b'] Gy[b,i,b'] (mirror of absorb_left)."""
    gx = np.asarray(gx, dtype=np.float64)
    gy = np.asarray(gy, dtype=np.float64)
    assert gx.shape[1] == gy.shape[1]
    out = np.zeros((gx.shape[0], gy.shape[0]))
    for i in range(gx.shape[1]):
        out += gx[:, i, :] @ f @ gy[:, i, :].T
    return out


def left_envs(xc, yc, start=None):
    """L_0 = start (default [[1]]), L_{k+1} = absorb_left(L_k, Gx_k, Gy_k); returns L_0..L_N."""
    xc, yc = _f64(xc), _f64(yc)
    e = np.ones((1, 1)) if start is None else np.asarray(start, dtype=np.float64)
    envs = [e]
    for gx, gy in zip(xc, yc):
        e = absorb_left(e, gx, gy)
        envs.append(e)
    return envs


def right_envs(xc, yc, end=None):
    """F_N = end (default [[1]]), F_k = absorb_right(F_{k+1}, Gx_k, Gy_k); returns F_0..F_N."""
    xc, yc = _f64(xc), _f64(yc)
    f = np.ones((1, 1)) if end is None else np.asarray(end, dtype=np.float64)
    envs = [f]
    for gx, gy in zip(reversed(xc), reversed(yc)):
        f = absorb_right(f, gx, gy)
        envs.append(f)
    return envs[::-1]


def contract_full(xc, yc):
    """<X, Y>: every position contracted (Fig. 1b's all-mode contraction to a scalar)."""
    assert len(xc) == len(yc)
    return float(left_envs(xc, yc)[-1][0, 0])


# --------------------------------------------------------------------------
# Compensated accumulation for reference values (Ogita, Rump and Oishi,
# "Accurate Sum and Dot Product", SIAM J. Sci. Comput. 26(6), 2005): the
# error-free transformations of a sum (Knuth's TwoSum) and of a product
# (Dekker's TwoProduct with Veltkamp's splitting), and their Dot2, a dot
# product as accurate as one computed in twice the working precision.  The
# arithmetic is elementwise numpy float64, which rounds every operation to
# nearest and never fuses a multiply with an add (the transformations rely on
# both).  The sweep below carries each environment as an unevaluated pair
# hi + lo, so that no intermediate rounding is left uncompensated.
# --------------------------------------------------------------------------
_VELTKAMP = 134217729.0  # 2^27 + 1


def two_sum(a, b):
    """(s, e) with s = fl(a + b) and s + e = a + b exactly (Knuth)."""
    s = a + b
    z = s - a
    e = (a - (s - z)) + (b - z)
    return s, e


def _split(a):
    """(hi, lo) with a = hi + lo exactly, each of at most 26 significant bits (Veltkamp)."""
    c = _VELTKAMP * a
    hi = c - (c - a)
    return hi, a - hi


def two_product(a, b):
    """(p, e) with p = fl(a * b) and p + e = a * b exactly (Dekker)."""
    p = a * b
    a1, a2 = _split(a)
    b1, b2 = _split(b)
    e = a2 * b2 - (((p - a1 * b1) - a2 * b1) - a1 * b2)
    return p, e


def dot2_dd(x, y):
    """Dot2 over the last axis (vectorised over the leading ones), returned
    unrounded as a pair (hi, lo): the running sum p is kept with the exact
    errors of every product and every addition, those errors are summed in a
    second accumulator s, and hi + lo = p + s exactly.  The error of hi + lo
    against the exact dot product is at most gamma_n^2 sum |x_k y_k| (plus the
    rounding of s), gamma_n = n u / (1 - n u)."""
    x, y = np.broadcast_arrays(np.asarray(x, dtype=np.float64), np.asarray(y, dtype=np.float64))
    p, s = two_product(x[..., 0], y[..., 0])
    for k in range(1, x.shape[-1]):
        h, r = two_product(x[..., k], y[..., k])
        p, q = two_sum(p, h)
        s = s + (q + r)
    return two_sum(p, s)


def absorb_left_dd(ehi, elo, gx, gy):
    """absorb_left on an environment held as E = ehi + elo, in two Dot2 stages
    that keep their results as pairs:
        T[a][i][b'] = sum_b E[a,b] Gy[b,i,b']         (2 R^y terms: hi and lo)
        E'[a',b']   = sum_{a,i} Gx[a,i,a'] T[a,i,b']  (2 R^x I terms)
    Returns (E'hi, E'lo)."""
    gx = np.asarray(gx, dtype=np.float64)
    gy = np.asarray(gy, dtype=np.float64)
    assert gx.shape[1] == gy.shape[1]
    rx, i_dim, rx2 = gx.shape
    ry2 = gy.shape[2]
    e2 = np.concatenate([ehi, elo], axis=1)                      # [a][b | b]
    gyy = np.concatenate([gy, gy], axis=0).transpose(1, 2, 0)    # [i][b'][b | b]
    thi, tlo = dot2_dd(e2[:, None, None, :], gyy[None, :, :, :])  # [a][i][b']
    t2 = np.concatenate([thi.reshape(rx * i_dim, ry2), tlo.reshape(rx * i_dim, ry2)], axis=0)  # [(a,i) | (a,i)][b']
    gxx = np.concatenate([gx.reshape(rx * i_dim, rx2)] * 2, axis=0)                           # [(a,i) | (a,i)][a']
    return dot2_dd(gxx.T[:, None, :], t2.T[None, :, :])           # [a'][b']


def contract_full_dd(xc, yc):
    """<X, Y> by the left-to-right sweep with double-double environments
    (absorb_left_dd); returns the float64 nearest to the final pair."""
    assert len(xc) == len(yc)
    xc, yc = _f64(xc), _f64(yc)
    ehi, elo = np.ones((1, 1)), np.zeros((1, 1))
    for gx, gy in zip(xc, yc):
        ehi, elo = absorb_left_dd(ehi, elo, gx, gy)
    return float(ehi[0, 0] + elo[0, 0])


# --------------------------------------------------------------------------
# Partial contraction, chain layout (Algorithm 2 steps 4-6)
# --------------------------------------------------------------------------
def end_block(mask):
    """Classify a contracted set: ("lead", s) if S = {0..s-1}, ("trail", s) if
    S = {N-s..N-1}, else None.  The empty set counts as leading."""
    n = len(mask)
    s = int(sum(1 for v in mask if v))
    if all(bool(mask[k]) == (k < s) for k in range(n)):
        return ("lead", s)
    if all(bool(mask[k]) == (k >= n - s) for k in range(n)):
        return ("trail", s)
    return None


def _swap_rank_legs(g):
    """The paper's (.)^{T[1;3]}: exchange the first and third modes of a core."""
    return np.ascontiguousarray(np.transpose(g, (2, 1, 0)))


def partial_chain(xc, yc, mask):
    """Partial contraction over an end block S, returned as one TT (chain layout).

    Leading S = {0..s-1} (the case of Algorithm 2 after its step-1 permutation):
      K = L_s, the left environment over S (step 4 generalised);
      C[a',i,b] = sum_a Gx_s[a,i,a'] K[a,b];
      cores = Gx_{N-1}^T, ..., Gx_{s+1}^T, C, Gy_s, ..., Gy_{N-1}   (step 5,
      X's cores walked backwards with their rank legs exchanged);
      perm: axis p < m is X-free mode m-1-p, axis m+q is Y-free mode q.
    Trailing S = {m..N-1}, m = N - s (the mirror image):
      K = F_m, the right environment over S;
      C[a,i,b] = sum_{a'} Gx_{m-1}[a,i,a'] K[a',b];
      cores = Gx_0, ..., Gx_{m-2}, C, Gy_{m-1}^T, ..., Gy_0^T;
      perm: axis p < m is X-free mode p, axis m+q is Y-free mode m-1-q.
    Returns (cores, perm) with Z_rho = Z.transpose(perm) (step 6 as a relabelling).
    """
    xc, yc = _f64(xc), _f64(yc)
    n = len(xc)
    blk = end_block(mask)
    if blk is None:
        raise ValueError("chain layout needs the contracted modes to form a leading or trailing block")
    side, s = blk
    if s == n:
        raise ValueError("all modes contracted: use contract_full")
    m = n - s
    if side == "lead":
        k = left_envs(xc[:s], yc[:s])[-1]
        gx = xc[s]
        c = np.einsum("aiu,ab->uib", gx, k)
        cores = [_swap_rank_legs(xc[j]) for j in range(n - 1, s, -1)] + [c] + [yc[j].copy() for j in range(s, n)]
        perm = [m - 1 - p for p in range(m)] + [m + q for q in range(m)]
    else:
        k = right_envs(xc[m:], yc[m:])[0]
        gx = xc[m - 1]
        c = np.einsum("aiu,ub->aib", gx, k)
        cores = [xc[j].copy() for j in range(m - 1)] + [c] + [_swap_rank_legs(yc[j]) for j in range(m - 1, -1, -1)]
        perm = list(range(m)) + [m + (m - 1 - q) for q in range(m)]
    return cores, perm


def chain_to_dense(cores, perm):
    """Dense Z in Eq. 8 order from a chain-layout TT and its perm."""
    zr = tt_to_dense(cores)
    return np.transpose(zr, np.argsort(perm))


# --------------------------------------------------------------------------
# Partial contraction, merged (TT-matrix) layout, any S
# --------------------------------------------------------------------------
def partial_merged(xc, yc, mask):
    """Partial contraction over any S as a TT over the free positions.

    Free positions f_0 < ... < f_{m-1}.  Core t is the Kronecker pair
      W_t[(a,b), i, j, (a',b')] = Gx_{f_t}[a,i,a'] Gy_{f_t}[b,j,b']
    (pair index a*R^y + b).  The left environment of the contracted modes
    before f_0 is absorbed on the left of W_0; the contracted modes between f_t
    and f_{t+1} (and after f_{m-1}) are absorbed on the right of W_t by running
    the left-environment step on every row (r, i, j) of W_t.  Core t is returned
    shaped (r_t, I_{f_t}, J_{f_t}, r_{t+1}); axes of the represented tensor
    interleave (i_{f_0}, j_{f_0}, i_{f_1}, j_{f_1}, ...), so perm[2t] = t and
    perm[2t+1] = m + t.
    """
    xc, yc = _f64(xc), _f64(yc)
    n = len(xc)
    free = [k for k in range(n) if not mask[k]]
    if not free:
        raise ValueError("all modes contracted: use contract_full")
    m = len(free)
    el = left_envs(xc[: free[0]], yc[: free[0]])[-1]
    cores = []
    for t, f in enumerate(free):
        gx, gy = xc[f], yc[f]
        rx, i_dim, rx2 = gx.shape
        ry, j_dim, ry2 = gy.shape
        w = np.einsum("aiu,bjv->abijuv", gx, gy).reshape(rx * ry, i_dim, j_dim, rx2, ry2)
        if t == 0:
            w = np.einsum("ab,abijuv->ijuv", el, w.reshape(rx, ry, i_dim, j_dim, rx2, ry2))[None]
        nxt = free[t + 1] if t + 1 < m else n
        run = range(f + 1, nxt)
        rows = w.reshape(-1, rx2, ry2)
        out_rows = []
        for e in rows:
            for k in run:
                e = absorb_left(e, xc[k], yc[k])
            out_rows.append(e.reshape(-1))
        r_left = w.shape[0]
        w = np.stack(out_rows).reshape(r_left, i_dim, j_dim, -1)
        cores.append(w)
    perm = []
    for t in range(m):
        perm += [t, m + t]
    return cores, perm


def merged_to_dense(cores, perm):
    """Dense Z in Eq. 8 order from merged cores (r, I, J, r')."""
    acc = None
    dims = []
    for w in cores:
        r, i_dim, j_dim, r2 = w.shape
        dims += [i_dim, j_dim]
        g = np.asarray(w, dtype=np.float64).reshape(r, i_dim * j_dim, r2)
        acc = g.reshape(i_dim * j_dim, r2) if acc is None else np.tensordot(acc, g, axes=([acc.ndim - 1], [0]))
    zr = acc.reshape(dims)
    return np.transpose(zr, np.argsort(perm))


def transfer_matrix(gx, gy):
    """One contracted mode as a matrix over pair indices (a R^y + b):
    T[(a,b), (a',b')] = sum_i Gx[a,i,a'] Gy[b,i,b'] (Eq. 8's sum over the
    shared index, written for every left pair (a,b) at once)."""
    gx, gy = np.asarray(gx, dtype=np.float64), np.asarray(gy, dtype=np.float64)
    rx, _, rx2 = gx.shape
    ry, _, ry2 = gy.shape
    return np.einsum("aiu,biv->abuv", gx, gy).reshape(rx * ry, rx2 * ry2)


def partial_factored(xc, yc, mask):
    """Partial contraction over any S in factored form.

    With free positions f_0 < ... < f_{m-1},
      Z[i_F; j_F] = T_0 W_{f_0}[i_0, j_0] T_1 ... W_{f_{m-1}} T_m,
      W_f[i, j][(a,b), (a',b')] = Gx_f[a,i,a'] Gy_f[b,j,b'],
    T_t the product of the transfer matrices of the contracted modes between
    free positions (T_0 a 1 x R^xR^y row: the modes before f_0 starting from
    the rank-1 end; T_m a column: the modes after f_{m-1}); None for a run
    with no mode (the identity).  Returns (free positions, [T_0 .. T_m])."""
    xc, yc = _f64(xc), _f64(yc)
    n = len(xc)
    free = [k for k in range(n) if not mask[k]]
    if not free:
        raise ValueError("all modes contracted: use contract_full")
    m = len(free)
    runs = []
    for t in range(m + 1):
        k0 = 0 if t == 0 else free[t - 1] + 1
        k1 = n if t == m else free[t]
        if k1 <= k0:
            runs.append(None)
            continue
        acc = transfer_matrix(xc[k0], yc[k0])
        for k in range(k0 + 1, k1):
            acc = acc @ transfer_matrix(xc[k], yc[k])
        runs.append(acc)
    return free, runs


def factored_to_dense(xc, yc, free, runs):
    """Dense Z in Eq. 8 order (X's free modes, then Y's) from the factored
    form: the chain T_0 W_{f_0} T_1 ... T_m multiplied out."""
    xc, yc = _f64(xc), _f64(yc)
    m = len(free)
    acc = np.ones((1, 1))  # rows: (i_0, j_0, ..., i_{t-1}, j_{t-1}); columns: the pair index
    dims = []
    for t, f in enumerate(free):
        if runs[t] is not None:
            acc = acc @ runs[t]
        gx, gy = xc[f], yc[f]
        rx, i_dim, rx2 = gx.shape
        ry, j_dim, ry2 = gy.shape
        w = np.einsum("aiu,bjv->abijuv", gx, gy).reshape(rx * ry, i_dim * j_dim * rx2 * ry2)
        acc = (acc @ w).reshape(-1, rx2 * ry2)
        dims += [i_dim, j_dim]
    if runs[m] is not None:
        acc = acc @ runs[m]
    zr = acc.reshape(dims)
    order = [2 * t for t in range(m)] + [2 * t + 1 for t in range(m)]
    return np.transpose(zr, order)


# --------------------------------------------------------------------------
# Gradients
# --------------------------------------------------------------------------
def grad_sweep(xc, yc, start=None, end=None):
    """Gradients of z = <start | sweep over all modes | end> w.r.t. every core.

    With L_k the left environments from ``start`` and F_k the right ones from
    ``end``, z is linear in each core and
      dz/dGx_k[:, i, :] = L_k Gy_k[:, i, :] F_{k+1}^T,
      dz/dGy_k[:, i, :] = L_k^T Gx_k[:, i, :] F_{k+1}.
    """
    xc, yc = _f64(xc), _f64(yc)
    le = left_envs(xc, yc, start)
    fe = right_envs(xc, yc, end)
    gx_out, gy_out = [], []
    for k, (gx, gy) in enumerate(zip(xc, yc)):
        dgx = np.zeros_like(gx)
        dgy = np.zeros_like(gy)
        for i in range(gx.shape[1]):
            dgx[:, i, :] = le[k] @ gy[:, i, :] @ fe[k + 1].T
            dgy[:, i, :] = le[k].T @ gx[:, i, :] @ fe[k + 1]
        gx_out.append(dgx)
        gy_out.append(dgy)
    return gx_out, gy_out


def grad_full(xc, yc, cot=1.0):
    """d(cot * <X,Y>)/dG for every core of X and Y."""
    gx, gy = grad_sweep(xc, yc)
    return [cot * g for g in gx], [cot * g for g in gy]


def grad_partial_chain(xc, yc, mask, dz):
    """Back-propagate cotangents ``dz`` of the chain-layout cores to X and Y.

    The emitted cores are copies (or leg-swapped copies) of free cores, plus C,
    which is bilinear in the boundary core and K; K is the environment over S,
    so its cotangent dK seeds ``grad_sweep`` on the contracted block.
    """
    xc, yc = _f64(xc), _f64(yc)
    dz = _f64(dz)
    n = len(xc)
    side, s = end_block(mask)
    m = n - s
    gx = [np.zeros_like(g) for g in xc]
    gy = [np.zeros_like(g) for g in yc]
    if side == "lead":
        k = left_envs(xc[:s], yc[:s])[-1]
        for p, j in enumerate(range(n - 1, s, -1)):
            gx[j] = _swap_rank_legs(dz[p])
        dc = dz[m - 1]  # C[a',i,b] = sum_a Gx_s[a,i,a'] K[a,b]
        gx[s] = np.einsum("ab,uib->aiu", k, dc)
        dk = np.einsum("aiu,uib->ab", xc[s], dc)
        for q, j in enumerate(range(s, n)):
            gy[j] = dz[m + q].copy()
        if s > 0:
            sx, sy = grad_sweep(xc[:s], yc[:s], None, dk)
            gx[:s], gy[:s] = sx, sy
    else:
        k = right_envs(xc[m:], yc[m:])[0]
        for j in range(m - 1):
            gx[j] = dz[j].copy()
        dc = dz[m - 1]  # C[a,i,b] = sum_u Gx_{m-1}[a,i,u] K[u,b]
        gx[m - 1] = np.einsum("aib,ub->aiu", dc, k)
        dk = np.einsum("aiu,aib->ub", xc[m - 1], dc)
        for q, j in enumerate(range(m - 1, -1, -1)):
            gy[j] = _swap_rank_legs(dz[m + q])
        sx, sy = grad_sweep(xc[m:], yc[m:], dk, None)
        gx[m:], gy[m:] = sx, sy
    return gx, gy


# --------------------------------------------------------------------------
# TT decomposition of a dense tensor (Section II, TT-SVD) and contractions
# of TTs of different orders over pairs of end modes (Eq. 8 with (n, m) pairs)
# --------------------------------------------------------------------------
def tt_svd(x, eps=0.0):
    """A TT of the dense tensor x whose reconstruction error is at most
    eps * ||x||_F (the accuracy guarantee of the paper's TT-SVD, Section II).

    Built from the right: the part of x not yet factored is a matrix
    (left modes) x (I_k R_{k+1}); its SVD U S V^T gives core k = the leading
    rows of V^T (right-orthonormal) and the rest U S carries on to the next
    mode to the left.  Each SVD drops the largest set of trailing singular
    values whose 2-norm is at most eps ||x||_F / sqrt(N-1); the N-1 dropped
    parts are orthogonal, so the total error is at most eps ||x||_F.
    """
    x = np.asarray(x, dtype=np.float64)
    dims = x.shape
    n = len(dims)
    if n == 1:
        return [x.reshape(1, dims[0], 1).copy()]
    tol = eps * np.linalg.norm(x) / np.sqrt(n - 1)
    rest = x.reshape(-1, 1)  # (I_0 ... I_{N-1}) x R_N with R_N = 1
    right_rank = 1
    cores = [None] * n
    for k in range(n - 1, 0, -1):
        mat = rest.reshape(-1, dims[k] * right_rank)
        u, sv, vt = np.linalg.svd(mat, full_matrices=False)
        # keep r values: the smallest r with ||sv[r:]|| <= tol (at least one)
        dropped = np.sqrt(np.cumsum(sv[::-1] ** 2))[::-1]  # dropped[r] = ||sv[r:]||
        keep = len(sv)
        while keep > 1 and dropped[keep - 1] <= tol:
            keep -= 1
        cores[k] = vt[:keep].reshape(keep, dims[k], right_rank)
        rest = u[:, :keep] * sv[:keep]
        right_rank = keep
    cores[0] = rest.reshape(1, dims[0], right_rank)
    return cores


def tt_round(cores, eps=0.0):
    """TT rounding: the tensor the TT represents, re-expressed with ranks
    chosen by the TT-SVD's truncation rule (Section II) so that the result is
    within eps ||X||_F.

    First the cores are made right-orthonormal from the right: core k's
    transposed unfolding (I_k R_{k+1}) x R_k = Q R (QR), core k becomes Q^T and
    R^T is multiplied into core k-1; then ||X||_F = ||G_0||_F.  Then from the
    left each core's unfolding (R_k I_k) x R_{k+1} = U S V^T keeps the
    smallest rank r >= 1 whose dropped singular values have 2-norm
    <= eps ||X||_F / sqrt(N - 1); the core becomes U's r columns and the r rows
    of S V^T are multiplied into core k+1.  The parts dropped at the N-1 steps
    are orthogonal, so the total error is at most eps ||X||_F."""
    cores = [np.array(c, dtype=np.float64) for c in cores]
    n = len(cores)
    for k in range(n - 1, 0, -1):
        r0, i_dim, r1 = cores[k].shape
        q, r = np.linalg.qr(cores[k].reshape(r0, i_dim * r1).T)
        cores[k] = q.T.reshape(-1, i_dim, r1)
        cores[k - 1] = np.einsum("aib,cb->aic", cores[k - 1], r)
    if n == 1:
        return cores
    tol = eps * np.linalg.norm(cores[0]) / np.sqrt(n - 1)
    for k in range(n - 1):
        r0, i_dim, r1 = cores[k].shape
        u, sv, vt = np.linalg.svd(cores[k].reshape(r0 * i_dim, r1), full_matrices=False)
        dropped = np.sqrt(np.cumsum(sv[::-1] ** 2))[::-1]  # dropped[r] = ||sv[r:]||
        keep = len(sv)
        while keep > 1 and dropped[keep - 1] <= tol:
            keep -= 1
        cores[k] = u[:, :keep].reshape(r0, i_dim, keep)
        cores[k + 1] = np.einsum("ab,bic->aic", sv[:keep, None] * vt[:keep], cores[k + 1])
    return cores


def reverse_tt(cores):
    """The same tensor with its modes in reverse order: the cores taken last
    to first, each with its rank legs exchanged (the paper's (.)^{T[1;3]})."""
    return [_swap_rank_legs(np.asarray(g, dtype=np.float64)) for g in reversed(cores)]


def tcp_pairs(x, y, pairs):
    """Eq. 8 over several (n, m) pairs for dense tensors of any orders: mode
    pairs[t][0] of x is summed against mode pairs[t][1] of y.  Result axes:
    the free modes of x ascending, then the free modes of y ascending."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    letters = string.ascii_letters
    xs = [letters[k] for k in range(x.ndim)]
    ys = [letters[x.ndim + k] for k in range(y.ndim)]
    for n, m in pairs:
        assert x.shape[n] == y.shape[m]
        ys[m] = xs[n]
    cx = {n for n, _ in pairs}
    cy = {m for _, m in pairs}
    out = [xs[k] for k in range(x.ndim) if k not in cx] + [ys[k] for k in range(y.ndim) if k not in cy]
    return np.einsum("".join(xs) + "," + "".join(ys) + "->" + "".join(out), x, y)


def _end_walks(modes, order):
    """The ways the positions `modes` form an end block of a TT of the given
    order: (positions listed from the end of the train inward, whether the
    block is the trailing one).  A block covering the whole train has both."""
    s = len(modes)
    ms = sorted(modes)
    walks = []
    if ms == list(range(s)):
        walks.append((list(range(s)), False))
    if ms == list(range(order - s, order)):
        walks.append((list(range(order - 1, order - 1 - s, -1)), True))
    return walks


def partial_chain_pairs(xc, yc, pairs):
    """Partial contraction of TTs of orders N and M over the mode pairs
    (n_t, m_t) (Eq. 8 applied to each pair), as one chain TT.

    The n_t form a block at one end of X and the m_t a block at one end of Y,
    paired in the order in which the two blocks are met walking from the ends
    of the trains inward (e.g. Example 1's single pair, or X's modes 0, 1
    against Y's modes M-1, M-2).  An operand whose block is the trailing one
    is reversed first (reverse_tt), so both blocks lead; then
      K = the left environment over the s pairs,
      C[a', i, b] = sum_a X'_s[a, i, a'] K[a, b]       (N > s), or
      C[a, j, b'] = sum_b K[a, b] Y'_s[b, j, b']       (N = s, a of size 1),
      cores = X'_{N-1}^T, ..., X'_{s+1}^T, C, Y'_s, ..., Y'_{M-1}
    (when X has no free mode, the C of the second form takes Y'_s's place).
    Returns (cores, perm): axis p of the chain TT is axis perm[p] of Eq. 8's Z
    (free modes of X ascending, then free modes of Y ascending).
    """
    xc, yc = _f64(xc), _f64(yc)
    n_x, n_y = len(xc), len(yc)
    pairs = [(int(a), int(b)) for a, b in pairs]
    s = len(pairs)
    pair_of = dict(pairs)
    found = None
    if s > 0 and len(pair_of) == s:
        for walk_x, rev_x in _end_walks([a for a, _ in pairs], n_x):
            for walk_y, rev_y in _end_walks([b for _, b in pairs], n_y):
                if found is None and [pair_of[a] for a in walk_x] == walk_y:
                    found = (rev_x, rev_y)
    if found is None:
        raise ValueError("the paired modes must form an end block of each operand, met in the same order from the ends")
    rev_x, rev_y = found
    if s == n_x and s == n_y:
        raise ValueError("every mode contracted: use contract_full")
    xr = reverse_tt(xc) if rev_x else xc
    yr = reverse_tt(yc) if rev_y else yc
    # original mode index of position j of the (possibly reversed) operand
    ox = [(n_x - 1 - j) if rev_x else j for j in range(n_x)]
    oy = [(n_y - 1 - j) if rev_y else j for j in range(n_y)]
    k = left_envs(xr[:s], yr[:s])[-1]
    x_free = [j for j in range(n_x) if j >= s]
    y_free = [j for j in range(n_y) if j >= s]
    if x_free:
        c = np.einsum("aiu,ab->uib", xr[s], k)
        cores = [_swap_rank_legs(xr[j]) for j in range(n_x - 1, s, -1)] + [c] + [yr[j].copy() for j in y_free]
    else:
        c = np.einsum("ab,bjv->ajv", k, yr[s])
        cores = [c] + [yr[j].copy() for j in y_free[1:]]
    axes_x = [ox[j] for j in reversed(x_free)]
    axes_y = [oy[j] for j in y_free]
    fx = sorted(ox[j] for j in x_free)
    fy = sorted(oy[j] for j in y_free)
    perm = [fx.index(a) for a in axes_x] + [len(fx) + fy.index(b) for b in axes_y]
    return cores, perm


# --------------------------------------------------------------------------
# Operation counts of Section IV
# --------------------------------------------------------------------------
def tcp_ops(i_dim, order):
    """Standard TCP of two order-N tensors with all modes I: I^(2N-1) (Section IV)."""
    return i_dim ** (2 * order - 1)


def ttcp_ops(i_dim, rank):
    """TTCP cost of one contracted mode at the front: K = A_x^T A_y, I R_1 P_1 with R_1 = P_1 = R."""
    return i_dim * rank * rank
