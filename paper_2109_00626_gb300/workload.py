"""Algorithmic work of a contraction (the cost model used for GFLOP/s and
roofline fractions; it is not part of the compute path).

flops of one contracted mode with core ranks (Rx -> Rx', Ry -> Ry') and mode
size I: the cheaper of the two evaluation orders of E' = sum_i A_i^T E B_i,
  2 * min(Rx Ry I Ry' + Rx I Rx' Ry',  Rx Ry I Rx' + Ry I Rx' Ry').
Section IV of the paper counts only K = A_x^T A_y (I R_1 P_1 multiply-adds for
one leading mode); over several modes each extra mode costs the above.
bytes: every core read once in its storage type, outputs written once; the
environment stays on chip and is not counted.
"""
from __future__ import annotations


def mode_flops(rx, rx2, ry, ry2, i_dim):
    a = rx * ry * i_dim * ry2 + rx * i_dim * rx2 * ry2
    b = rx * ry * i_dim * rx2 + ry * i_dim * rx2 * ry2
    return 2 * min(a, b)


def core_elems(modes, ranks):
    return sum(ranks[k] * modes[k] * ranks[k + 1] for k in range(len(modes)))


def full_flops(modes, rx, ry):
    return sum(mode_flops(rx[k], rx[k + 1], ry[k], ry[k + 1], modes[k]) for k in range(len(modes)))


def full_bytes(modes, rx, ry, elem_bytes):
    return (core_elems(modes, rx) + core_elems(modes, ry)) * elem_bytes


def end_block(mask):
    n = len(mask)
    s = sum(1 for v in mask if v)
    if all(bool(mask[k]) == (k < s) for k in range(n)):
        return "lead", s
    if all(bool(mask[k]) == (k >= n - s) for k in range(n)):
        return "trail", s
    return None, s


def partial_chain_flops(modes, rx, ry, mask):
    """Sweep over the contracted block plus the join of K into the boundary core."""
    side, s = end_block(mask)
    n = len(modes)
    ks = [k for k in range(n) if mask[k]]
    f = sum(mode_flops(rx[k], rx[k + 1], ry[k], ry[k + 1], modes[k]) for k in ks)
    if side == "lead":
        f += 2 * rx[s] * modes[s] * rx[s + 1] * ry[s]
    else:
        m = n - s
        f += 2 * rx[m - 1] * modes[m - 1] * rx[m] * ry[m]
    return f


def partial_chain_bytes(modes, rx, ry, mask, elem_bytes):
    """Contracted cores read once; free cores read and written once; C written."""
    side, s = end_block(mask)
    n = len(modes)
    rd = 0
    wr = 0
    for k in range(n):
        ex = rx[k] * modes[k] * rx[k + 1]
        ey = ry[k] * modes[k] * ry[k + 1]
        rd += ex + ey
        if not mask[k]:
            wr += ey
            kb = s if side == "lead" else n - s - 1
            if k == kb:
                wr += (rx[k + 1] if side == "lead" else rx[k]) * modes[k] * ry[k if side == "lead" else k + 1]
            else:
                wr += ex
    return (rd + wr) * elem_bytes


def factored_flops(modes, rx, ry, mask):
    """Work of the factored form over S: each environment run is one sweep;
    an interior run between free positions is swept once from every basis
    environment e_a e_b^T of its left pair rank (its first mode from a unit
    environment costs I R^x' R^y' multiply-adds)."""
    n = len(modes)
    free = [k for k in range(n) if not mask[k]]
    tot = 0
    for t in range(len(free) + 1):
        k0 = 0 if t == 0 else free[t - 1] + 1
        k1 = n if t == len(free) else free[t]
        if k1 <= k0:
            continue
        if t == 0 or t == len(free):
            tot += sum(mode_flops(rx[k], rx[k + 1], ry[k], ry[k + 1], modes[k]) for k in range(k0, k1))
            continue
        rows = rx[k0] * ry[k0]
        per = 2 * modes[k0] * rx[k0 + 1] * ry[k0 + 1]
        per += sum(mode_flops(rx[k], rx[k + 1], ry[k], ry[k + 1], modes[k]) for k in range(k0 + 1, k1))
        tot += rows * per
    return tot
