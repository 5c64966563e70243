"""Shared helpers for the test-suite (no oracle arithmetic here)."""
import numpy as np

import oracle as O


def to_dev(cores, dtype=None, device="cuda"):
    import torch

    out = []
    for c in cores:
        t = torch.from_numpy(np.ascontiguousarray(c))
        if dtype is not None:
            t = t.to(dtype)
        out.append(t.to(device).contiguous())
    return out


def to_host(cores):
    return [c.detach().cpu().double().numpy() for c in cores]


def norm_scale(x, y):
    """||X||_F ||Y||_F from the oracle's <X,X> and <Y,Y>."""
    return float(np.sqrt(O.contract_full(x, x) * O.contract_full(y, y)))


def cs_bound(xs, ys, side, s):
    """Per-entry Cauchy-Schwarz scale sqrt(Gx[a,a] Gy[b,b]) of the environment K
    over an end block (Gram environments of X and Y over the block)."""
    if side == "lead":
        gx = O.left_envs(xs[:s], xs[:s])[-1]
        gy = O.left_envs(ys[:s], ys[:s])[-1]
    else:
        n = len(xs)
        gx = O.right_envs(xs[n - s:], xs[n - s:])[0]
        gy = O.right_envs(ys[n - s:], ys[n - s:])[0]
    return np.sqrt(np.outer(np.diag(gx), np.diag(gy)))
