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


def dense_cs_scale(x, y, contracted):
    """Per-entry Cauchy-Schwarz scale of Eq. 8's Z over the contracted
    positions: |Z[i_F, j_F]| <= ||X[:, i_F]|| ||Y[:, j_F]||, the norms over the
    contracted indices (the entrywise form of the error measure of a partial
    contraction).  Shape and axis order of Z (X's free modes, then Y's)."""
    xd = O.tt_to_dense(x)
    yd = O.tt_to_dense(y)
    ax = tuple(contracted)
    gx = np.sqrt(np.sum(xd * xd, axis=ax)) if ax else np.abs(xd)
    gy = np.sqrt(np.sum(yd * yd, axis=ax)) if ax else np.abs(yd)
    return np.multiply.outer(gx, gy)


def dense_cs_eps(got, want, x, y, contracted):
    """max |Z - Z*| / (the per-entry Cauchy-Schwarz scale) over all entries."""
    scale = dense_cs_scale(x, y, contracted)
    return float(np.max(np.abs(np.asarray(got) - np.asarray(want)) / np.maximum(scale, 1e-300)))


def grad_cs_scale(x, y):
    """Per-entry Cauchy-Schwarz scale of the gradients of z = <X, Y>:
    dz/dGx_k[a, i, a'] = <X with core k replaced by the unit e_(a,i,a'), Y>, so
    |dz/dGx_k[a, i, a']| <= sqrt(Lx_k[a, a] Rx_{k+1}[a', a']) ||Y||, with Lx / Rx
    the Gram environments of X (and the mirror for Y).  Returns the scale
    arrays for every core of X, then of Y (shapes of the cores)."""
    lx, rx = O.left_envs(x, x), O.right_envs(x, x)
    ly, ry = O.left_envs(y, y), O.right_envs(y, y)
    nx = np.sqrt(max(O.contract_full(x, x), 0.0))
    ny = np.sqrt(max(O.contract_full(y, y), 0.0))
    out_x, out_y = [], []
    for k in range(len(x)):
        sx = np.sqrt(np.outer(np.diag(lx[k]), np.diag(rx[k + 1]))) * ny
        sy = np.sqrt(np.outer(np.diag(ly[k]), np.diag(ry[k + 1]))) * nx
        out_x.append(np.broadcast_to(sx[:, None, :], x[k].shape))
        out_y.append(np.broadcast_to(sy[:, None, :], y[k].shape))
    return out_x + out_y


def grad_cs_eps(got, want, scales):
    """max over every core entry of |g - g*| / its Cauchy-Schwarz scale."""
    return max(float(np.max(np.abs(g - w) / np.maximum(s, 1e-300))) for g, w, s in zip(got, want, scales))
