"""Seeded synthetic tensor-train inputs.

This module only *draws* inputs; it holds none of the contraction arithmetic, so
both the CPU oracle and the CUDA path can be fed from it without sharing any of
the method.  Everything is numpy on the host; the caller moves arrays to the
device.

Conventions (tensor-train format, Def. 7 / Eq. 9 of the paper):
  * a TT of order N is a list of N cores, core k shaped (R_{k-1}, I_k, R_k),
    C-contiguous, right rank fastest; R_0 = R_N = 1 (Example 1).
  * cores are i.i.d. N(0, sigma^2) with sigma = 1 / sqrt(I_k * R_k), so that
    E ||X||_F^2 = 1 (the Gaussian workload of Example 2, rescaled).

Workloads (names give their sizes):
  * ``small_fp64``     order 4, I=8, ranks (1,4,4,4,1), float64
  * ``order10_r64``    order 10, I=16, internal ranks 64, float32
  * ``batch4096``      4096 pairs: order U{4..12}, I_k U{2..32} shared by the
                       pair, ranks U{4..128} per bond and per operand, float32;
                       even pairs full, odd pairs partial over an end block of
                       floor(N/2) modes (leading or trailing by a coin).  Its
                       15 GB of cores are drawn on the device
                       (:func:`batch4096_device`); :func:`batch_pair` draws
                       host cores of the same shapes for small tests.
  * ``order16_r256``   order 16, I=32, internal ranks 256, log-normal core
                       scales exp(N(0,1)); float32 master copy (BF16 forms
                       round it)
  * ``order12_r64``    order 12, I=16, ranks 64, float32 (adjoint workload)
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "tt_ranks",
    "random_tt",
    "rank1_tt",
    "cp_tt",
    "pair",
    "small_fp64",
    "order10_r64",
    "order16_r256",
    "order12_r64",
    "batch4096_spec",
    "batch_pair",
    "to_bf16_f32",
    "batch4096_device",
]


def tt_ranks(order: int, r: int) -> list[int]:
    """Bond ranks (1, r, ..., r, 1) for an order-``order`` TT."""
    return [1] + [r] * (order - 1) + [1]


def random_tt(rng: np.random.Generator, modes, ranks, dtype=np.float64, log_scale_sigma: float = 0.0):
    """Gaussian TT cores, core k ~ N(0, 1/(I_k R_k)) elementwise.

    With ``log_scale_sigma`` > 0 every core is also multiplied by exp(N(0, s^2))
    (one scalar per core) to spread the magnitudes of intermediate results.
    """
    modes = [int(m) for m in modes]
    ranks = [int(r) for r in ranks]
    assert len(ranks) == len(modes) + 1 and ranks[0] == 1 and ranks[-1] == 1
    cores = []
    for k, I in enumerate(modes):
        shape = (ranks[k], I, ranks[k + 1])
        sigma = 1.0 / np.sqrt(I * ranks[k + 1])
        g = rng.standard_normal(shape) * sigma
        if log_scale_sigma > 0.0:
            g = g * np.exp(rng.standard_normal() * log_scale_sigma)
        cores.append(np.ascontiguousarray(g.astype(dtype)))
    return cores


def rank1_tt(vectors, dtype=np.float64):
    """TT with all ranks 1 whose k-th core holds the vector ``vectors[k]``."""
    return [np.asarray(v, dtype=dtype).reshape(1, -1, 1).copy() for v in vectors]


def cp_tt(factors, dtype=np.float64):
    """TT with diagonal interior slices: G_k[r, i, r'] = delta(r, r') u_k^r[i].

    ``factors[k]`` is an (R, I_k) array of vectors u_k^r.  The first core is
    (1, I_1, R) with G_1[0, i, r] = u_1^r[i], the last (R, I_N, 1) with
    G_N[r, i, 0] = u_N^r[i].  The TT then equals sum_r (outer_k u_k^r), a CP
    tensor of rank R.
    """
    n = len(factors)
    cores = []
    for k, f in enumerate(factors):
        f = np.asarray(f, dtype=np.float64)
        R, I = f.shape
        if n == 1:
            g = f.sum(axis=0).reshape(1, I, 1)
        elif k == 0:
            g = f.T.reshape(1, I, R)
        elif k == n - 1:
            g = f.reshape(R, I, 1)
        else:
            g = np.zeros((R, I, R))
            for r in range(R):
                g[r, :, r] = f[r]
        cores.append(np.ascontiguousarray(g.astype(dtype)))
    return cores


def pair(seed: int, modes, ranks_x, ranks_y, dtype=np.float64, log_scale_sigma: float = 0.0):
    """Two independent Gaussian TTs drawn from one seeded stream (X first)."""
    rng = np.random.default_rng(seed)
    x = random_tt(rng, modes, ranks_x, dtype, log_scale_sigma)
    y = random_tt(rng, modes, ranks_y, dtype, log_scale_sigma)
    return x, y


def small_fp64(seed: int = 0):
    """Order 4, all modes 8, ranks (1,4,4,4,1), float64.  Partial: modes 3,4."""
    modes = [8] * 4
    r = [1, 4, 4, 4, 1]
    return pair(seed, modes, r, r, np.float64)


def order10_r64(seed: int = 0, dtype=np.float32):
    """Order 10, modes 16, internal ranks 64.  Partial: modes 1-6."""
    modes = [16] * 10
    r = tt_ranks(10, 64)
    return pair(seed, modes, r, r, dtype)


def order16_r256(seed: int = 0, dtype=np.float32):
    """Order 16, modes 32, internal ranks 256, log-normal core scales (sigma 1)."""
    modes = [32] * 16
    r = tt_ranks(16, 256)
    return pair(seed, modes, r, r, dtype, log_scale_sigma=1.0)


def order12_r64(seed: int = 0, dtype=np.float32):
    """Order 12, modes 16, ranks 64.  Partial: modes 1-8 contracted, 9-12 free."""
    modes = [16] * 12
    r = tt_ranks(12, 64)
    return pair(seed, modes, r, r, dtype)


def batch4096_spec(n_pairs: int = 4096, seed: int = 0):
    """Shapes of the uneven batch, without drawing any core values.

    Returns a list of dicts with keys ``modes``, ``ranks_x``, ``ranks_y``,
    ``kind`` ("full" or "partial") and ``mask`` (1 = contracted mode; for full
    pairs all ones).  Pair p uses the stream default_rng([seed, p]); the core
    values of pair p are drawn afterwards from the same stream by
    :func:`batch_pair`.
    """
    specs = []
    for p in range(n_pairs):
        rng = np.random.default_rng([seed, p])
        specs.append(_batch_shape(rng, p))
    return specs


def _batch_shape(rng, p):
    n = int(rng.integers(4, 13))
    modes = [int(v) for v in rng.integers(2, 33, size=n)]
    rx = [1] + [int(v) for v in rng.integers(4, 129, size=n - 1)] + [1]
    ry = [1] + [int(v) for v in rng.integers(4, 129, size=n - 1)] + [1]
    lead = bool(rng.integers(0, 2))
    if p % 2 == 0:
        kind = "full"
        mask = [1] * n
    else:
        kind = "partial"
        s = n // 2
        mask = [0] * n
        for k in range(s):
            mask[k if lead else n - 1 - k] = 1
    return {"modes": modes, "ranks_x": rx, "ranks_y": ry, "kind": kind, "mask": mask}


def batch_pair(p: int, seed: int = 0, dtype=np.float32):
    """Shape and cores of pair ``p`` of the uneven batch."""
    rng = np.random.default_rng([seed, p])
    spec = _batch_shape(rng, p)
    x = random_tt(rng, spec["modes"], spec["ranks_x"], dtype)
    y = random_tt(rng, spec["modes"], spec["ranks_y"], dtype)
    return spec, x, y


def random_sets_pair(p: int, seed: int = 0, dtype=np.float32):
    """Pair ``p`` of the random-contracted-set batch: order U{4..12}, mode
    sizes U{2..32} shared by the pair, internal ranks U{4..16} per bond and
    operand, and S = a uniformly drawn set of floor(N/2) modes (any
    positions).  Stream default_rng([seed, 1, p]); shape first, then the
    cores of X and Y."""
    rng = np.random.default_rng([seed, 1, p])
    n = int(rng.integers(4, 13))
    modes = [int(v) for v in rng.integers(2, 33, size=n)]
    rx = [1] + [int(v) for v in rng.integers(4, 17, size=n - 1)] + [1]
    ry = [1] + [int(v) for v in rng.integers(4, 17, size=n - 1)] + [1]
    sset = set(int(v) for v in rng.choice(n, size=n // 2, replace=False))
    mask = [1 if k in sset else 0 for k in range(n)]
    x = random_tt(rng, modes, rx, dtype)
    y = random_tt(rng, modes, ry, dtype)
    return mask, x, y


def to_bf16_f32(a: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest even), kept as float32.

    Used to give the oracle exactly the values a BF16-stored core holds.
    """
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32)
    nan = np.isnan(a)
    if nan.any():
        out = out.copy()
        out[nan] = np.nan
    return out


def batch4096_device(n_pairs: int = 4096, seed: int = 0, device="cuda", dtype=None, subset=None):
    """Cores of the uneven batch drawn on the device (the shapes are those of
    :func:`batch4096_spec`).  Core k of X (Y) of pair p is filled from a
    torch CUDA generator seeded with (seed, p, side, k), N(0, 1/(I_k R_k)).
    All cores of the batch live in one arena (16-byte aligned views), so the
    whole 15 GB batch is drawn in a few seconds.  Returns (specs, pairs) with
    pairs[p] = (x_cores, y_cores, mask or None).  With ``subset`` (a list of
    pair indices, e.g. one rank's shard) only those pairs are drawn, with the
    same values as in the whole batch, and specs/pairs follow that list."""
    import torch

    dtype = dtype or torch.float32
    specs_all = batch4096_spec(n_pairs, seed)
    ids = list(range(n_pairs)) if subset is None else [int(p) for p in subset]
    specs = [specs_all[p] for p in ids]
    esize = torch.tensor([], dtype=dtype).element_size()
    align = max(1, 16 // esize)
    sizes = []
    for s in specs:
        for ranks in (s["ranks_x"], s["ranks_y"]):
            for k, I in enumerate(s["modes"]):
                n = ranks[k] * I * ranks[k + 1]
                sizes.append((n + align - 1) // align * align)
    arena = torch.empty(sum(sizes), dtype=dtype, device=device)
    gen = torch.Generator(device=device)
    off = 0
    pairs = []
    for p, s in zip(ids, specs):
        sides = []
        for side, ranks in enumerate((s["ranks_x"], s["ranks_y"])):
            cores = []
            for k, I in enumerate(s["modes"]):
                shape = (ranks[k], I, ranks[k + 1])
                n = shape[0] * shape[1] * shape[2]
                view = arena[off : off + n].view(shape)
                gen.manual_seed(((seed * 1_000_003 + p) * 2 + side) * 64 + k)
                view.normal_(0.0, 1.0 / float(np.sqrt(I * ranks[k + 1])), generator=gen)
                cores.append(view)
                off += (n + align - 1) // align * align
            sides.append(cores)
        pairs.append((sides[0], sides[1], None if s["kind"] == "full" else s["mask"]))
    return specs, pairs
