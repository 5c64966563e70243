"""First-order rounding-error model of the environment sweep (test infrastructure).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the tests use it to
state, for a given pair of TTs, how far a sweep carried out in reduced
precision may be from the float64 oracle.  It is a standard probabilistic
first-order analysis (each rounding is an independent relative perturbation
of zero mean; Higham, "Accuracy and Stability of Numerical Algorithms",
2nd ed., 2002, Sections 2.8 and 3.1), applied to the sweep of Algorithm 2
step 4 generalised to every mode (Eq. 8 applied mode after mode):

    z = <L_k, R_k>  for every k,   L_{k+1} = sum_i A_i^T (L_k B_i),

with L_k the left environment before mode k, R_k the right environment over
modes k..N-1, A_i / B_i the i-th slices of the cores of X / Y.  A relative
perturbation d of one quantity q changes z, to first order, by
(dz/dq) q d; independent perturbations add in variance.  The model sums:

  e    L_k rounded before the first product of mode k:
       sum_ab (R_k L_k)[a,b]^2
  t    T_i = L_k B_i rounded before the second product:
       sum_i sum_ab (T_i (A_i R_{k+1}))[a,b]^2     (elementwise product)
  core every core entry rounded once:  sum (G * dz/dG)^2 (both operands;
       dz/dGx_k[:, i, :] = L_k Gy_k[:, i, :] R_{k+1}^T and its mirror)
  prod an independent error on every single product term of both GEMMs:
       sum over the terms t of (t * w)^2, w the weight dz/d(output)
  acc  float32 accumulation of a sum of n terms, taken as n roundings of
       partial sums of the size of the whole sum's terms: n * sum (t * w)^2

Each entry of ``rounds`` gives the relative standard deviation of one kind
and the modes it applies to; the result is the predicted standard deviation
of z - z* (an absolute number, in the units of z).

Coherent part.  A tensor-core accumulator that adds each step's products to
its float32 value with a rounding toward zero (as Fasi, Higham, Mikaitis and
Pranesh observed for earlier NVIDIA tensor cores: "Numerical behavior of
NVIDIA tensor cores", PeerJ Computer Science 7:e330, 2021) loses on average
half an ulp of the running sum, always toward zero.  For a sum of n_r such
steps whose partial sums grow like the final value o, the mean loss is about
(n_r / 2) 2^-24 |o| and has the sign that shrinks o; every output of a stage
shrinks by the same relative amount, so z does too: the stage contributes a
relative bias of -(n_r / 2) 2^-24 to z whatever the signs of the data.
``tc_bias`` sums this over the tensor-core stages of the full contraction.
"""
from __future__ import annotations

import numpy as np

from .tt_oracle import left_envs, right_envs

U_BF16 = 2.0**-8   # unit roundoff of bfloat16 (8 significant bits)
U_F32 = 2.0**-24   # unit roundoff of float32

# Standard deviation of the relative error of round-to-nearest to p
# significant bits, for significands spread log-uniformly over an octave:
# the absolute error is uniform on half an ulp either side (variance
# ulp^2 / 12), and E[1/m^2] = 3 / (8 ln 2) for m in [1, 2).
_RN_STD = float(np.sqrt((4.0 / 12.0) * 3.0 / (8.0 * np.log(2.0))))  # times u


def rn_std(u):
    """Relative standard deviation of one round-to-nearest with unit roundoff u."""
    return _RN_STD * u


def sweep_error_sigma(xc, yc, rounds, modes=None):
    """Predicted standard deviation of the error of <X, Y> from a sweep whose
    roundings are described by ``rounds`` (keys "e", "t", "core", "prod",
    "acc"; each a relative standard deviation, 0 or missing = exact).
    ``modes`` limits every kind to the listed 0-based modes (default: every
    mode; "core" then means the cores of those modes, of both operands).
    """
    xc = [np.asarray(c, dtype=np.float64) for c in xc]
    yc = [np.asarray(c, dtype=np.float64) for c in yc]
    n = len(xc)
    le = left_envs(xc, yc)
    re = right_envs(xc, yc)
    s_e = rounds.get("e", 0.0)
    s_t = rounds.get("t", 0.0)
    s_c = rounds.get("core", 0.0)
    s_p = rounds.get("prod", 0.0)
    s_a = rounds.get("acc", 0.0)
    var = 0.0
    sel = range(n) if modes is None else modes
    for k in sel:
        lk, rk1 = le[k], re[k + 1]
        gx, gy = xc[k], yc[k]
        if s_e:
            var += s_e**2 * float(np.sum((re[k] * lk) ** 2))
        lk2 = lk * lk
        for i in range(gx.shape[1]):
            a, b = gx[:, i, :], gy[:, i, :]
            t = lk @ b                      # T_i = L_k B_i
            w = a @ rk1                     # dz/dT_i
            if s_t:
                var += s_t**2 * float(np.sum((t * w) ** 2))
            if s_p or s_a:
                # terms of GEMM 1: L_k[a,c] B[c,b'], weight w[a,b'];
                # terms of GEMM 2: A[a,a'] T[a,b'], weight rk1[a',b']
                sq1 = float(np.sum((lk2 @ (b * b)) * (w * w)))
                sq2 = float(np.sum(((a * a).T @ (t * t)) * (rk1 * rk1)))
                if s_p:
                    var += s_p**2 * (sq1 + sq2)
                if s_a:
                    var += s_a**2 * (lk.shape[1] * sq1 + a.shape[0] * gx.shape[1] * sq2)
    if s_c:
        for k in sel:
            lk, rk1 = le[k], re[k + 1]
            for i in range(xc[k].shape[1]):
                gxi = lk @ yc[k][:, i, :] @ rk1.T      # dz/dGx_k[:, i, :]
                gyi = lk.T @ xc[k][:, i, :] @ rk1      # dz/dGy_k[:, i, :]
                var += s_c**2 * float(np.sum((xc[k][:, i, :] * gxi) ** 2) + np.sum((yc[k][:, i, :] * gyi) ** 2))
    return float(np.sqrt(var))


def tc_rounds(prec):
    """The roundings of the tensor-core full contraction, by product form.

    The first mode (left rank 1) and the last mode (right rank 1) run on the
    CUDA cores in float32 (the last one summed in float64); every interior
    mode takes E and each T_i through the tensor cores:
      "bf16": E and T_i rounded to bfloat16 (the cores are bfloat16 already,
              or rounded once on the way in; the reference is then the oracle
              on the rounded cores), products exact, sums in float32;
      "bf16x3": every operand (E, T_i, core entries) held as hi + lo
              bfloat16 pieces, so its representation error is the rounding
              of lo (u^2 relative), and each product drops lo*lo (a further
              u^2 relative per product term); sums in float32.
    Returns (rounds, interior_only) for sweep_error_sigma."""
    if prec == "bf16":
        s = rn_std(U_BF16)
        return {"e": s, "t": s, "acc": rn_std(U_F32)}, True
    if prec == "bf16x3":
        s = rn_std(U_BF16) ** 2
        return {"e": s, "t": s, "core": s, "prod": s, "acc": rn_std(U_F32)}, True
    raise ValueError(prec)


def tc_error_sigma(xc, yc, prec):
    """sweep_error_sigma for the tensor-core full contraction of ``prec``."""
    rounds, interior = tc_rounds(prec)
    n = len(xc)
    modes = list(range(1, n - 1)) if interior else None
    sig = sweep_error_sigma(xc, yc, rounds, modes)
    # the float32 first and last modes: accumulation only
    ends = [k for k in (0, n - 1) if k not in (modes or [])]
    if ends:
        sig = float(np.hypot(sig, sweep_error_sigma(xc, yc, {"acc": rn_std(U_F32)}, ends)))
    return sig


def acc_bias_rel(n_roundings):
    """Mean relative shrinkage of a sum accumulated by n_roundings additions
    that round toward zero (half an ulp of float32 each, partial sums growing
    like the final value)."""
    return 0.5 * n_roundings * U_F32


def tc_bias(xc, yc, prec, cluster=16):
    """Predicted coherent relative bias of the tensor-core full contraction
    (a negative number: z is shrunk), from the accumulation roundings of each
    interior mode: GEMM 1 accumulates T over ceil(R^y_k / 16) steps of 16 and
    GEMM 2 accumulates P over ceil(R^x_k / 16) steps per slice and
    ceil(I_k / cluster) slices (the slices of a mode are spread over the
    CTAs of a cluster, whose partial P's are then added on the CUDA cores,
    rounding to nearest); the split form issues three products per step."""
    m = {"bf16": 1, "bf16x3": 3}[prec]
    n = len(xc)
    rel = 0.0
    for k in range(1, n - 1):
        rx, i_dim, _ = np.shape(xc[k])
        ry = np.shape(yc[k])[0]
        n_t = m * -(-ry // 16)
        n_p = m * -(-rx // 16) * -(-i_dim // cluster)
        rel += acc_bias_rel(n_t) + acc_bias_rel(n_p)
    return -rel


def tc_bound(xc, yc, prec, z_ref, k_sigma=8.0):
    """The GPU tests' bound on |z - z*| for the tensor-core form ``prec``:
    k_sigma predicted standard deviations of the random part, plus twice the
    predicted coherent bias (|z*| times tc_bias)."""
    return k_sigma * tc_error_sigma(xc, yc, prec) + 2.0 * abs(tc_bias(xc, yc, prec)) * abs(z_ref)


U_TF32 = 2.0**-11  # unit roundoff of tf32 (11 significant bits)


def tf32_rounds(prec):
    """Roundings of the tf32 tensor-core sweep (every mode but the float64
    last one of a one-sided full contraction runs on the tensor cores):
      "tf32":   E, each T_i and every core entry rounded to tf32 (nearest);
      "tf32x3": each of them held as hi = tf32(x) (nearest) and lo = x - hi,
                lo read by the tensor core with its low 13 bits dropped (a
                rounding toward zero to tf32's 11 bits: twice the standard
                deviation of one to nearest, on a value whose size relative to
                x has standard deviation rn_std(2^-11)); all four products
                hi*hi + hi*lo + lo*hi + lo*lo formed.
    Sums in float32 in both."""
    if prec == "tf32":
        s = rn_std(U_TF32)
        return {"e": s, "t": s, "core": s, "acc": rn_std(U_F32)}
    if prec == "tf32x3":
        s = 2.0 * rn_std(U_TF32) ** 2
        return {"e": s, "t": s, "core": s, "acc": rn_std(U_F32)}
    raise ValueError(prec)


def tf32_modes(n, two_sided):
    """Modes of an order-n full contraction that run on the tensor cores."""
    return list(range(n)) if two_sided else list(range(n - 1))


def tf32_bias(xc, yc, prec, two_sided, cluster=16):
    """Predicted coherent relative bias (negative) of the tf32 sweep: every
    tensor-core mode accumulates T over passes x ceil(R^y_k / 8) steps and P
    over passes x ceil(R^x_k / 8) steps per slice, ceil(I_k / cluster) slices
    per CTA; passes = 2 for the split form (the other operand's hi, then lo),
    1 for tf32."""
    m = {"tf32": 1, "tf32x3": 2}[prec]
    rel = 0.0
    for k in tf32_modes(len(xc), two_sided):
        rx, i_dim, _ = np.shape(xc[k])
        ry = np.shape(yc[k])[0]
        rel += acc_bias_rel(m * -(-ry // 8)) + acc_bias_rel(m * -(-rx // 8) * -(-i_dim // cluster))
    return -rel


def tf32_bound(xc, yc, prec, z_ref, two_sided, cluster=16, k_sigma=8.0):
    """The tests' bound on |z - z*| for the tf32 forms: k_sigma standard
    deviations of the random part plus twice the coherent bias."""
    modes = tf32_modes(len(xc), two_sided)
    sig = sweep_error_sigma(xc, yc, tf32_rounds(prec), modes)
    rest = [k for k in range(len(xc)) if k not in modes]
    if rest:
        sig = float(np.hypot(sig, sweep_error_sigma(xc, yc, {"acc": rn_std(U_F32)}, rest)))
    return k_sigma * sig + 2.0 * abs(tf32_bias(xc, yc, prec, two_sided, cluster)) * abs(z_ref)
