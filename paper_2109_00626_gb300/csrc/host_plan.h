// Host-side helpers shared by the C-ABI translation units: descriptor
// validation, sweep parameter filling and the chain-layout plan.
#pragma once

#include <string.h>

#include <algorithm>

#include "ttc_internal.h"

namespace ttc {

inline int elem_bytes(int dtype) {
  switch (dtype) {
    case TT_F64: return 8;
    case TT_F32: return 4;
    case TT_BF16: return 2;
    default: return 0;
  }
}

inline size_t align256(size_t v) { return (v + 255) & ~static_cast<size_t>(255); }

inline int check_desc(const tt_desc* d) {
  if (d == nullptr || d->order < 1 || d->order > kMaxOrder || d->modes == nullptr || d->ranks == nullptr ||
      d->cores == nullptr)
    return TT_ERR_ARG;
  if (elem_bytes(d->dtype) == 0) return TT_ERR_DTYPE;
  if (d->ranks[0] != 1 || d->ranks[d->order] != 1) return TT_ERR_SHAPE;
  for (int k = 0; k < d->order; ++k) {
    if (d->modes[k] < 1 || d->ranks[k + 1] < 1) return TT_ERR_SHAPE;
    if (d->cores[k] == nullptr) return TT_ERR_ARG;
  }
  return TT_OK;
}

// Same order and dtype; equal mode sizes wherever mask is set (mask NULL = all).
inline int check_pair(const tt_desc* x, const tt_desc* y, const uint8_t* mask) {
  int rc = check_desc(x);
  if (rc != TT_OK) return rc;
  rc = check_desc(y);
  if (rc != TT_OK) return rc;
  if (x->order != y->order) return TT_ERR_SHAPE;
  if (x->dtype != y->dtype) return TT_ERR_DTYPE;
  for (int k = 0; k < x->order; ++k)
    if ((mask == nullptr || mask[k]) && x->modes[k] != y->modes[k]) return TT_ERR_SHAPE;
  return TT_OK;
}

// Classify the contracted set: 0 = leading block {0..s-1}, 1 = trailing block
// {N-s..N-1}, -1 = neither (the empty set counts as leading); *s_out = |S|.
inline int end_block(const uint8_t* mask, int n, int* s_out) {
  int s = 0;
  for (int k = 0; k < n; ++k) s += mask[k] ? 1 : 0;
  *s_out = s;
  bool lead = true, trail = true;
  for (int k = 0; k < n; ++k) {
    if ((mask[k] != 0) != (k < s)) lead = false;
    if ((mask[k] != 0) != (k >= n - s)) trail = false;
  }
  if (lead) return 0;
  if (trail) return 1;
  return -1;
}

inline int max_rank(const tt_desc* d) {
  int r = 1;
  for (int k = 0; k <= d->order; ++k) r = std::max(r, d->ranks[k]);
  return r;
}

inline int rank_cap(int dtype) { return dtype == TT_F64 ? 64 : 128; }

inline int pow2_floor(int v) {
  int c = 1;
  while (c * 2 <= v) c *= 2;
  return c;
}

// Fill a left-to-right sweep over modes [k0, k1) of (x, y).
inline void fill_left(SweepParams& p, const tt_desc* x, const tt_desc* y, int k0, int k1) {
  p.n_steps = k1 - k0;
  p.transposed = 0;
  p.transposed_y = 0;
  for (int j = 0; j < p.n_steps; ++j) {
    const int k = k0 + j;
    SweepStep& st = p.step[j];
    st.gx = x->cores[k];
    st.gy = y->cores[k];
    st.I = x->modes[k];
    st.rin_x = x->ranks[k];
    st.rout_x = x->ranks[k + 1];
    st.rin_y = y->ranks[k];
    st.rout_y = y->ranks[k + 1];
  }
}

// Fill a right-to-left sweep over modes k1-1 down to k0.
inline void fill_right(SweepParams& p, const tt_desc* x, const tt_desc* y, int k0, int k1) {
  p.n_steps = k1 - k0;
  p.transposed = 1;
  p.transposed_y = 1;
  for (int j = 0; j < p.n_steps; ++j) {
    const int k = k1 - 1 - j;
    SweepStep& st = p.step[j];
    st.gx = x->cores[k];
    st.gy = y->cores[k];
    st.I = x->modes[k];
    st.rin_x = x->ranks[k + 1];
    st.rout_x = x->ranks[k];
    st.rin_y = y->ranks[k + 1];
    st.rout_y = y->ranks[k];
  }
}

inline int sweep_max_rank(const SweepParams& p) {
  int r = std::max(p.rx0, p.ry0);
  for (int j = 0; j < p.n_steps; ++j)
    r = std::max({r, p.step[j].rin_x, p.step[j].rout_x, p.step[j].rin_y, p.step[j].rout_y});
  if (p.emit.enabled) r = std::max({r, p.emit.ra, p.emit.rb, p.emit.ry});
  return r;
}

inline int sweep_max_mode(const SweepParams& p) {
  int m = 1;
  for (int j = 0; j < p.n_steps; ++j) m = std::max(m, p.step[j].I);
  if (p.emit.enabled) m = std::max(m, p.emit.I);
  return m;
}

inline int launch_sweep(const SweepParams& p, int dtype, cudaStream_t s) {
  const int rmax = sweep_max_rank(p);
  if (rmax > rank_cap(dtype)) return TT_ERR_TOO_LARGE;
  const int eb = elem_bytes(dtype);
  const int want = pow2_floor(std::min(16, sweep_max_mode(p)));
  const int C = sweep_cluster_size(rmax, eb, want);
  if (C < 1) return TT_ERR_CUDA;
  cudaError_t err = dtype == TT_F64 ? launch_sweep_f64(p, rmax, C, s) : launch_sweep_f32(p, rmax, C, s);
  return err == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

struct ChainPlan {
  int side;  // 0 lead, 1 trail
  int s, m;
  int n;
  // output cores
  int order;
  int modes[2 * kMaxOrder];
  int ranks[2 * kMaxOrder + 1];
  int perm[2 * kMaxOrder];
  // K shape
  int kx, ky;
};

inline int chain_plan(const tt_desc* x, const tt_desc* y, const uint8_t* mask, ChainPlan* cp) {
  const int n = x->order;
  int s = 0;
  const int side = end_block(mask, n, &s);
  if (s == n) return TT_ERR_ARG;
  if (side < 0) return TT_ERR_LAYOUT;
  const int m = n - s;
  cp->side = side;
  cp->s = s;
  cp->m = m;
  cp->n = n;
  cp->order = 2 * m;
  if (side == 0) {
    // Gx_{N-1}^T .. Gx_{s+1}^T, C, Gy_s .. Gy_{N-1}
    for (int p = 0; p < m - 1; ++p) {
      const int k = n - 1 - p;
      cp->modes[p] = x->modes[k];
      cp->ranks[p] = x->ranks[k + 1];
    }
    cp->modes[m - 1] = x->modes[s];
    cp->ranks[m - 1] = x->ranks[s + 1];
    for (int q = 0; q < m; ++q) {
      cp->modes[m + q] = y->modes[s + q];
      cp->ranks[m + q] = y->ranks[s + q];
    }
    cp->ranks[2 * m] = 1;
    for (int p = 0; p < m; ++p) cp->perm[p] = m - 1 - p;
    for (int q = 0; q < m; ++q) cp->perm[m + q] = m + q;
    cp->kx = x->ranks[s];
    cp->ky = y->ranks[s];
  } else {
    // Gx_0 .. Gx_{m-2}, C, Gy_{m-1}^T .. Gy_0^T
    for (int p = 0; p < m; ++p) {
      cp->modes[p] = x->modes[p];
      cp->ranks[p] = x->ranks[p];
    }
    for (int q = 0; q < m; ++q) {
      const int k = m - 1 - q;
      cp->modes[m + q] = y->modes[k];
      cp->ranks[m + q] = y->ranks[k + 1];
    }
    cp->ranks[2 * m] = 1;
    for (int p = 0; p < m; ++p) cp->perm[p] = p;
    for (int q = 0; q < m; ++q) cp->perm[m + q] = m + (m - 1 - q);
    cp->kx = x->ranks[m];
    cp->ky = y->ranks[m];
  }
  return TT_OK;
}

// Check that z describes exactly the chain-layout output of cp.
inline int check_chain_output(const tt_desc* x, const ChainPlan& cp, const tt_desc* z) {
  const int rc = check_desc(z);
  if (rc != TT_OK) return rc;
  if (z->order != cp.order || z->dtype != x->dtype) return TT_ERR_SHAPE;
  for (int q = 0; q < cp.order; ++q)
    if (z->modes[q] != cp.modes[q] || z->ranks[q] != cp.ranks[q]) return TT_ERR_SHAPE;
  return TT_OK;
}

// Sweep parameters of a chain-layout partial contraction: the sweep over the
// contracted block followed by the fused emission of C and the free cores.
inline int build_partial(const tt_desc* x, const tt_desc* y, const ChainPlan& cp, const tt_desc* z,
                         int64_t* z_log2_dev, int32_t* status_dev, SweepParams* out) {
  SweepParams& p = *out;
  memset(&p, 0, sizeof(p));
  const int n = cp.n, m = cp.m, sS = cp.s;
  if (sS > 0) {
    if (cp.side == 0) fill_left(p, x, y, 0, sS);
    else fill_right(p, x, y, m, n);
  }
  p.rx0 = 1;
  p.ry0 = 1;
  p.final_scalar = 0;
  p.renorm_bits = x->dtype == TT_F64 ? kRenormBitsF64 : kRenormBitsF32;
  p.status = status_dev;
  EmitParams& ep = p.emit;
  ep.enabled = 1;
  const int kb = cp.side == 0 ? sS : m - 1;
  ep.gx = x->cores[kb];
  ep.ra = x->ranks[kb];
  ep.I = x->modes[kb];
  ep.rb = x->ranks[kb + 1];
  ep.lead = cp.side == 0 ? 1 : 0;
  ep.ry = cp.ky;
  ep.c_out = z->cores[m - 1];
  ep.z_log2_out = z_log2_dev;
  auto add = [&](const void* src, void* dst, int r0, int I, int r1, int swap) -> int {
    if (!swap && src == dst) return TT_OK;  // output aliases its input: nothing to copy
    if (swap && src == dst) return TT_ERR_ARG;
    if (static_cast<int64_t>(r0) * I * r1 >= (int64_t(1) << 31)) return TT_ERR_TOO_LARGE;
    CopyTask& t = ep.copy[ep.n_copies++];
    t.src = src;
    t.dst = dst;
    t.r0 = r0;
    t.I = I;
    t.r1 = r1;
    t.swap = swap;
    return TT_OK;
  };
  int rc = TT_OK;
  if (cp.side == 0) {
    for (int q = 0; q < m - 1 && rc == TT_OK; ++q) {
      const int k = n - 1 - q;
      rc = add(x->cores[k], z->cores[q], x->ranks[k], x->modes[k], x->ranks[k + 1], 1);
    }
    for (int q = 0; q < m && rc == TT_OK; ++q) {
      const int k = sS + q;
      rc = add(y->cores[k], z->cores[m + q], y->ranks[k], y->modes[k], y->ranks[k + 1], 0);
    }
  } else {
    for (int q = 0; q < m - 1 && rc == TT_OK; ++q)
      rc = add(x->cores[q], z->cores[q], x->ranks[q], x->modes[q], x->ranks[q + 1], 0);
    for (int q = 0; q < m && rc == TT_OK; ++q) {
      const int k = m - 1 - q;
      rc = add(y->cores[k], z->cores[m + q], y->ranks[k], y->modes[k], y->ranks[k + 1], 1);
    }
  }
  return rc;
}

// Sweep parameters of a full contraction.
inline void build_full(const tt_desc* x, const tt_desc* y, double* out_dev, int64_t* out_log2_dev,
                       int32_t* status_dev, SweepParams* out) {
  SweepParams& p = *out;
  memset(&p, 0, sizeof(p));
  fill_left(p, x, y, 0, x->order);
  p.rx0 = 1;
  p.ry0 = 1;
  p.final_scalar = 1;
  p.renorm_bits = x->dtype == TT_F64 ? kRenormBitsF64 : kRenormBitsF32;
  p.z_out = out_dev;
  p.z_out_log2 = out_log2_dev;
  p.status = status_dev;
}

// Workspace of a full contraction run from both ends (sweep.cu): the two
// meeting environments, their scales and the arrival counter.
struct TwoSidedLayout {
  int h = 0;  // modes [0, h) sweep left to right, [h, N) right to left
  int rx = 1, ry = 1;
  size_t off_el = 0, off_er = 0, off_ll = 0, off_lr = 0, off_ctr = 0, bytes = 0;
};

inline TwoSidedLayout two_sided_layout(const tt_desc* x, const tt_desc* y) {
  TwoSidedLayout L;
  const int n = x->order;
  L.h = n / 2;
  L.rx = x->ranks[L.h];
  L.ry = y->ranks[L.h];
  const size_t env = align256(static_cast<size_t>(L.rx) * L.ry * elem_bytes(x->dtype));
  L.off_el = 0;
  L.off_er = env;
  L.off_ll = 2 * env;
  L.off_lr = L.off_ll + 256;
  L.off_ctr = L.off_lr + 256;
  L.bytes = L.off_ctr + 256;
  return L;
}

// Parameters of the two half sweeps into a workspace laid out by L.
inline void build_two_sided(const tt_desc* x, const tt_desc* y, const TwoSidedLayout& L, void* ws, double* out_dev,
                            int64_t* out_log2_dev, int32_t* status_dev, TwoSidedParams* tp) {
  char* w = static_cast<char*>(ws);
  const int n = x->order;
  for (int side = 0; side < 2; ++side) {
    SweepParams& p = tp->half[side];
    memset(&p, 0, sizeof(p));
    if (side == 0) fill_left(p, x, y, 0, L.h);
    else fill_right(p, x, y, L.h, n);
    p.rx0 = 1;
    p.ry0 = 1;
    p.final_scalar = 0;
    p.renorm_bits = x->dtype == TT_F64 ? kRenormBitsF64 : kRenormBitsF32;
    p.e_out = w + (side == 0 ? L.off_el : L.off_er);
    p.e_out_log2 = reinterpret_cast<int64_t*>(w + (side == 0 ? L.off_ll : L.off_lr));
    p.status = status_dev;
  }
  tp->rx = L.rx;
  tp->ry = L.ry;
  tp->z_out = out_dev;
  tp->z_out_log2 = out_log2_dev;
  tp->status = status_dev;
  tp->counter = reinterpret_cast<int*>(w + L.off_ctr);
}

inline int check_same_shape(const tt_desc* a, const tt_desc* g) {
  const int rc = check_desc(g);
  if (rc != TT_OK) return rc;
  if (g->order != a->order || g->dtype != a->dtype) return TT_ERR_SHAPE;
  for (int k = 0; k < a->order; ++k)
    if (g->modes[k] != a->modes[k] || g->ranks[k] != a->ranks[k]) return TT_ERR_SHAPE;
  return TT_OK;
}

// Workspace layout of tt_contract_backward.
// Where the folded cores of a rank-1 contraction go (adjoint_r1.cu): M_k at
// element offset moff[k], 16-byte aligned; returns the total elements.
inline int64_t r1_fold_layout(const tt_desc* x, int64_t* moff) {
  int64_t off = 0;
  for (int k = 0; k < x->order; ++k) {
    if (moff != nullptr) moff[k] = off;
    off += (static_cast<int64_t>(x->ranks[k]) * x->ranks[k + 1] + 3) & ~static_cast<int64_t>(3);
  }
  return off;
}

// The full contraction of a Y of rank 1 (the sum of a TT's entries and the
// like; order >= 2) folds X's cores with y and runs one chain of
// vector-matrix products.
inline bool full_is_r1(const tt_desc* x, const tt_desc* y) {
  return x->order >= 2 && max_rank(y) == 1 && max_rank(x) <= kR1MaxRank && x->dtype != TT_BF16;
}
inline size_t full_r1_bytes(const tt_desc* x) {
  return align256(static_cast<size_t>(r1_fold_layout(x, nullptr)) * elem_bytes(x->dtype));
}

struct BackwardPlan {
  ChainPlan cp;
  int partial = 0;
  int r1 = 0;  // full contraction with Y of rank 1 everywhere: vector adjoint (adjoint_r1.cu)
  size_t off_lvec = 0, off_fvec = 0, off_llog = 0, off_flog = 0, off_m = 0, off_mt = 0;
  int64_t vstride = 1;
  int rmax = 1;
  int64_t env_elems = 1;
  // Every left environment L_0..L_{N-1} of the block (written by the forward
  // sweep, or by the adjoint's own forward pass) and every right environment
  // F_1..F_N (written by the backward walk): the gradients of all modes are
  // then formed by one launch over every (mode, slice), off the walk's
  // critical path.  2N environments of R^x R^y elements.
  size_t off_k = 0, off_klog2 = 0, off_dk = 0, off_ckpt = 0, off_ckpt_log2 = 0, off_fenv = 0, off_fenv_log2 = 0;
  // leg-swapped copies of the block's cores (X then Y, mode by mode, each
  // 256-byte aligned): the right-to-left sweep and the gradients read them
  size_t off_swap = 0;
  int k0 = 0, k1 = 0;  // the block
  size_t ws_bytes = 0;
};

inline size_t swap_core_bytes(const tt_desc* d, int k) {
  return align256(static_cast<size_t>(d->ranks[k]) * d->modes[k] * d->ranks[k + 1] * elem_bytes(d->dtype));
}

inline int adjoint_rank_cap(int dtype) { return dtype == TT_F64 ? 32 : 64; }

inline int backward_plan(const tt_desc* x, const tt_desc* y, const uint8_t* mask, int layout, int prec, int stride,
                         BackwardPlan* bp) {
  int rc = check_pair(x, y, mask);
  if (rc != TT_OK) return rc;
  if (prec != TT_P_NATIVE) return TT_ERR_UNSUPPORTED;
  if (x->dtype == TT_BF16) return TT_ERR_UNSUPPORTED;
  if (stride < 0) return TT_ERR_ARG;
  const int n = x->order;
  bp->partial = mask != nullptr;
  int nblock = n;
  if (mask != nullptr) {
    if (layout != TT_LAYOUT_CHAIN) return TT_ERR_UNSUPPORTED;
    rc = chain_plan(x, y, mask, &bp->cp);
    if (rc != TT_OK) return rc;
    nblock = std::max(1, bp->cp.s);
  }
  const int rmax = std::max(max_rank(x), max_rank(y));
  bp->rmax = rmax;
  if (mask == nullptr && max_rank(y) == 1) {
    // environments are vectors: keep all of them, no checkpoints
    if (max_rank(x) > kR1MaxRank) return TT_ERR_TOO_LARGE;
    bp->r1 = 1;
    const int eb1 = elem_bytes(x->dtype);
    bp->vstride = max_rank(x);
    const size_t vbytes = align256(static_cast<size_t>(n + 1) * bp->vstride * eb1);
    size_t off1 = 0;
    bp->off_lvec = off1;
    off1 += vbytes;
    bp->off_fvec = off1;
    off1 += vbytes;
    bp->off_llog = off1;
    off1 += align256(sizeof(int64_t) * (n + 1));
    bp->off_flog = off1;
    off1 += align256(sizeof(int64_t) * (n + 1));
    const size_t mbytes = align256(static_cast<size_t>(r1_fold_layout(x, nullptr)) * eb1);
    bp->off_m = off1;
    off1 += mbytes;
    bp->off_mt = off1;
    off1 += mbytes;
    bp->ws_bytes = off1;
    return TT_OK;
  }
  if (rmax > adjoint_rank_cap(x->dtype) && (mask == nullptr || bp->cp.s > 0)) return TT_ERR_TOO_LARGE;
  if (mask != nullptr && rmax > rank_cap(x->dtype)) return TT_ERR_TOO_LARGE;
  const int eb = elem_bytes(x->dtype);
  bp->env_elems = static_cast<int64_t>(max_rank(x)) * max_rank(y);
  size_t off = 0;
  if (mask != nullptr) {
    bp->off_k = off;
    off += align256(static_cast<size_t>(bp->cp.kx) * bp->cp.ky * eb);
    bp->off_klog2 = off;
    off += 256;
    bp->off_dk = off;
    off += align256(static_cast<size_t>(kDkGroups) * bp->cp.kx * bp->cp.ky * eb);  // partial sums of dK
  }
  bp->off_ckpt = off;
  off += align256(static_cast<size_t>(nblock) * bp->env_elems * eb);
  bp->off_ckpt_log2 = off;
  off += align256(sizeof(int64_t) * nblock);
  bp->off_fenv = off;
  off += align256(static_cast<size_t>(nblock) * bp->env_elems * eb);
  bp->off_fenv_log2 = off;
  off += align256(sizeof(int64_t) * nblock);
  if (mask == nullptr) {
    bp->k0 = 0;
    bp->k1 = n;
  } else if (bp->cp.side == 0) {
    bp->k0 = 0;
    bp->k1 = bp->cp.s;
  } else {
    bp->k0 = bp->cp.m;
    bp->k1 = n;
  }
  bp->off_swap = off;
  for (int k = bp->k0; k < bp->k1; ++k) off += swap_core_bytes(x, k) + swap_core_bytes(y, k);
  bp->ws_bytes = off;
  return TT_OK;
}

// Plan of a merged-layout partial contraction (see merged.cu).  Every output
// core has workspace of its own (its run's map M, M's row scales, P and four
// scale slots), so that the cores can be built concurrently.
struct MergedPlan {
  int m = 0;
  int free_pos[kMaxOrder];
  int run_k1[kMaxOrder];  // the run after free position f is [f + 1, run_k1)
  int rmax = 1;
  size_t off_m[kMaxOrder], off_mexp[kMaxOrder], off_p[kMaxOrder];
  size_t off_el = 0, off_v = 0, off_w0 = 0, off_slots = 0, ws_bytes = 0;
};

// int64 scale slots: 0 = E_L, then per core t at 1 + 4 t: M, P, W_0, V
constexpr int kMergedSlotsPerCore = 4;

constexpr int64_t kMergedCoreCap = int64_t(1) << 30;  // elements per merged core (and per intermediate)

inline int merged_plan(const tt_desc* x, const tt_desc* y, const uint8_t* mask, MergedPlan* mp) {
  const int n = x->order;
  int m = 0;
  for (int k = 0; k < n; ++k)
    if (!mask[k]) mp->free_pos[m++] = k;
  if (m == 0) return TT_ERR_ARG;
  mp->m = m;
  const int eb = elem_bytes(x->dtype);
  int rmax = 1;
  const int f0 = mp->free_pos[0];
  for (int k = 0; k <= f0; ++k) rmax = std::max({rmax, x->ranks[k], y->ranks[k]});
  int64_t mt[kMaxOrder], qt[kMaxOrder], pt[kMaxOrder], w0 = 0;
  for (int t = 0; t < m; ++t) {
    const int f = mp->free_pos[t];
    const int nxt = t + 1 < m ? mp->free_pos[t + 1] : n;
    mp->run_k1[t] = nxt;
    const int64_t rows = static_cast<int64_t>(t == 0 ? 1 : x->ranks[f] * y->ranks[f]) * x->modes[f] * y->modes[f];
    const int64_t q = static_cast<int64_t>(x->ranks[f + 1]) * y->ranks[f + 1];  // rows of M
    const int64_t C = static_cast<int64_t>(x->ranks[nxt]) * y->ranks[nxt];      // 1 at the end
    if (rows * C > kMergedCoreCap) return TT_ERR_TOO_LARGE;
    mt[t] = qt[t] = pt[t] = 0;
    if (nxt > f + 1) {
      const int64_t pe = static_cast<int64_t>(x->ranks[f]) * x->modes[f] * y->ranks[f + 1] * C;
      if (q * C > kMergedCoreCap || pe > kMergedCoreCap) return TT_ERR_TOO_LARGE;
      mt[t] = q * C;
      qt[t] = q;
      if (t > 0) pt[t] = pe;
      if (t == 0) w0 = static_cast<int64_t>(x->modes[f]) * y->modes[f] * q;
    }
    for (int k = f + 1; k <= nxt && k <= n; ++k) rmax = std::max({rmax, x->ranks[k], y->ranks[k]});
  }
  mp->rmax = rmax;
  if (rmax > rank_cap(x->dtype)) return TT_ERR_TOO_LARGE;
  const int kx = x->ranks[f0], ky = y->ranks[f0];
  size_t off = 0;
  mp->off_slots = off;
  off += align256(static_cast<size_t>(1 + kMergedSlotsPerCore * m) * sizeof(int64_t));
  mp->off_el = off;
  off += align256(static_cast<size_t>(kx) * ky * eb);
  mp->off_v = off;
  off += align256(static_cast<size_t>(kx) * y->modes[f0] * y->ranks[f0 + 1] * eb);
  mp->off_w0 = off;
  off += align256(static_cast<size_t>(w0) * eb);
  for (int t = 0; t < m; ++t) {
    mp->off_m[t] = off;
    off += align256(static_cast<size_t>(mt[t]) * eb);
    mp->off_mexp[t] = off;
    off += align256(static_cast<size_t>(qt[t]) * sizeof(int64_t));
    mp->off_p[t] = off;
    off += align256(static_cast<size_t>(pt[t]) * eb);
  }
  mp->ws_bytes = off;
  return TT_OK;
}

// ---- planning of the batched engine (pair_engine.cuh) ----
//
// For every contracted mode but the float64 last one, choose the evaluation
// order (0: E B_i first, 1: A_i^T E first) and the slices per panel g that
// minimise a model of the engine's time (eng_mode_cost).  The two autotuned
// knobs: `level` (0..2) caps the T panel at 1/4, 1/2 or all of the engine's
// budget, `rcap` (0 = none, else 1, 2, 4) caps the replica thread groups
// that split the second product.
inline int eng_r4(int v) { return (v + 3) & ~3; }
inline int eng_pow2_floor(int v) { return v <= 1 ? 1 : pow2_floor(v); }

struct EngGeom {
  int v, tiles_cap, tbuf, stage, wmax;
};
inline EngGeom eng_geom(int dtype) {
  if (dtype == TT_F64)
    return {EngLimits<double>::V, EngLimits<double>::TILES, EngLimits<double>::TBUF, EngLimits<double>::STAGE,
            EngLimits<double>::WMAX};
  return {EngLimits<float>::V, EngLimits<float>::TILES, EngLimits<float>::TBUF, EngLimits<float>::STAGE,
          EngLimits<float>::WMAX};
}

inline int eng_r8(int v) { return (v + 7) & ~7; }

// Largest slices per panel the engine accepts for a mode (stage width and
// T-panel budget r8(m) * r8(g n_pad) <= budget); mirrors pair_engine.cuh.
inline int eng_gmax(const EngGeom& eg, int m, int n, int u, int I, int budget) {
  const int n4 = eng_r4(n), u4 = eng_r4(u);
  const int gw = std::max(1, eg.wmax / std::max(n4, u4));
  const int gt = std::max(1, ((budget / eng_r8(m)) & ~7) / n4);
  return std::max(1, std::min({I, gw, gt}));
}

// Model time (per-thread multiply-adds) of one mode of sizes m, k, n, u with
// I slices in panels of g: one or two 4x4 tiles per thread (as the engine
// picks), k (GEMM1) and m (GEMM2, per slice of a replica group) steps per
// panel, plus a fixed cost per streamed chunk.
inline double eng_mode_cost(const EngGeom& eg, bool f64, int m, int k, int n, int u, int I, int g, int rcap = 0) {
  const int NT = kEngThreads;
  constexpr double kChunk = 200.0;  // stage hand-off and pipeline bubble per streamed chunk
  const int n_pad = eng_r4(n), u_pad = eng_r4(u), m_pad = eng_r4(m);
  const int lwf = eng_r4(g * n_pad) + eg.v, lws = g * u_pad + eg.v;
  const int kcf = eng_pow2_floor(std::min(32, eg.stage / lwf)), kcs = eng_pow2_floor(std::min(32, eg.stage / lws));
  const int tiles1 = (m_pad / 4) * (eng_r4(g * n_pad) / 4);
  const int tiles2 = (u_pad / 4) * (n_pad / 4);
  int rep = std::min(g, NT / 32);
  rep = std::min(rep, std::max(1, NT / tiles2));
  rep = std::min(rep, std::max(1, eg.tbuf / (eng_r8(u) * eng_r8(n))));
  if (rcap > 0) rep = std::min(rep, rcap);
  rep = eng_pow2_floor(rep);
  const int ntr = NT / rep;
  const bool one = f64 || (tiles1 <= NT && tiles2 <= ntr);  // one 4x4 tile per thread, else two
  const double fpk = one ? 16.0 : 32.0;                     // multiply-adds per thread per step
  auto panel = [&](int gc) {
    const double t1 = fpk * k + kChunk * ((k + kcf - 1) / kcf);
    const double t2 = ((gc + rep - 1) / rep) * fpk * m + kChunk * ((m + kcs - 1) / kcs);
    return t1 + t2;
  };
  const int full = I / g, rest = I - full * g;
  double t = full * panel(g) + (rest > 0 ? panel(rest) : 0.0);
  t += 4.0 * rep * ((u * (n_pad / 4) + NT - 1) / NT);  // reduction of the replica partials
  return t;
}

// Tile configuration codes of the batched engine: level + 3 * rcap index.
constexpr int kTileConfigs = 12;
constexpr int kDefaultTileConfig = 2;  // full panel budget, no replica cap
inline int config_level(int cfg) { return cfg % 3; }
inline int config_rcap(int cfg) {
  static const int caps[4] = {0, 1, 2, 4};
  return caps[(cfg / 3) & 3];
}

inline void plan_engine_steps(SweepParams& p, int dtype, int cfg) {
  const int level = config_level(cfg), rcap = config_rcap(cfg);
  const EngGeom eg = eng_geom(dtype);
  const bool f64 = dtype == TT_F64;
  const int budget = eg.tiles_cap >> (2 - std::max(0, std::min(2, level)));
  const int n_modes = p.final_scalar ? p.n_steps - 1 : p.n_steps;
  static const int cand[] = {1, 2, 3, 4, 5, 6, 8, 10, 12, 16, 20, 24, 32, 48, 64, 96, 128};
  for (int j = 0; j < p.n_steps; ++j) {
    SweepStep& st = p.step[j];
    st.ord = 0;
    st.g = 1;
    st.rcap = rcap;
    if (j >= n_modes) continue;
    double best = 1e300;
    for (int ord = 0; ord < 2; ++ord) {
      const int m = ord == 0 ? st.rin_x : st.rin_y, k = ord == 0 ? st.rin_y : st.rin_x;
      const int n = ord == 0 ? st.rout_y : st.rout_x, u = ord == 0 ? st.rout_x : st.rout_y;
      const int gmax = eng_gmax(eg, m, n, u, st.I, budget);
      auto consider = [&](int g) {
        const double c = eng_mode_cost(eg, f64, m, k, n, u, st.I, g, rcap);
        if (c < best) {
          best = c;
          st.ord = ord;
          st.g = g;
        }
      };
      for (int g : cand)
        if (g <= gmax) consider(g);
      consider(gmax);
    }
  }
}

// Flops of one contracted mode, the cheaper of the two evaluation orders.
inline double mode_flops(int rx, int rx2, int ry, int ry2, int I) {
  const double a = double(rx) * ry * I * ry2 + double(rx) * I * rx2 * ry2;
  const double b = double(rx) * ry * I * rx2 + double(ry) * I * rx2 * ry2;
  return 2.0 * std::min(a, b);
}

inline double sweep_flops(const SweepParams& p) {
  double f = 0.0;
  for (int j = 0; j < p.n_steps; ++j) {
    const SweepStep& s = p.step[j];
    f += mode_flops(s.rin_x, s.rout_x, s.rin_y, s.rout_y, s.I);
  }
  if (p.emit.enabled) {
    const EmitParams& e = p.emit;
    f += 2.0 * e.ra * e.I * e.rb * e.ry;
    for (int t = 0; t < e.n_copies; ++t) f += 0.25 * e.copy[t].r0 * e.copy[t].I * e.copy[t].r1;  // copy cost proxy
  }
  return f;
}

}  // namespace ttc
