// Host side of the C ABI: validation, workspace sizing and kernel dispatch.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ttc_internal.h"

namespace ttc {

std::atomic<uint64_t> g_launches{0};

static int elem_bytes(int dtype) {
  switch (dtype) {
    case TT_F64: return 8;
    case TT_F32: return 4;
    case TT_BF16: return 2;
    default: return 0;
  }
}

static size_t align256(size_t v) { return (v + 255) & ~static_cast<size_t>(255); }

int check_desc(const tt_desc* d) {
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
int check_pair(const tt_desc* x, const tt_desc* y, const uint8_t* mask) {
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

// ("lead", s) -> +s, ("trail", s) -> -s - 1... encoded as side (0 lead, 1 trail) and s; -1 if neither.
int end_block(const uint8_t* mask, int n, int* s_out) {
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

static int max_rank(const tt_desc* d) {
  int r = 1;
  for (int k = 0; k <= d->order; ++k) r = std::max(r, d->ranks[k]);
  return r;
}

static int rank_cap(int dtype) { return dtype == TT_F64 ? 64 : 128; }

static int pow2_floor(int v) {
  int c = 1;
  while (c * 2 <= v) c *= 2;
  return c;
}

// Fill a left-to-right sweep over modes [k0, k1) of (x, y).
static void fill_left(SweepParams& p, const tt_desc* x, const tt_desc* y, int k0, int k1) {
  p.n_steps = k1 - k0;
  p.transposed = 0;
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
static void fill_right(SweepParams& p, const tt_desc* x, const tt_desc* y, int k0, int k1) {
  p.n_steps = k1 - k0;
  p.transposed = 1;
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

static int sweep_max_rank(const SweepParams& p) {
  int r = std::max(p.rx0, p.ry0);
  for (int j = 0; j < p.n_steps; ++j)
    r = std::max({r, p.step[j].rin_x, p.step[j].rout_x, p.step[j].rin_y, p.step[j].rout_y});
  if (p.emit.enabled) r = std::max({r, p.emit.ra, p.emit.rb, p.emit.ry});
  return r;
}

static int sweep_max_mode(const SweepParams& p) {
  int m = 1;
  for (int j = 0; j < p.n_steps; ++j) m = std::max(m, p.step[j].I);
  if (p.emit.enabled) m = std::max(m, p.emit.I);
  return m;
}

int launch_sweep(const SweepParams& p, int dtype, cudaStream_t s) {
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

static int chain_plan(const tt_desc* x, const tt_desc* y, const uint8_t* mask, ChainPlan* cp) {
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

}  // namespace ttc

using namespace ttc;

extern "C" {

const char* tt_error_string(int code) {
  switch (code) {
    case TT_OK: return "ok";
    case TT_ERR_ARG: return "invalid argument";
    case TT_ERR_SHAPE: return "shape mismatch";
    case TT_ERR_DTYPE: return "dtype or precision not provided";
    case TT_ERR_LAYOUT: return "layout needs the contracted modes to form an end block";
    case TT_ERR_TOO_LARGE: return "rank, mode size or output exceeds the supported cap";
    case TT_ERR_WS: return "workspace too small";
    case TT_ERR_CUDA: return "CUDA runtime error";
    case TT_ERR_UNSUPPORTED: return "not implemented in this build";
    default: return "unknown error";
  }
}

uint64_t tt_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int tt_workspace_bytes(int op, const tt_desc* x, const tt_desc* y, const uint8_t* mask, int layout, int prec,
                       size_t* bytes) {
  if (bytes == nullptr) return TT_ERR_ARG;
  *bytes = 0;
  if (op == TT_OP_FULL) {
    const int rc = check_pair(x, y, nullptr);
    return rc;
  }
  if (op == TT_OP_PARTIAL) {
    if (mask == nullptr) return TT_ERR_ARG;
    int rc = check_pair(x, y, mask);
    if (rc != TT_OK) return rc;
    if (layout != TT_LAYOUT_CHAIN) return TT_ERR_UNSUPPORTED;
    ChainPlan cp;
    rc = chain_plan(x, y, mask, &cp);
    if (rc != TT_OK) return rc;
    *bytes = 0;  // the environment K stays in shared memory
    return TT_OK;
  }
  (void)prec;
  return TT_ERR_UNSUPPORTED;
}

int tt_contract_full(const tt_desc* x, const tt_desc* y, int prec, double* out_dev, int64_t* out_log2_dev,
                     int32_t* status_dev, void* ws, size_t ws_bytes, tt_stream stream) {
  (void)ws;
  (void)ws_bytes;
  int rc = check_pair(x, y, nullptr);
  if (rc != TT_OK) return rc;
  if (out_dev == nullptr) return TT_ERR_ARG;
  if (prec != TT_P_NATIVE) return TT_ERR_UNSUPPORTED;
  if (x->dtype == TT_BF16) return TT_ERR_UNSUPPORTED;
  SweepParams p;
  memset(&p, 0, sizeof(p));
  fill_left(p, x, y, 0, x->order);
  p.final_scalar = 1;
  p.renorm_bits = x->dtype == TT_F64 ? kRenormBitsF64 : kRenormBitsF32;
  p.z_out = out_dev;
  p.z_out_log2 = out_log2_dev;
  p.status = status_dev;
  return launch_sweep(p, x->dtype, reinterpret_cast<cudaStream_t>(stream));
}

int tt_partial_shape(const tt_desc* x, const tt_desc* y, const uint8_t* mask, int layout, int32_t* z_order,
                     int32_t* z_modes, int32_t* z_ranks, int32_t* z_perm) {
  if (mask == nullptr || z_order == nullptr || z_modes == nullptr || z_ranks == nullptr || z_perm == nullptr)
    return TT_ERR_ARG;
  int rc = check_pair(x, y, mask);
  if (rc != TT_OK) return rc;
  if (layout == TT_LAYOUT_CHAIN) {
    ChainPlan cp;
    rc = chain_plan(x, y, mask, &cp);
    if (rc != TT_OK) return rc;
    *z_order = cp.order;
    for (int p = 0; p < cp.order; ++p) {
      z_modes[p] = cp.modes[p];
      z_ranks[p] = cp.ranks[p];
      z_perm[p] = cp.perm[p];
    }
    z_ranks[cp.order] = 1;
    return TT_OK;
  }
  if (layout == TT_LAYOUT_MERGED) {
    const int n = x->order;
    int m = 0;
    int free_pos[kMaxOrder];
    for (int k = 0; k < n; ++k)
      if (!mask[k]) free_pos[m++] = k;
    if (m == 0) return TT_ERR_ARG;
    *z_order = m;
    z_ranks[0] = 1;
    for (int t = 0; t < m; ++t) {
      const int f = free_pos[t];
      z_modes[t] = x->modes[f] * y->modes[f];
      z_ranks[t + 1] = t + 1 < m ? x->ranks[free_pos[t + 1]] * y->ranks[free_pos[t + 1]] : 1;
      z_perm[2 * t] = t;
      z_perm[2 * t + 1] = m + t;
    }
    return TT_OK;
  }
  return TT_ERR_ARG;
}

int tt_contract_partial(const tt_desc* x, const tt_desc* y, const uint8_t* mask, int layout, int prec,
                        const tt_desc* z, int64_t* z_log2_dev, int32_t* status_dev, void* ws, size_t ws_bytes,
                        tt_stream stream) {
  if (mask == nullptr) return TT_ERR_ARG;
  int rc = check_pair(x, y, mask);
  if (rc != TT_OK) return rc;
  if (prec != TT_P_NATIVE) return TT_ERR_UNSUPPORTED;
  if (x->dtype == TT_BF16) return TT_ERR_UNSUPPORTED;
  if (layout != TT_LAYOUT_CHAIN) return TT_ERR_UNSUPPORTED;
  ChainPlan cp;
  rc = chain_plan(x, y, mask, &cp);
  if (rc != TT_OK) return rc;
  rc = check_desc(z);
  if (rc != TT_OK) return rc;
  if (z->order != cp.order || z->dtype != x->dtype) return TT_ERR_SHAPE;
  for (int p = 0; p < cp.order; ++p)
    if (z->modes[p] != cp.modes[p] || z->ranks[p] != cp.ranks[p]) return TT_ERR_SHAPE;
  (void)ws;
  (void)ws_bytes;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int n = cp.n, m = cp.m, sS = cp.s;

  SweepParams p;
  memset(&p, 0, sizeof(p));
  // 1. K = environment over the contracted block (empty block: K = [1])
  if (sS > 0) {
    if (cp.side == 0) fill_left(p, x, y, 0, sS);
    else fill_right(p, x, y, m, n);
  }
  p.rx0 = 1;
  p.ry0 = 1;
  p.final_scalar = 0;
  p.renorm_bits = x->dtype == TT_F64 ? kRenormBitsF64 : kRenormBitsF32;
  p.status = status_dev;

  // 2. boundary core C, fused behind the sweep
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

  // 3. free cores
  auto add = [&](const void* src, void* dst, int r0, int I, int r1, int swap) -> int {
    if (!swap && src == dst) return TT_OK;
    if (swap && src == dst) return TT_ERR_ARG;
    CopyTask& t = ep.copy[ep.n_copies++];
    t.src = src;
    t.dst = dst;
    t.r0 = r0;
    t.I = I;
    t.r1 = r1;
    t.swap = swap;
    return TT_OK;
  };
  if (cp.side == 0) {
    for (int q = 0; q < m - 1; ++q) {
      const int k = n - 1 - q;
      if (add(x->cores[k], z->cores[q], x->ranks[k], x->modes[k], x->ranks[k + 1], 1) != TT_OK) return TT_ERR_ARG;
    }
    for (int q = 0; q < m; ++q) {
      const int k = sS + q;
      add(y->cores[k], z->cores[m + q], y->ranks[k], y->modes[k], y->ranks[k + 1], 0);
    }
  } else {
    for (int q = 0; q < m - 1; ++q) add(x->cores[q], z->cores[q], x->ranks[q], x->modes[q], x->ranks[q + 1], 0);
    for (int q = 0; q < m; ++q) {
      const int k = m - 1 - q;
      if (add(y->cores[k], z->cores[m + q], y->ranks[k], y->modes[k], y->ranks[k + 1], 1) != TT_OK) return TT_ERR_ARG;
    }
  }
  return launch_sweep(p, x->dtype, s);
}

int tt_batch_plan(const tt_batch* batch, tt_plan** plan, size_t* packed_bytes, size_t* ws_bytes) {
  (void)batch;
  (void)plan;
  (void)packed_bytes;
  (void)ws_bytes;
  return TT_ERR_UNSUPPORTED;
}

int tt_batch_pack(const tt_plan* plan, void* packed_host, size_t packed_bytes) {
  (void)plan;
  (void)packed_host;
  (void)packed_bytes;
  return TT_ERR_UNSUPPORTED;
}

int tt_contract_batched(const tt_plan* plan, const void* packed_dev, double* out_dev, int64_t* out_log2_dev,
                        int32_t* status_dev, void* ws, size_t ws_bytes, tt_stream stream) {
  (void)plan;
  (void)packed_dev;
  (void)out_dev;
  (void)out_log2_dev;
  (void)status_dev;
  (void)ws;
  (void)ws_bytes;
  (void)stream;
  return TT_ERR_UNSUPPORTED;
}

int tt_plan_info(const tt_plan* plan, int32_t p, int32_t* n_pairs, int32_t* tile_config) {
  (void)plan;
  (void)p;
  (void)n_pairs;
  (void)tile_config;
  return TT_ERR_UNSUPPORTED;
}

void tt_plan_free(tt_plan* plan) { (void)plan; }

int tt_contract_backward(const tt_desc* x, const tt_desc* y, const uint8_t* mask, int layout, int prec,
                         const double* cot_dev, const tt_desc* dz, const tt_desc* gx, const tt_desc* gy,
                         int32_t ckpt_stride, int32_t* status_dev, void* ws, size_t ws_bytes, tt_stream stream) {
  (void)x;
  (void)y;
  (void)mask;
  (void)layout;
  (void)prec;
  (void)cot_dev;
  (void)dz;
  (void)gx;
  (void)gy;
  (void)ckpt_stride;
  (void)status_dev;
  (void)ws;
  (void)ws_bytes;
  (void)stream;
  return TT_ERR_UNSUPPORTED;
}

}  // extern "C"
