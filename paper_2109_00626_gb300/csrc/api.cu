// Host side of the C ABI: validation, workspace sizing and kernel dispatch.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "host_plan.h"

namespace ttc {

std::atomic<uint64_t> g_launches{0};

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
  build_full(x, y, out_dev, out_log2_dev, status_dev, &p);
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
  rc = check_chain_output(x, cp, z);
  if (rc != TT_OK) return rc;
  (void)ws;
  (void)ws_bytes;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SweepParams p;
  rc = build_partial(x, y, cp, z, z_log2_dev, status_dev, &p);
  if (rc != TT_OK) return rc;
  return launch_sweep(p, x->dtype, s);
}

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
