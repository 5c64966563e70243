// Host orchestration of the tensor-core full contraction (tc_sweep.cu):
// operand conversion, tensor maps, and the chain of per-mode launches.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "host_plan.h"

namespace ttc {

struct TcPlan {
  int x3 = 0;           // split products
  int convert = 0;      // float32 cores converted to bfloat16 (hi, and lo when x3)
  int64_t elems_x[kMaxOrder], elems_y[kMaxOrder];
  size_t off_hx[kMaxOrder], off_hy[kMaxOrder], off_lx[kMaxOrder], off_ly[kMaxOrder];
  size_t off_env[2][3];  // [ping/pong][hi, lo, f32]
  size_t off_bmax[2], off_l[2], off_parts;
  size_t ws_bytes = 0;
};

static size_t a1k(size_t v) { return (v + 1023) & ~static_cast<size_t>(1023); }

// Precision routes: BF16 storage + NATIVE; F32 storage + BF16 (rounded) or BF16X3 (split).
int tc_full_plan(const tt_desc* x, const tt_desc* y, int prec, TcPlan* tp) {
  const int n = x->order;
  if (x->dtype == TT_BF16 && prec == TT_P_NATIVE) {
    tp->x3 = 0;
    tp->convert = 0;
  } else if (x->dtype == TT_F32 && (prec == TT_P_BF16 || prec == TT_P_BF16X3)) {
    tp->x3 = prec == TT_P_BF16X3;
    tp->convert = 1;
  } else {
    return TT_ERR_DTYPE;
  }
  if (n < 3) return TT_ERR_UNSUPPORTED;
  for (int k = 1; k < n; ++k) {
    const int rx = x->ranks[k], ry = y->ranks[k];
    if ((rx != 128 && rx != 256) || ry % 64 != 0 || ry > 256) return TT_ERR_UNSUPPORTED;
  }
  size_t off = 0;
  for (int k = 0; k < n; ++k) {
    tp->elems_x[k] = static_cast<int64_t>(x->ranks[k]) * x->modes[k] * x->ranks[k + 1];
    tp->elems_y[k] = static_cast<int64_t>(y->ranks[k]) * y->modes[k] * y->ranks[k + 1];
    if (tp->convert) {
      tp->off_hx[k] = off;
      off += a1k(tp->elems_x[k] * 2);
      tp->off_hy[k] = off;
      off += a1k(tp->elems_y[k] * 2);
      if (tp->x3) {
        tp->off_lx[k] = off;
        off += a1k(tp->elems_x[k] * 2);
        tp->off_ly[k] = off;
        off += a1k(tp->elems_y[k] * 2);
      }
    }
  }
  const size_t env = 256 * 256;
  for (int b = 0; b < 2; ++b) {
    tp->off_env[b][0] = off;
    off += a1k(env * 2);
    tp->off_env[b][1] = off;
    off += a1k(env * 2);
    tp->off_env[b][2] = off;
    off += a1k(env * 4);
    tp->off_bmax[b] = off;
    off += a1k(1024 * sizeof(int));
    tp->off_l[b] = off;
    off += 1024;
  }
  int imax = 1;
  for (int k = 0; k < n; ++k) imax = std::max(imax, x->modes[k]);
  tp->off_parts = off;  // one float64 partial per block of the last-mode kernel: 32 row blocks x ceil(I / 32)
  off += a1k(sizeof(double) * 32 * ((imax + 31) / 32));
  tp->ws_bytes = off;
  return TT_OK;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point, so the
// library does not link libcuda (it loads on machines without a driver).
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

static int make_map(CUtensorMap* m, const void* ptr, int r0, int I, int r1) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (enc == nullptr) return TT_ERR_CUDA;
  cuuint64_t gdim[3] = {static_cast<cuuint64_t>(r1), static_cast<cuuint64_t>(I), static_cast<cuuint64_t>(r0)};
  cuuint64_t gstride[2] = {static_cast<cuuint64_t>(r1) * 2, static_cast<cuuint64_t>(I) * r1 * 2};
  cuuint32_t box[3] = {64, 1, 64};
  cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(ptr), gdim,
                                            gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? TT_OK : TT_ERR_CUDA;
}

int tc_full_launch(const tt_desc* x, const tt_desc* y, int prec, double* out, int64_t* out_log2, int32_t* status,
                   void* ws, size_t ws_bytes, cudaStream_t s) {
  TcPlan tp;
  int rc = tc_full_plan(x, y, prec, &tp);
  if (rc != TT_OK) return rc;
  if (ws == nullptr || ws_bytes < tp.ws_bytes) return TT_ERR_WS;
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return TT_ERR_ARG;
  char* w = static_cast<char*>(ws);
  const int n = x->order;
  // bfloat16 operands (converted from float32 when needed)
  std::vector<const void*> hx(n), hy(n), lx(n), ly(n);
  for (int k = 0; k < n; ++k) {
    if (tp.convert) {
      hx[k] = w + tp.off_hx[k];
      hy[k] = w + tp.off_hy[k];
      lx[k] = tp.x3 ? w + tp.off_lx[k] : nullptr;
      ly[k] = tp.x3 ? w + tp.off_ly[k] : nullptr;
      if (tc_split(static_cast<const float*>(x->cores[k]), w + tp.off_hx[k], tp.x3 ? w + tp.off_lx[k] : nullptr,
                   tp.elems_x[k], s) != cudaSuccess ||
          tc_split(static_cast<const float*>(y->cores[k]), w + tp.off_hy[k], tp.x3 ? w + tp.off_ly[k] : nullptr,
                   tp.elems_y[k], s) != cudaSuccess)
        return TT_ERR_CUDA;
    } else {
      hx[k] = x->cores[k];
      hy[k] = y->cores[k];
      lx[k] = hx[k];
      ly[k] = hy[k];
    }
  }
  // first mode: float32 masters for the split variant, the bfloat16 operands otherwise
  const bool f32_ends = tp.x3 != 0;
  const void* x0 = f32_ends ? x->cores[0] : hx[0];
  const void* y0 = f32_ends ? y->cores[0] : hy[0];
  int cur = 0;
  if (tc_first(x0, y0, f32_ends, x->modes[0], x->ranks[1], y->ranks[1], reinterpret_cast<float*>(w + tp.off_env[0][2]),
               w + tp.off_env[0][0], w + tp.off_env[0][1], reinterpret_cast<int*>(w + tp.off_bmax[0]),
               reinterpret_cast<int64_t*>(w + tp.off_l[0]), status, s) != cudaSuccess)
    return TT_ERR_CUDA;
  int nbmax = x->ranks[1];
  for (int k = 1; k < n - 1; ++k) {
    TcModeParams p;
    memset(&p, 0, sizeof(p));
    const int I = x->modes[k];
    if (make_map(&p.gx_hi, hx[k], x->ranks[k], I, x->ranks[k + 1]) != TT_OK ||
        make_map(&p.gy_hi, hy[k], y->ranks[k], I, y->ranks[k + 1]) != TT_OK ||
        make_map(&p.gx_lo, lx[k], x->ranks[k], I, x->ranks[k + 1]) != TT_OK ||
        make_map(&p.gy_lo, ly[k], y->ranks[k], I, y->ranks[k + 1]) != TT_OK)
      return TT_ERR_CUDA;
    p.x3 = tp.x3;
    p.rx = x->ranks[k];
    p.rx2 = x->ranks[k + 1];
    p.ry = y->ranks[k];
    p.ry2 = y->ranks[k + 1];
    p.I = I;
    p.e_hi = reinterpret_cast<const __nv_bfloat16*>(w + tp.off_env[cur][0]);
    p.e_lo = reinterpret_cast<const __nv_bfloat16*>(w + tp.off_env[cur][1]);
    p.bmax_in = reinterpret_cast<const int*>(w + tp.off_bmax[cur]);
    p.n_bmax_in = nbmax;
    p.l_in = reinterpret_cast<const int64_t*>(w + tp.off_l[cur]);
    const int nxt = 1 - cur;
    p.eo_hi = reinterpret_cast<__nv_bfloat16*>(w + tp.off_env[nxt][0]);
    p.eo_lo = reinterpret_cast<__nv_bfloat16*>(w + tp.off_env[nxt][1]);
    p.eo_f32 = reinterpret_cast<float*>(w + tp.off_env[nxt][2]);
    p.bmax_out = reinterpret_cast<int*>(w + tp.off_bmax[nxt]);
    p.l_out = reinterpret_cast<int64_t*>(w + tp.off_l[nxt]);
    p.status = status;
    int C = tc_cluster_size(tp.x3 != 0, pow2_floor(std::min(16, I)));
    if (C < 1) return TT_ERR_CUDA;
    while (p.rx2 % C != 0) C /= 2;
    if (tc_mode(p, C, s) != cudaSuccess) return TT_ERR_CUDA;
    nbmax = C * (p.ry2 / 64);
    cur = nxt;
  }
  const void* xl = f32_ends ? x->cores[n - 1] : hx[n - 1];
  const void* yl = f32_ends ? y->cores[n - 1] : hy[n - 1];
  if (tc_last(reinterpret_cast<const float*>(w + tp.off_env[cur][2]), xl, yl, f32_ends, x->modes[n - 1], x->ranks[n - 1],
              y->ranks[n - 1], reinterpret_cast<double*>(w + tp.off_parts),
              reinterpret_cast<const int64_t*>(w + tp.off_l[cur]), out, out_log2, status, s) != cudaSuccess)
    return TT_ERR_CUDA;
  return TT_OK;
}

}  // namespace ttc

namespace ttc {
size_t tc_full_ws(const tt_desc* x, const tt_desc* y, int prec, int* rc) {
  TcPlan tp;
  *rc = tc_full_plan(x, y, prec, &tp);
  return *rc == TT_OK ? tp.ws_bytes : 0;
}
}  // namespace ttc
