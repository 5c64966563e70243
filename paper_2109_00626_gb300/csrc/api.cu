// Host side of the C ABI: validation, workspace sizing and kernel dispatch.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "host_plan.h"

namespace ttc {

std::atomic<uint64_t> g_launches{0};

}  // namespace ttc

using namespace ttc;

namespace ttc {

struct TcPlan;
int tc_full_plan(const tt_desc* x, const tt_desc* y, int prec, TcPlan* tp);
int tc_full_launch(const tt_desc* x, const tt_desc* y, int prec, double* out, int64_t* out_log2, int32_t* status,
                   void* ws, size_t ws_bytes, cudaStream_t s);
size_t tc_full_ws(const tt_desc* x, const tt_desc* y, int prec, int* rc);

// Auxiliary streams of one device for the independent per-core chains of a
// merged-layout contraction: forked from the caller's stream by an event and
// joined back into it by one event per auxiliary stream, so the contraction
// stays ordered on the caller's stream (and captures into a graph as such).
struct ForkStreams {
  static constexpr int kAux = 3;
  cudaStream_t aux[kAux];
  cudaEvent_t fork, done[kAux];
  bool ok = false;
};
static std::mutex g_fork_mu;  // guards g_fork and the use of its events
static ForkStreams g_fork[64];

static ForkStreams* fork_streams() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  ForkStreams& f = g_fork[dev];
  if (!f.ok) {
    for (int i = 0; i < ForkStreams::kAux; ++i)
      if (cudaStreamCreateWithFlags(&f.aux[i], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&f.done[i], cudaEventDisableTiming) != cudaSuccess)
        return nullptr;
    if (cudaEventCreateWithFlags(&f.fork, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    f.ok = true;
  }
  return &f;
}

// Output core t of a merged-layout contraction on stream s (see merged.cu).
static int merged_core(const tt_desc* x, const tt_desc* y, const tt_desc* z, const MergedPlan& mp, int t, char* w,
                       int32_t* status_dev, cudaStream_t s) {
  const int n = x->order;
  const int f0 = mp.free_pos[0];
  const int f = mp.free_pos[t];
  const int k0 = f + 1, k1 = mp.run_k1[t];
  const bool run = k1 > k0;
  const bool trail = run && k1 == n;
  const int rx = x->ranks[f], ry = y->ranks[f], I = x->modes[f], J = y->modes[f];
  const int rx2 = x->ranks[f + 1], ry2 = y->ranks[f + 1];
  const int C = x->ranks[k1] * y->ranks[k1];
  int64_t* slots = reinterpret_cast<int64_t*>(w + mp.off_slots);
  int64_t* emax = slots + 1 + kMergedSlotsPerCore * t;  // M; then P, W_0, V
  void* mbuf = w + mp.off_m[t];
  // the run's map M on the right leg: E_R of a right-to-left sweep for a
  // trailing run (one scale), the transfer matrix otherwise (a scale per row)
  const int64_t* mexp = emax;
  if (trail) {
    SweepParams p;
    memset(&p, 0, sizeof(p));
    fill_right(p, x, y, k0, n);
    p.rx0 = 1;
    p.ry0 = 1;
    p.renorm_bits = x->dtype == TT_F64 ? kRenormBitsF64 : kRenormBitsF32;
    p.e_out = mbuf;
    p.e_out_log2 = emax;
    p.status = status_dev;
    const int rc = launch_sweep(p, x->dtype, s);
    if (rc != TT_OK) return rc;
  } else if (run) {
    if (cudaMemsetAsync(emax, 0xC0, sizeof(int64_t), s) != cudaSuccess) return TT_ERR_CUDA;
    TransferParams tp;
    memset(&tp, 0, sizeof(tp));
    SweepParams sp;
    memset(&sp, 0, sizeof(sp));
    fill_left(sp, x, y, k0, k1);
    tp.n_steps = sp.n_steps;
    memcpy(tp.step, sp.step, sizeof(tp.step));
    tp.m = mbuf;
    tp.mexp = reinterpret_cast<int64_t*>(w + mp.off_mexp[t]);
    tp.emax = emax;
    tp.status = status_dev;
    if (launch_transfer(tp, x->dtype, s) != cudaSuccess) return TT_ERR_CUDA;
    mexp = tp.mexp;
  }
  if (t == 0) {
    // the left core with E_L, the left environment of the contracted modes
    // before f_0 (none when f_0 = 0), folded in
    if (f0 > 0) {
      SweepParams p;
      memset(&p, 0, sizeof(p));
      fill_left(p, x, y, 0, f0);
      p.rx0 = 1;
      p.ry0 = 1;
      p.renorm_bits = x->dtype == TT_F64 ? kRenormBitsF64 : kRenormBitsF32;
      p.e_out = w + mp.off_el;
      p.e_out_log2 = slots;
      p.status = status_dev;
      const int rc = launch_sweep(p, x->dtype, s);
      if (rc != TT_OK) return rc;
    }
    KronParams kp;
    memset(&kp, 0, sizeof(kp));
    kp.gx = x->cores[f];
    kp.gy = y->cores[f];
    kp.rx = rx;
    kp.ry = ry;
    kp.I = I;
    kp.J = J;
    kp.rx2 = rx2;
    kp.ry2 = ry2;
    kp.out = run ? static_cast<void*>(w + mp.off_w0) : z->cores[0];
    kp.el = f0 > 0 ? w + mp.off_el : nullptr;
    kp.el_log2 = f0 > 0 ? slots : nullptr;
    kp.tmp = w + mp.off_v;
    kp.vexp = emax + 3;
    kp.wexp = emax + 2;
    kp.scale_out = run ? 0 : 1;  // with a run the scale is applied after M
    kp.status = status_dev;
    if (cudaMemsetAsync(kp.vexp, 0xC0, sizeof(int64_t), s) != cudaSuccess) return TT_ERR_CUDA;
    if (launch_kron0(kp, 1, x->dtype, s) != cudaSuccess || launch_kron0(kp, 2, x->dtype, s) != cudaSuccess)
      return TT_ERR_CUDA;
    if (run) {
      ScaledGemmParams g;
      memset(&g, 0, sizeof(g));
      g.a = w + mp.off_w0;
      g.lda = static_cast<int64_t>(rx2) * ry2;
      g.b = mbuf;
      g.ldb = C;
      g.out = z->cores[0];
      g.ldo = C;
      g.rows = I * J;
      g.K = rx2 * ry2;
      g.C = C;
      g.nz = 1;
      g.mexp = mexp;
      g.es = trail ? 0 : 1;
      g.emax = emax;
      g.out_log2 = kp.wexp;
      g.status = status_dev;
      if (launch_scaled_gemm(g, x->dtype, s) != cudaSuccess) return TT_ERR_CUDA;
    }
    return TT_OK;
  }
  ZRowsParams zp;
  memset(&zp, 0, sizeof(zp));
  zp.gx = x->cores[f];
  zp.gy = y->cores[f];
  zp.out = z->cores[t];
  zp.rx = rx;
  zp.ry = ry;
  zp.I = I;
  zp.J = J;
  zp.rx2 = rx2;
  zp.ry2 = ry2;
  zp.C = C;
  zp.status = status_dev;
  if (run) {
    // P[a][i][b'][col] = sum_a' Gx[a][i][a'] M[(a', b')][col]
    ScaledGemmParams g;
    memset(&g, 0, sizeof(g));
    g.a = x->cores[f];
    g.lda = rx2;
    g.b = mbuf;
    g.ldb = static_cast<int64_t>(ry2) * C;
    g.bz = C;
    g.out = w + mp.off_p[t];
    g.ldo = static_cast<int64_t>(ry2) * C;
    g.oz = C;
    g.rows = rx * I;
    g.K = rx2;
    g.C = C;
    g.nz = ry2;
    g.mexp = mexp;
    g.es = trail ? 0 : ry2;
    g.ez = trail ? 0 : 1;
    g.emax = emax;
    g.oexp = emax + 1;
    g.status = status_dev;
    if (cudaMemsetAsync(g.oexp, 0xC0, sizeof(int64_t), s) != cudaSuccess) return TT_ERR_CUDA;
    if (launch_scaled_gemm(g, x->dtype, s) != cudaSuccess) return TT_ERR_CUDA;
    zp.p = w + mp.off_p[t];
    zp.e = emax;
    zp.ep = emax + 1;
  }
  if (launch_zrows(zp, run, x->dtype, s) != cudaSuccess) return TT_ERR_CUDA;
  return TT_OK;
}

static int contract_merged(const tt_desc* x, const tt_desc* y, const uint8_t* mask, const tt_desc* z,
                           int64_t* z_log2_dev, int32_t* status_dev, void* ws, size_t ws_bytes, tt_stream stream) {
  MergedPlan mp;
  int rc = merged_plan(x, y, mask, &mp);
  if (rc != TT_OK) return rc;
  rc = check_desc(z);
  if (rc != TT_OK) return rc;
  if (z->order != mp.m || z->dtype != x->dtype) return TT_ERR_SHAPE;
  {
    int32_t order = 0, modes[2 * kMaxOrder], ranks[2 * kMaxOrder + 1], perm[2 * kMaxOrder];
    rc = tt_partial_shape(x, y, mask, TT_LAYOUT_MERGED, &order, modes, ranks, perm);
    if (rc != TT_OK) return rc;
    for (int t = 0; t < order; ++t)
      if (z->modes[t] != modes[t] || z->ranks[t] != ranks[t]) return TT_ERR_SHAPE;
  }
  if (ws_bytes < mp.ws_bytes || ws == nullptr) return TT_ERR_WS;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  // the output cores: independent chains, core 0 on the caller's stream and
  // the others on the auxiliary streams
  std::lock_guard<std::mutex> lock(g_fork_mu);
  ForkStreams* fs = mp.m > 1 ? fork_streams() : nullptr;
  if (mp.m > 1 && fs == nullptr) return TT_ERR_CUDA;
  const int n_aux = fs != nullptr ? std::min(ForkStreams::kAux, mp.m - 1) : 0;
  if (n_aux > 0) {
    if (cudaEventRecord(fs->fork, s) != cudaSuccess) return TT_ERR_CUDA;
    for (int i = 0; i < n_aux; ++i)
      if (cudaStreamWaitEvent(fs->aux[i], fs->fork, 0) != cudaSuccess) return TT_ERR_CUDA;
  }
  for (int t = 0; t < mp.m && rc == TT_OK; ++t)
    rc = merged_core(x, y, z, mp, t, w, status_dev, t == 0 ? s : fs->aux[(t - 1) % n_aux]);
  // join even after an error, so that no work is left unordered behind the caller's stream
  for (int i = 0; i < n_aux; ++i)
    if (cudaEventRecord(fs->done[i], fs->aux[i]) != cudaSuccess || cudaStreamWaitEvent(s, fs->done[i], 0) != cudaSuccess)
      rc = rc == TT_OK ? TT_ERR_CUDA : rc;
  if (rc != TT_OK) return rc;
  if (z_log2_dev != nullptr && cudaMemsetAsync(z_log2_dev, 0, sizeof(int64_t), s) != cudaSuccess) return TT_ERR_CUDA;
  return TT_OK;
}

}  // namespace ttc

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
    int rc = check_pair(x, y, nullptr);
    if (rc != TT_OK) return rc;
    if (x->dtype == TT_BF16 || prec == TT_P_BF16 || prec == TT_P_BF16X3) {
      *bytes = tc_full_ws(x, y, prec, &rc);
      return rc;
    }
    if (prec != TT_P_NATIVE && prec != TT_P_TF32X3 && prec != TT_P_TF32) return TT_ERR_UNSUPPORTED;
    if (x->order >= 2) *bytes = two_sided_layout(x, y).bytes;  // both-ends sweep
    if (prec == TT_P_NATIVE && full_is_r1(x, y)) *bytes = std::max(*bytes, full_r1_bytes(x));
    return TT_OK;
  }
  if (op == TT_OP_PARTIAL) {
    if (mask == nullptr) return TT_ERR_ARG;
    int rc = check_pair(x, y, mask);
    if (rc != TT_OK) return rc;
    if (layout == TT_LAYOUT_MERGED) {
      MergedPlan mp;
      rc = merged_plan(x, y, mask, &mp);
      if (rc != TT_OK) return rc;
      *bytes = mp.ws_bytes;
      return TT_OK;
    }
    if (layout != TT_LAYOUT_CHAIN) return TT_ERR_ARG;
    ChainPlan cp;
    rc = chain_plan(x, y, mask, &cp);
    if (rc != TT_OK) return rc;
    *bytes = 0;  // the environment K stays in shared memory
    return TT_OK;
  }
  if (op == TT_OP_BACKWARD) {
    BackwardPlan bp;
    const int rc = backward_plan(x, y, mask, layout, prec, 0, &bp);
    if (rc != TT_OK) return rc;
    *bytes = bp.ws_bytes;
    return TT_OK;
  }
  return TT_ERR_ARG;
}

int tt_contract_full(const tt_desc* x, const tt_desc* y, int prec, double* out_dev, int64_t* out_log2_dev,
                     int32_t* status_dev, void* ws, size_t ws_bytes, tt_stream stream) {
  int rc = check_pair(x, y, nullptr);
  if (rc != TT_OK) return rc;
  if (out_dev == nullptr) return TT_ERR_ARG;
  if (x->dtype == TT_BF16 || prec == TT_P_BF16 || prec == TT_P_BF16X3)
    return tc_full_launch(x, y, prec, out_dev, out_log2_dev, status_dev, ws, ws_bytes,
                          reinterpret_cast<cudaStream_t>(stream));
  const bool tf32 = prec == TT_P_TF32X3 || prec == TT_P_TF32;
  if (prec != TT_P_NATIVE && !tf32) return TT_ERR_UNSUPPORTED;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SweepParams p;
  build_full(x, y, out_dev, out_log2_dev, status_dev, &p);
  const int rmax = sweep_max_rank(p);
  if (tf32) {
    if (x->dtype != TT_F32) return TT_ERR_DTYPE;
    if (rmax > kTf32MaxRank) return TT_ERR_UNSUPPORTED;
    const bool x3 = prec == TT_P_TF32X3;
    const int want = pow2_floor(std::min(16, sweep_max_mode(p)));
    const int C = tf32_cluster_size(want);
    if (C < 1) return TT_ERR_CUDA;
    if (x->order >= 2 && ws != nullptr && C >= 1) {
      const TwoSidedLayout L = two_sided_layout(x, y);
      if (ws_bytes >= L.bytes) {
        TwoSidedParams tp;
        build_two_sided(x, y, L, ws, out_dev, out_log2_dev, status_dev, &tp);
        if (cudaMemsetAsync(tp.counter, 0, 128, s) != cudaSuccess) return TT_ERR_CUDA;  // join counters
        return launch_tf32_two_sided(tp, x3, C, s) == cudaSuccess ? TT_OK : TT_ERR_CUDA;
      }
    }
    return launch_tf32_sweep(p, x3, C, s) == cudaSuccess ? TT_OK : TT_ERR_CUDA;
  }
  if (full_is_r1(x, y) && ws != nullptr && ws_bytes >= full_r1_bytes(x)) {
    // Y of rank 1: fold X's cores with y, then one chain of vector-matrix products
    AdjR1Params rp;
    memset(&rp, 0, sizeof(rp));
    rp.n = x->order;
    for (int k = 0; k < x->order; ++k) {
      AdjStep& st = rp.step[k];
      st.gx = x->cores[k];
      st.gy = y->cores[k];
      st.I = x->modes[k];
      st.rx = x->ranks[k];
      st.rx2 = x->ranks[k + 1];
      st.ry = 1;
      st.ry2 = 1;
    }
    r1_fold_layout(x, rp.moff);
    rp.mbuf = ws;
    rp.renorm_bits = x->dtype == TT_F64 ? kRenormBitsF64 : kRenormBitsF32;
    rp.fwd = 1;
    rp.z_out = out_dev;
    rp.z_out_log2 = out_log2_dev;
    rp.status = status_dev;
    return launch_full_r1(rp, x->dtype, s) == cudaSuccess ? TT_OK : TT_ERR_CUDA;
  }
  if (rmax > rank_cap(x->dtype)) return TT_ERR_TOO_LARGE;
  if (x->order >= 2 && ws != nullptr) {
    // with a workspace, sweep from both ends on two clusters at once
    const TwoSidedLayout L = two_sided_layout(x, y);
    const int want = pow2_floor(std::min(16, sweep_max_mode(p)));
    const int C = sweep_cluster_size(rmax, elem_bytes(x->dtype), want);
    if (ws_bytes >= L.bytes && C >= 2) {
      TwoSidedParams tp;  // copied by the launch
      build_two_sided(x, y, L, ws, out_dev, out_log2_dev, status_dev, &tp);
      if (cudaMemsetAsync(tp.counter, 0, 128, s) != cudaSuccess) return TT_ERR_CUDA;  // join counters
      return launch_two_sided(tp, x->dtype, rmax, C, s) == cudaSuccess ? TT_OK : TT_ERR_CUDA;
    }
  }
  return launch_sweep(p, x->dtype, s);
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

// Chain-layout partial contraction; with bws set (a backward workspace laid
// out by bp), K and its scale -- and, for a leading block, the left-environment
// checkpoints of the adjoint -- are also written into it.
static int contract_chain(const tt_desc* x, const tt_desc* y, const uint8_t* mask, int prec, const tt_desc* z,
                          int64_t* z_log2_dev, char* bws, const BackwardPlan* bp, int32_t* status_dev,
                          tt_stream stream) {
  if (mask == nullptr) return TT_ERR_ARG;
  int rc = check_pair(x, y, mask);
  if (rc != TT_OK) return rc;
  const bool tf32 = prec == TT_P_TF32X3 || prec == TT_P_TF32;
  if (prec != TT_P_NATIVE && !(tf32 && bws == nullptr)) return TT_ERR_UNSUPPORTED;
  if (x->dtype == TT_BF16) return TT_ERR_UNSUPPORTED;
  if (tf32 && x->dtype != TT_F32) return TT_ERR_DTYPE;
  ChainPlan cp;
  rc = chain_plan(x, y, mask, &cp);
  if (rc != TT_OK) return rc;
  rc = check_chain_output(x, cp, z);
  if (rc != TT_OK) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SweepParams p;
  rc = build_partial(x, y, cp, z, z_log2_dev, status_dev, &p);
  if (rc != TT_OK) return rc;
  if (bws != nullptr) {
    p.e_out = bws + bp->off_k;
    p.e_out_log2 = reinterpret_cast<int64_t*>(bws + bp->off_klog2);
    if (cp.side == 0 && cp.s > 0) {
      // every left environment L_0 .. L_{s-1} of the block
      p.ckpt = bws + bp->off_ckpt;
      p.ckpt_log2 = reinterpret_cast<int64_t*>(bws + bp->off_ckpt_log2);
      p.ckpt_stride = 1;
      p.ckpt_n = cp.s;
      p.ckpt_elems = bp->env_elems;
    }
  }
  if (tf32) {
    if (sweep_max_rank(p) > kTf32MaxRank) return TT_ERR_UNSUPPORTED;
    const int C = tf32_cluster_size(pow2_floor(std::min(16, sweep_max_mode(p))));
    if (C < 1) return TT_ERR_CUDA;
    return launch_tf32_sweep(p, prec == TT_P_TF32X3, C, s) == cudaSuccess ? TT_OK : TT_ERR_CUDA;
  }
  return launch_sweep(p, x->dtype, s);
}

int tt_contract_partial(const tt_desc* x, const tt_desc* y, const uint8_t* mask, int layout, int prec,
                        const tt_desc* z, int64_t* z_log2_dev, int32_t* status_dev, void* ws, size_t ws_bytes,
                        tt_stream stream) {
  if (mask == nullptr) return TT_ERR_ARG;
  if (layout == TT_LAYOUT_MERGED) {
    const int rc = check_pair(x, y, mask);
    if (rc != TT_OK) return rc;
    if (prec != TT_P_NATIVE) return TT_ERR_UNSUPPORTED;
    if (x->dtype == TT_BF16) return TT_ERR_UNSUPPORTED;
    return contract_merged(x, y, mask, z, z_log2_dev, status_dev, ws, ws_bytes, stream);
  }
  if (layout != TT_LAYOUT_CHAIN) return TT_ERR_ARG;
  return contract_chain(x, y, mask, prec, z, z_log2_dev, nullptr, nullptr, status_dev, stream);
}

int tt_contract_partial_k(const tt_desc* x, const tt_desc* y, const uint8_t* mask, int prec, const tt_desc* z,
                          int64_t* z_log2_dev, int32_t* status_dev, void* ws, size_t ws_bytes, tt_stream stream) {
  BackwardPlan bp;
  const int rc = backward_plan(x, y, mask, TT_LAYOUT_CHAIN, prec, 0, &bp);
  if (rc != TT_OK) return rc;
  if (ws == nullptr || ws_bytes < bp.ws_bytes) return TT_ERR_WS;
  return contract_chain(x, y, mask, prec, z, z_log2_dev, static_cast<char*>(ws), &bp, status_dev, stream);
}
static int backward_impl(const tt_desc* x, const tt_desc* y, const uint8_t* mask, int layout, int prec,
                         const double* cot_dev, const tt_desc* dz, const tt_desc* gx, const tt_desc* gy,
                         int32_t ckpt_stride, int from_forward, int32_t* status_dev, void* ws, size_t ws_bytes,
                         tt_stream stream) {
  BackwardPlan bp;
  int rc = backward_plan(x, y, mask, layout, prec, ckpt_stride, &bp);
  if (rc != TT_OK) return rc;
  rc = check_same_shape(x, gx);
  if (rc == TT_OK) rc = check_same_shape(y, gy);
  if (rc != TT_OK) return rc;
  if (ws_bytes < bp.ws_bytes || (bp.ws_bytes > 0 && ws == nullptr)) return TT_ERR_WS;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  const int eb = elem_bytes(x->dtype);
  const int n = x->order;

  const int renorm_bits = x->dtype == TT_F64 ? kRenormBitsF64 : kRenormBitsF32;
  char* const lenv = w + bp.off_ckpt;
  int64_t* const lenv_log2 = reinterpret_cast<int64_t*>(w + bp.off_ckpt_log2);
  char* const fenv = w + bp.off_fenv;
  int64_t* const fenv_log2 = reinterpret_cast<int64_t*>(w + bp.off_fenv_log2);
  const int64_t env_bytes = bp.env_elems * eb;
  // Adjoint of the sweep over modes [k0, k1): L_1..L_{nb-1} by a left-to-right
  // sweep from the left seed (unless the forward sweep stored them),
  // F_{nb-1}..F_1 by a right-to-left sweep from the right seed, each storing
  // the environment before every mode, then the gradients of every slice.
  // leg-swapped copies of the block's cores [bp.k0, bp.k1) (the copy tasks,
  // and where each copy lands)
  const void* swx[kMaxOrder];
  const void* swy[kMaxOrder];
  SwapParams sp;
  memset(&sp, 0, sizeof(sp));
  {
    char* q = w + bp.off_swap;
    for (int k = bp.k0; k < bp.k1; ++k)
      for (int side = 0; side < 2; ++side) {
        const tt_desc* d = side == 0 ? x : y;
        CopyTask& t = sp.copy[sp.n_copies++];
        t.src = d->cores[k];
        t.dst = q;
        t.r0 = d->ranks[k];
        t.I = d->modes[k];
        t.r1 = d->ranks[k + 1];
        t.swap = 1;
        (side == 0 ? swx : swy)[k - bp.k0] = q;
        q += swap_core_bytes(d, k);
      }
  }
  bool swapped = false;  // set once the copies are enqueued
  auto adjoint_block = [&](int k0, int k1, const void* l_seed, const void* f_seed, int seed_parts, const double* cot,
                           bool l_given) -> int {
    const int nb = k1 - k0;
    if (!swapped && launch_swap_copies(sp, x->dtype, s) != cudaSuccess) return TT_ERR_CUDA;
    if (nb > 1 && !l_given) {
      SweepParams lp;
      memset(&lp, 0, sizeof(lp));
      fill_left(lp, x, y, k0, k1 - 1);
      lp.rx0 = x->ranks[k0];
      lp.ry0 = y->ranks[k0];
      lp.e_seed = l_seed;
      lp.e_seed_parts = seed_parts;
      lp.renorm_bits = renorm_bits;
      lp.ckpt = lenv;
      lp.ckpt_log2 = lenv_log2;
      lp.ckpt_stride = 1;
      lp.ckpt_n = nb - 1;
      lp.ckpt_elems = bp.env_elems;
      lp.e_out = lenv + (nb - 1) * env_bytes;
      lp.e_out_log2 = lenv_log2 + (nb - 1);
      lp.status = status_dev;
      const int r = launch_sweep(lp, x->dtype, s);
      if (r != TT_OK) return r;
    }
    if (nb > 1) {
      // F_{k+1} lands at slot k - k0 and its scale at slot nb - 1 - (k - k0);
      // the sweep runs left to right over the leg-swapped cores in reverse
      // order (E' = sum_i Gx_i E Gy_i^T)
      SweepParams rp;
      memset(&rp, 0, sizeof(rp));
      rp.n_steps = nb - 1;
      for (int j = 0; j < nb - 1; ++j) {
        const int k = k1 - 1 - j;
        SweepStep& st = rp.step[j];
        st.gx = swx[k - k0];
        st.gy = swy[k - k0];
        st.I = x->modes[k];
        st.rin_x = x->ranks[k + 1];
        st.rout_x = x->ranks[k];
        st.rin_y = y->ranks[k + 1];
        st.rout_y = y->ranks[k];
      }
      rp.rx0 = x->ranks[k1];
      rp.ry0 = y->ranks[k1];
      rp.e_seed = f_seed;
      rp.e_seed_parts = seed_parts;
      rp.renorm_bits = renorm_bits;
      rp.ckpt = fenv + (nb - 1) * env_bytes;
      rp.ckpt_log2 = fenv_log2;
      rp.ckpt_stride = 1;
      rp.ckpt_n = nb - 1;
      rp.ckpt_elems = -bp.env_elems;
      rp.e_out = fenv;
      rp.e_out_log2 = fenv_log2 + (nb - 1);
      rp.status = status_dev;
      const int r = launch_sweep(rp, x->dtype, s);
      if (r != TT_OK) return r;
    }
    AdjointParams ap;
    memset(&ap, 0, sizeof(ap));
    ap.n = nb;
    for (int j = 0; j < nb; ++j) {
      const int k = k0 + j;
      AdjStep& st = ap.step[j];
      st.gx = x->cores[k];
      st.gy = y->cores[k];
      st.dgx = gx->cores[k];
      st.dgy = gy->cores[k];
      st.I = x->modes[k];
      st.rx = x->ranks[k];
      st.rx2 = x->ranks[k + 1];
      st.ry = y->ranks[k];
      st.ry2 = y->ranks[k + 1];
      st.gxs = swx[j];
      ap.total_slices += st.I;
    }
    ap.l_seed = l_seed;
    ap.f_seed = f_seed;
    ap.seed_parts = seed_parts;
    ap.cot = cot;
    ap.lenv = lenv;
    ap.lenv_log2 = lenv_log2;
    ap.fenv = fenv;
    ap.fenv_log2 = fenv_log2;
    ap.env_elems = bp.env_elems;
    ap.status = status_dev;
    return launch_adjoint_grads(ap, x->dtype, bp.rmax, s) == cudaSuccess ? TT_OK : TT_ERR_CUDA;
  };

  if (mask == nullptr && bp.r1) {
    if (cot_dev == nullptr) return TT_ERR_ARG;
    AdjR1Params rp;
    memset(&rp, 0, sizeof(rp));
    rp.n = n;
    for (int k = 0; k < n; ++k) {
      AdjStep& st = rp.step[k];
      st.gx = x->cores[k];
      st.gy = y->cores[k];
      st.dgx = gx->cores[k];
      st.dgy = gy->cores[k];
      st.I = x->modes[k];
      st.rx = x->ranks[k];
      st.rx2 = x->ranks[k + 1];
      st.ry = 1;
      st.ry2 = 1;
    }
    rp.lvec = w + bp.off_lvec;
    rp.fvec = w + bp.off_fvec;
    rp.llog = reinterpret_cast<int64_t*>(w + bp.off_llog);
    rp.flog = reinterpret_cast<int64_t*>(w + bp.off_flog);
    rp.vstride = bp.vstride;
    rp.mbuf = w + bp.off_m;
    rp.mtbuf = w + bp.off_mt;
    r1_fold_layout(x, rp.moff);
    rp.renorm_bits = renorm_bits;
    rp.cot = cot_dev;
    rp.status = status_dev;
    return launch_adjoint_r1(rp, x->dtype, s) == cudaSuccess ? TT_OK : TT_ERR_CUDA;
  }
  if (mask == nullptr) {
    if (cot_dev == nullptr) return TT_ERR_ARG;
    return adjoint_block(0, n, nullptr, nullptr, 1, cot_dev, false);
  }

  const ChainPlan& cp = bp.cp;
  rc = check_chain_output(x, cp, dz);
  if (rc != TT_OK) return rc;
  const int m = cp.m, sS = cp.s;
  const void* kbuf = w + bp.off_k;
  const int64_t* klog2 = reinterpret_cast<int64_t*>(w + bp.off_klog2);
  void* dkbuf = w + bp.off_dk;

  // 1. K again (the environment over the contracted block), unless the
  //    forward pass left it in the workspace
  if (!from_forward) {
    SweepParams p;
    memset(&p, 0, sizeof(p));
    if (sS > 0) {
      if (cp.side == 0) fill_left(p, x, y, 0, sS);
      else fill_right(p, x, y, m, n);
    }
    p.rx0 = 1;
    p.ry0 = 1;
    p.renorm_bits = renorm_bits;
    p.e_out = w + bp.off_k;
    p.e_out_log2 = reinterpret_cast<int64_t*>(w + bp.off_klog2);
    p.status = status_dev;
    rc = launch_sweep(p, x->dtype, s);
    if (rc != TT_OK) return rc;
  }
  // 2. boundary-core gradient, dK, free-core gradients
  ChainAdjParams cap;
  memset(&cap, 0, sizeof(cap));
  const int kb = cp.side == 0 ? sS : m - 1;
  cap.gx = x->cores[kb];
  cap.ra = x->ranks[kb];
  cap.I = x->modes[kb];
  cap.rb = x->ranks[kb + 1];
  cap.lead = cp.side == 0 ? 1 : 0;
  cap.ry = cp.ky;
  cap.k = kbuf;
  cap.k_log2 = klog2;
  cap.dc = dz->cores[m - 1];
  cap.dgx = gx->cores[kb];
  cap.dk = sS > 0 ? dkbuf : nullptr;
  cap.dk_parts = std::max(1, std::min(cap.I, kDkGroups));
  cap.status = status_dev;
  auto add = [&](const void* src, void* dst, int r0, int I, int r1, int swap) {
    CopyTask& t = cap.copy[cap.n_copies++];
    t.src = src;
    t.dst = dst;
    t.r0 = r0;
    t.I = I;
    t.r1 = r1;
    t.swap = swap;
  };
  if (cp.side == 0) {
    for (int q = 0; q < m - 1; ++q) {
      const int k = n - 1 - q;  // dz[q] is [R_{k+1}][I_k][R_k]
      add(dz->cores[q], gx->cores[k], x->ranks[k + 1], x->modes[k], x->ranks[k], 1);
    }
    for (int q = 0; q < m; ++q) {
      const int k = sS + q;
      add(dz->cores[m + q], gy->cores[k], y->ranks[k], y->modes[k], y->ranks[k + 1], 0);
    }
  } else {
    for (int q = 0; q < m - 1; ++q) add(dz->cores[q], gx->cores[q], x->ranks[q], x->modes[q], x->ranks[q + 1], 0);
    for (int q = 0; q < m; ++q) {
      const int k = m - 1 - q;  // dz[m+q] is [R^y_{k+1}][I_k][R^y_k]
      add(dz->cores[m + q], gy->cores[k], y->ranks[k + 1], y->modes[k], y->ranks[k], 1);
    }
  }
  if (sS > 0 && cap.n_copies + sp.n_copies <= kMaxCopies) {
    // the leg-swapped copies ride along with the free-core copies
    for (int t = 0; t < sp.n_copies; ++t) cap.copy[cap.n_copies++] = sp.copy[t];
    swapped = true;
  }
  if (launch_chain_adjoint(cap, x->dtype, s) != cudaSuccess) return TT_ERR_CUDA;
  // 3. adjoint of the sweep over the contracted block, seeded with dK (the
  //    sum of the chain adjoint's partials); for a leading block the forward
  //    pass of tt_contract_partial_k stored the left environments
  if (sS > 0) {
    if (cp.side == 0) return adjoint_block(0, sS, nullptr, dkbuf, cap.dk_parts, nullptr, from_forward != 0);
    return adjoint_block(m, n, dkbuf, nullptr, cap.dk_parts, nullptr, false);
  }
  return TT_OK;
}

int tt_contract_backward(const tt_desc* x, const tt_desc* y, const uint8_t* mask, int layout, int prec,
                         const double* cot_dev, const tt_desc* dz, const tt_desc* gx, const tt_desc* gy,
                         int32_t ckpt_stride, int32_t* status_dev, void* ws, size_t ws_bytes, tt_stream stream) {
  return backward_impl(x, y, mask, layout, prec, cot_dev, dz, gx, gy, ckpt_stride, 0, status_dev, ws, ws_bytes,
                       stream);
}

int tt_contract_backward_k(const tt_desc* x, const tt_desc* y, const uint8_t* mask, int prec, const tt_desc* dz,
                           const tt_desc* gx, const tt_desc* gy, int32_t* status_dev, void* ws, size_t ws_bytes,
                           tt_stream stream) {
  if (mask == nullptr) return TT_ERR_ARG;
  return backward_impl(x, y, mask, TT_LAYOUT_CHAIN, prec, nullptr, dz, gx, gy, 0, 1, status_dev, ws, ws_bytes,
                       stream);
}

}  // extern "C"
