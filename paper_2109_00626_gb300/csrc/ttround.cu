// TT rounding: a TT re-expressed with smaller ranks, within eps ||X||_F of the
// tensor it represents (the TT-SVD's truncation rule of Section II applied to
// a tensor that is already a TT; for instance a merged-layout result, whose
// ranks R^x R^y are products of the operands' ranks).
//
// Two sweeps over the cores, each a chain of SVDs of single-core unfoldings
// (svd_common.cuh):
//   1. right to left, nothing dropped but exactly-zero singular values: each
//      core's unfolding (r_{k-1}) x (I_k r_k) = U S V^T, the core becomes the
//      rows of V^T (right-orthonormal) and U S is multiplied into core k-1.
//      It is carried out as a left-to-right sweep of the reversed TT (cores
//      in reverse order, rank legs swapped), so one routine serves both.
//      Afterwards ||X||_F = ||G_0||_F.
//   2. left to right with the truncation rule: core k's unfolding
//      (r_{k-1} I_k) x r_k = U S V^T keeps the smallest rank whose dropped
//      singular values have 2-norm <= eps ||X||_F / sqrt(N - 1) (then at most
//      max_rank); the core becomes U's columns and S V^T is multiplied into
//      core k + 1.  The right-orthonormal rest makes each dropped part an
//      orthogonal error term, so the total error is at most eps ||X||_F.
// One CTA of 1024 threads runs both sweeps; the cores live in the workspace.
#include <math.h>
#include <string.h>

#include "host_plan.h"
#include "svd_common.cuh"

namespace ttc {

struct RoundParams {
  int order;
  int32_t modes[kMaxOrder];
  int32_t ranks[kMaxOrder + 1];  // the input's
  const void* in[kMaxOrder];
  void* out[kMaxOrder];
  int32_t* ranks_out;
  int32_t* status;
  void* area_a;          // the reversed TT: core k at off_a[k], capacity of input core N-1-k
  void* area_b;          // the TT: core k at off_b[k], capacity of input core k
  int64_t off_a[kMaxOrder];
  int64_t off_b[kMaxOrder];
  void* mbuf;            // the largest core (an unfolding's copy; the next core's product)
  void* sbuf;            // the largest core (the transpose of a tall unfolding)
  void* svt;             // the largest rank squared
  void* qt;              // kSvdMaxP^2
  double* sig;
  int32_t* ord;
  double eps;
  int max_rank;
  size_t smem_bytes;
};

// dst[b][i][a] = src[a][i][b] for a core [ra][I][rb] (its rank legs swapped).
template <typename T>
__device__ void swap_legs(T* __restrict__ dst, const T* __restrict__ src, int ra, int I, int rb) {
  const int64_t n = static_cast<int64_t>(ra) * I * rb;
  for (int64_t e = threadIdx.x; e < n; e += kSvdThreads) {
    const int b = static_cast<int>(e % rb);
    const int64_t t = e / rb;
    const int i = static_cast<int>(t % I), a = static_cast<int>(t / I);
    dst[(static_cast<int64_t>(b) * I + i) * ra + a] = src[e];
  }
}

// One left-to-right sweep: cores k = 0 .. N-2 of `area` (ranks rk[], updated)
// replaced by their unfolding's U, S V^T multiplied into core k + 1.  Every
// CTA of the cluster calls it (the SVDs are shared); the rest is the leader's.
template <typename T>
__device__ void lr_sweep(const RoundParams& p, T* area, const int64_t* off, const int32_t* modes, int* rk,
                         double delta2, int max_rank, const SvdShared<T>& sh, SvdCluster& cl) {
  const int tid = threadIdx.x;
  const bool leader = cl.rank == 0;
  T* mbuf = static_cast<T*>(p.mbuf);
  T* svt = static_cast<T*>(p.svt);
  for (int k = 0; k + 1 < p.order; ++k) {
    T* core = area + off[k];
    T* next = area + off[k + 1];
    const int m = rk[k] * modes[k], n = rk[k + 1];
    if (leader) {
      const int64_t mn = static_cast<int64_t>(m) * n;
      for (int64_t e = tid; e < mn; e += kSvdThreads) mbuf[e] = core[e];
      __syncthreads();
    }
    const int r = svd_factor<T>(mbuf, static_cast<T*>(p.sbuf), static_cast<T*>(p.qt), p.sig, p.ord, m, n, delta2,
                                max_rank, core, svt, sh, cl);
    if (!leader) continue;
    // next <- (S V^T)[r x n] next[n x L]
    const int64_t L = static_cast<int64_t>(modes[k + 1]) * rk[k + 2];
    for (int64_t e = tid; e < r * L; e += kSvdThreads) {
      const int t = static_cast<int>(e / L);
      const int64_t l = e - t * L;
      const T* sr = svt + static_cast<int64_t>(t) * n;
      T acc = T(0);
      for (int a = 0; a < n; ++a) acc = fma(sr[a], next[a * L + l], acc);
      mbuf[e] = acc;
    }
    __syncthreads();
    for (int64_t e = tid; e < r * L; e += kSvdThreads) next[e] = mbuf[e];
    if (tid == 0) rk[k + 1] = r;
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(kSvdThreads, 1) ttround_kernel(const __grid_constant__ RoundParams p) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double red[kSvdWarps];
  __shared__ int s_rot, s_r;
  __shared__ T tile[32 * 33];
  __shared__ int rk[kMaxOrder + 1];
  __shared__ int32_t mrev[kMaxOrder];
  __shared__ int bc[16];
  __shared__ unsigned long long bcp[4];
  SvdCluster cl = svd_cluster_begin(p.status, bc, bcp);
  const bool leader = cl.rank == 0;
  const int tid = threadIdx.x;
  const int N = p.order;
  T* A = static_cast<T*>(p.area_a);
  T* B = static_cast<T*>(p.area_b);
  const SvdShared<T> sh{red, &s_rot, &s_r, tile, dsm, p.smem_bytes};

  if (leader) {
    // the reversed TT
    for (int k = 0; k < N; ++k) {
      const int s = N - 1 - k;
      swap_legs<T>(A + p.off_a[k], static_cast<const T*>(p.in[s]), p.ranks[s], p.modes[s], p.ranks[s + 1]);
    }
    if (tid <= N) rk[tid] = p.ranks[N - tid];
    if (tid < N) mrev[tid] = p.modes[N - 1 - tid];
    __syncthreads();
  }
  // 1. right-orthonormal cores (a left-to-right sweep of the reversed TT)
  lr_sweep<T>(p, A, p.off_a, mrev, rk, 0.0, 0, sh, cl);
  double delta2 = 0.0;
  if (leader) {
    // back to the original order
    for (int k = 0; k < N; ++k) {
      const int s = N - 1 - k;
      swap_legs<T>(B + p.off_b[k], A + p.off_a[s], rk[s], mrev[s], rk[s + 1]);
    }
    __syncthreads();
    if (tid == 0) {
      int tmp[kMaxOrder + 1];
      for (int k = 0; k <= N; ++k) tmp[k] = rk[N - k];
      for (int k = 0; k <= N; ++k) rk[k] = tmp[k];
    }
    __syncthreads();
    // ||X||_F = ||G_0||_F now
    double ss = 0.0;
    const int64_t n0 = static_cast<int64_t>(rk[0]) * p.modes[0] * rk[1];
    for (int64_t e = tid; e < n0; e += kSvdThreads) {
      const double v = static_cast<double>(B[p.off_b[0] + e]);
      ss += v * v;
    }
    const double nrm2 = block_sum(ss, red);
    if (tid == 0) {
      bc[8] = isfinite(nrm2) ? 1 : 0;
      if (!isfinite(nrm2)) atomicOr(p.status, TT_STATUS_NONFINITE);
    }
    delta2 = N > 1 ? p.eps * p.eps * nrm2 / (N - 1) : 0.0;
  }
  svd_barrier(cl);
  if (!svd_leader_flag(cl, 8)) {
    svd_barrier(cl);  // nobody leaves while a peer may still read its shared memory
    return;
  }
  // 2. truncation, left to right
  lr_sweep<T>(p, B, p.off_b, p.modes, rk, delta2, p.max_rank, sh, cl);
  if (leader) {
    for (int k = 0; k < N; ++k) {
      const int64_t n = static_cast<int64_t>(rk[k]) * p.modes[k] * rk[k + 1];
      T* dst = static_cast<T*>(p.out[k]);
      for (int64_t e = tid; e < n; e += kSvdThreads) dst[e] = B[p.off_b[k] + e];
    }
    if (tid <= N) p.ranks_out[tid] = rk[tid];
  }
  svd_barrier(cl);
}

struct RoundLayout {
  int64_t off_a[kMaxOrder], off_b[kMaxOrder];
  int64_t area, maxcore, maxsq;
  int pmax;
  size_t smem;
  size_t bytes;
};

static int round_layout(const tt_desc* x, int max_rank, RoundLayout* lo) {
  int rc = check_desc(x);
  if (rc != TT_OK) return rc;
  if (x->dtype != TT_F32 && x->dtype != TT_F64) return TT_ERR_DTYPE;
  if (max_rank < 0) return TT_ERR_ARG;
  const int N = x->order;
  const size_t eb = static_cast<size_t>(elem_bytes(x->dtype));
  auto size = [&](int k) { return static_cast<int64_t>(x->ranks[k]) * x->modes[k] * x->ranks[k + 1]; };
  int64_t oa = 0, ob = 0, mc = 1, ms = 1;
  int pm = 1;
  size_t smem = 0;
  for (int k = 0; k < N; ++k) {
    const int64_t sa = size(N - 1 - k), sb = size(k);
    lo->off_a[k] = oa;
    lo->off_b[k] = ob;
    oa += (sa + 3) & ~int64_t(3);  // 16-byte aligned starts
    ob += (sb + 3) & ~int64_t(3);
    mc = std::max(mc, sb);
    ms = std::max<int64_t>(ms, static_cast<int64_t>(x->ranks[k + 1]) * x->ranks[k + 1]);
    ms = std::max<int64_t>(ms, static_cast<int64_t>(x->ranks[k]) * x->ranks[k]);
    // the unfoldings of either sweep: (r I) x r' and (r' I) x r
    for (int side = 0; side < 2; ++side) {
      const int64_t m = static_cast<int64_t>(side ? x->ranks[k + 1] : x->ranks[k]) * x->modes[k];
      const int64_t n = side ? x->ranks[k] : x->ranks[k + 1];
      const int64_t ps = std::min(m, n);
      if (ps > kSvdMaxP) return TT_ERR_TOO_LARGE;
      pm = std::max(pm, static_cast<int>(ps));
      const size_t b = static_cast<size_t>(m * n + ps * ps) * eb;
      if (b <= kSvdSmemCap) smem = std::max(smem, b);
    }
    if (sb > (int64_t(1) << 31) - 1) return TT_ERR_TOO_LARGE;
  }
  lo->area = std::max(oa, ob);
  lo->maxcore = mc;
  lo->maxsq = ms;
  lo->pmax = pm;
  lo->smem = smem;
  lo->bytes = 2 * align256(static_cast<size_t>(lo->area) * eb) + 2 * align256(static_cast<size_t>(mc) * eb) +
              align256(static_cast<size_t>(ms) * eb) + align256(static_cast<size_t>(pm) * pm * eb) +
              align256(static_cast<size_t>(pm) * 8) + align256(static_cast<size_t>(pm) * 4);
  return TT_OK;
}

}  // namespace ttc

using namespace ttc;

extern "C" int tt_round_workspace(const tt_desc* x, int32_t max_rank, size_t* ws_bytes) {
  if (ws_bytes == nullptr) return TT_ERR_ARG;
  RoundLayout lo;
  const int rc = round_layout(x, max_rank, &lo);
  if (rc != TT_OK) return rc;
  *ws_bytes = lo.bytes;
  return TT_OK;
}

extern "C" int tt_round(const tt_desc* x, double eps, int32_t max_rank, void* const* cores_out, int32_t* ranks_dev,
                        int32_t* status_dev, void* ws, size_t ws_bytes, tt_stream stream) {
  if (cores_out == nullptr || ranks_dev == nullptr || status_dev == nullptr || ws == nullptr) return TT_ERR_ARG;
  if (!(eps >= 0.0) || !isfinite(eps)) return TT_ERR_ARG;
  RoundLayout lo;
  int rc = round_layout(x, max_rank, &lo);
  if (rc != TT_OK) return rc;
  if (ws_bytes < lo.bytes) return TT_ERR_WS;
  for (int k = 0; k < x->order; ++k)
    if (cores_out[k] == nullptr) return TT_ERR_ARG;
  const size_t eb = static_cast<size_t>(elem_bytes(x->dtype));
  RoundParams p;
  memset(&p, 0, sizeof(p));
  p.order = x->order;
  for (int k = 0; k < x->order; ++k) {
    p.modes[k] = x->modes[k];
    p.in[k] = x->cores[k];
    p.out[k] = cores_out[k];
    p.off_a[k] = lo.off_a[k];
    p.off_b[k] = lo.off_b[k];
  }
  for (int k = 0; k <= x->order; ++k) p.ranks[k] = x->ranks[k];
  p.ranks_out = ranks_dev;
  p.status = status_dev;
  char* w = static_cast<char*>(ws);
  p.area_a = w;
  w += align256(static_cast<size_t>(lo.area) * eb);
  p.area_b = w;
  w += align256(static_cast<size_t>(lo.area) * eb);
  p.mbuf = w;
  w += align256(static_cast<size_t>(lo.maxcore) * eb);
  p.sbuf = w;
  w += align256(static_cast<size_t>(lo.maxcore) * eb);
  p.svt = w;
  w += align256(static_cast<size_t>(lo.maxsq) * eb);
  p.qt = w;
  w += align256(static_cast<size_t>(lo.pmax) * lo.pmax * eb);
  p.sig = reinterpret_cast<double*>(w);
  w += align256(static_cast<size_t>(lo.pmax) * 8);
  p.ord = reinterpret_cast<int32_t*>(w);
  p.eps = eps;
  p.max_rank = max_rank;
  // shared memory: the largest single-CTA SVD that fits, or the largest
  // cluster-spread one (both sweeps' unfoldings, at the input's ranks)
  auto smem_of = [&](int c) {
    size_t smem = lo.smem;
    if (c > 1)
      for (int k = 0; k < x->order; ++k)
        for (int side = 0; side < 2; ++side) {
          const int64_t m = static_cast<int64_t>(side ? x->ranks[k + 1] : x->ranks[k]) * x->modes[k];
          const int64_t n = side ? x->ranks[k] : x->ranks[k + 1];
          const int64_t ps = std::min(m, n), ls = std::max(m, n);
          if (ls >= (int64_t(1) << 30)) continue;
          const size_t d = dist_smem_elems(static_cast<int>(ps), static_cast<int>(ls), c) * eb;
          if (d <= kSvdSmemCap) smem = std::max(smem, d);
          const size_t rd = rowdist_smem_elems(static_cast<int>(ps), static_cast<int>(ls), c) * eb;
          if (rd <= kSvdSmemCap) smem = std::max(smem, rd);
        }
    return smem;
  };
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const cudaError_t err = x->dtype == TT_F64 ? svd_launch<RoundParams>(ttround_kernel<double>, p, smem_of, s)
                                             : svd_launch<RoundParams>(ttround_kernel<float>, p, smem_of, s);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return TT_ERR_CUDA;
  }
  count_launch();
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}
