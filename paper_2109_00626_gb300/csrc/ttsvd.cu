// TT decomposition of a dense tensor (the TT-SVD of Section II, whose
// accuracy guarantee is ||X - TT(X)||_F <= eps ||X||_F), and the dense mode
// permutation that the dense-input contraction (Alg. 2: the paired modes of
// each operand brought to the front before decomposing) applies first.
//
// The decomposition walks the modes left to right.  At mode k the part of X
// not yet factored is a matrix C of (r_{k-1} I_k) rows and prod_{j>k} I_j
// columns.  Its SVD C = U S V^T (one-sided Jacobi, svd_common.cuh) keeps the
// truncation rule of the TT-SVD: the smallest r >= 1 whose dropped singular
// values have 2-norm <= eps ||X||_F / sqrt(N - 1), capped by an optional
// maximum rank.  Core k is U's first r columns (left-orthonormal cores), and
// S V^T's first r rows carry on to mode k + 1.
//
// One CTA of 1024 threads runs the whole decomposition (the steps depend on
// each other's ranks); the matrices live in the caller's workspace, and an SVD
// whose vectors and accumulated rotations fit in 200 KB is swept in shared
// memory.
#include <math.h>
#include <string.h>

#include "host_plan.h"
#include "svd_common.cuh"

namespace ttc {

struct SvdParams {
  const void* x;
  int order;
  int32_t modes[kMaxOrder];
  void* cores[kMaxOrder];
  int32_t* ranks_out;  // [order + 1], device
  int32_t* status;
  void* buf0;          // two matrices of numel elements
  void* buf1;
  void* qt;            // kSvdMaxP^2 elements: the accumulated rotations, transposed
  double* sig;         // kSvdMaxP singular values
  int32_t* ord;        // kSvdMaxP: indices of the singular values, largest first
  int64_t numel;
  double eps;
  int max_rank;        // 0: no cap
  size_t smem_bytes;   // dynamic shared memory: an SVD whose vectors and rotations fit runs there
};

template <typename T>
__global__ void __launch_bounds__(kSvdThreads, 1) ttsvd_kernel(const __grid_constant__ SvdParams p) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double red[kSvdWarps];
  __shared__ int s_rot, s_r;
  __shared__ T tile[32 * 33];
  __shared__ int bc[16];
  __shared__ unsigned long long bcp[4];
  SvdCluster cl = svd_cluster_begin(p.status, bc, bcp);
  const bool leader = cl.rank == 0;
  const int tid = threadIdx.x;
  const T* x = static_cast<const T*>(p.x);
  T* cur = static_cast<T*>(p.buf0);
  T* oth = static_cast<T*>(p.buf1);
  T* Qt = static_cast<T*>(p.qt);
  const int N = p.order;

  // ||X||_F^2 (float64), and X copied into the first buffer (leader)
  double delta2 = 0.0;
  if (leader) {
    double ss = 0.0;
    for (int64_t e = tid; e < p.numel; e += kSvdThreads) {
      const T v = x[e];
      cur[e] = v;
      ss += static_cast<double>(v) * static_cast<double>(v);
    }
    const double nrm2 = block_sum(ss, red);
    if (tid == 0) {
      bc[8] = isfinite(nrm2) ? 1 : 0;
      if (!isfinite(nrm2)) atomicOr(p.status, TT_STATUS_NONFINITE);
      else p.ranks_out[0] = 1;
    }
    delta2 = N > 1 ? p.eps * p.eps * nrm2 / (N - 1) : 0.0;
  }
  svd_barrier(cl);
  if (!svd_leader_flag(cl, 8)) {
    svd_barrier(cl);  // nobody leaves while a peer may still read its shared memory
    return;
  }

  const SvdShared<T> sh{red, &s_rot, &s_r, tile, dsm, p.smem_bytes};
  int r_prev = 1;
  int64_t tail = p.numel;  // prod_{j >= k} I_j
  for (int k = 0; k + 1 < N; ++k) {
    tail /= p.modes[k];
    const int m = r_prev * p.modes[k];
    const int n = static_cast<int>(tail);
    const bool wide = m < n;
    // core k = U's columns; S V^T carries on (a wide M is read while S V^T is
    // written, so that goes to the other buffer)
    const int r = svd_factor<T>(cur, oth, Qt, p.sig, p.ord, m, n, delta2, p.max_rank, static_cast<T*>(p.cores[k]),
                                wide ? oth : cur, sh, cl);
    if (leader && tid == 0) p.ranks_out[k + 1] = r;
    if (wide) {
      T* sw = cur;
      cur = oth;
      oth = sw;
    }
    r_prev = r;
  }
  if (leader) {
    // last core: the remaining r_{N-1} x I_N matrix
    T* last = static_cast<T*>(p.cores[N - 1]);
    for (int64_t e = tid; e < static_cast<int64_t>(r_prev) * p.modes[N - 1]; e += kSvdThreads) last[e] = cur[e];
    if (tid == 0) p.ranks_out[N] = 1;
  }
  svd_barrier(cl);
}

// Output axis t: its size and the input stride it walks.
struct PermDims {
  int64_t dim[kMaxOrder];
  int64_t stride[kMaxOrder];
};

// out[j_0..j_{N-1}] = in[...] with output axis t = input axis axes[t].
template <typename T>
__global__ void dense_permute_kernel(const T* __restrict__ in, T* __restrict__ out, int order, PermDims d,
                                     int64_t numel) {
  for (int64_t o = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; o < numel;
       o += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int64_t rem = o, off = 0;
    for (int t = order - 1; t >= 0; --t) {
      const int64_t j = rem % d.dim[t];
      rem /= d.dim[t];
      off += j * d.stride[t];
    }
    out[o] = in[off];
  }
}

// Shapes: the largest ranks the decomposition can return (the unfolding
// sizes, capped) and the shorter side of every unfolding.
static int svd_caps(int order, const int32_t* modes, int max_rank, int32_t* cap, int* pmax, int64_t* numel) {
  if (order < 1 || order > kMaxOrder || modes == nullptr || cap == nullptr || max_rank < 0) return TT_ERR_ARG;
  int64_t n = 1;
  for (int k = 0; k < order; ++k) {
    if (modes[k] < 1) return TT_ERR_SHAPE;
    n *= modes[k];
    if (n > (int64_t(1) << 31) - 1) return TT_ERR_TOO_LARGE;
  }
  *numel = n;
  cap[0] = 1;
  int64_t tail = n;
  int pm = 1;
  for (int k = 0; k + 1 < order; ++k) {
    tail /= modes[k];
    const int64_t rows = static_cast<int64_t>(cap[k]) * modes[k];
    const int64_t short_side = std::min<int64_t>(rows, tail);
    if (short_side > kSvdMaxP) return TT_ERR_TOO_LARGE;
    pm = std::max(pm, static_cast<int>(short_side));
    int64_t c = short_side;
    if (max_rank > 0) c = std::min<int64_t>(c, max_rank);
    cap[k + 1] = static_cast<int32_t>(c);
  }
  cap[order] = 1;
  *pmax = pm;
  return TT_OK;
}

}  // namespace ttc

using namespace ttc;

extern "C" int tt_svd_workspace(int order, const int32_t* modes, int dtype, int32_t max_rank, int32_t* cap_ranks,
                                size_t* ws_bytes) {
  if (ws_bytes == nullptr) return TT_ERR_ARG;
  if (dtype != TT_F32 && dtype != TT_F64) return TT_ERR_DTYPE;
  int pmax = 0;
  int64_t numel = 0;
  const int rc = svd_caps(order, modes, max_rank, cap_ranks, &pmax, &numel);
  if (rc != TT_OK) return rc;
  const size_t eb = static_cast<size_t>(elem_bytes(dtype));
  *ws_bytes = 2 * align256(numel * eb) + align256(static_cast<size_t>(pmax) * pmax * eb) + align256(pmax * 8) +
              align256(pmax * 4);
  return TT_OK;
}

extern "C" int tt_svd(const void* x_dev, int order, const int32_t* modes, int dtype, double eps, int32_t max_rank,
                      void* const* cores_dev, int32_t* ranks_dev, int32_t* status_dev, void* ws, size_t ws_bytes,
                      tt_stream stream) {
  if (x_dev == nullptr || cores_dev == nullptr || ranks_dev == nullptr || status_dev == nullptr || ws == nullptr)
    return TT_ERR_ARG;
  if (!(eps >= 0.0) || !isfinite(eps)) return TT_ERR_ARG;
  int32_t cap[kMaxOrder + 1];
  size_t need = 0;
  int rc = tt_svd_workspace(order, modes, dtype, max_rank, cap, &need);
  if (rc != TT_OK) return rc;
  if (ws_bytes < need) return TT_ERR_WS;
  for (int k = 0; k < order; ++k)
    if (cores_dev[k] == nullptr) return TT_ERR_ARG;
  int pmax = 0;
  int64_t numel = 0;
  svd_caps(order, modes, max_rank, cap, &pmax, &numel);
  const size_t eb = static_cast<size_t>(elem_bytes(dtype));
  SvdParams p;
  memset(&p, 0, sizeof(p));
  p.x = x_dev;
  p.order = order;
  for (int k = 0; k < order; ++k) {
    p.modes[k] = modes[k];
    p.cores[k] = cores_dev[k];
  }
  p.ranks_out = ranks_dev;
  p.status = status_dev;
  char* w = static_cast<char*>(ws);
  p.buf0 = w;
  w += align256(numel * eb);
  p.buf1 = w;
  w += align256(numel * eb);
  p.qt = w;
  w += align256(static_cast<size_t>(pmax) * pmax * eb);
  p.sig = reinterpret_cast<double*>(w);
  w += align256(pmax * 8);
  p.ord = reinterpret_cast<int32_t*>(w);
  p.numel = numel;
  p.eps = eps;
  p.max_rank = max_rank;
  // shared memory for the largest SVD that fits, in one CTA or spread over a
  // cluster of c (sizes bounded by the caps)
  auto smem_of = [&](int c) {
    size_t smem = 0;
    int64_t tail = numel;
    for (int k = 0; k + 1 < order; ++k) {
      tail /= modes[k];
      const int64_t rows = static_cast<int64_t>(cap[k]) * modes[k];
      const int64_t ps = std::min<int64_t>(rows, tail), ls = std::max<int64_t>(rows, tail);
      const size_t b = static_cast<size_t>(rows * tail + ps * ps) * eb;
      if (b <= kSvdSmemCap) smem = std::max(smem, b);
      if (c > 1 && ls < (int64_t(1) << 30)) {
        const size_t d = dist_smem_elems(static_cast<int>(ps), static_cast<int>(ls), c) * eb;
        if (d <= kSvdSmemCap) smem = std::max(smem, d);
        const size_t rd = rowdist_smem_elems(static_cast<int>(ps), static_cast<int>(ls), c) * eb;
        if (rd <= kSvdSmemCap) smem = std::max(smem, rd);
      }
    }
    return smem;
  };
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const cudaError_t err = dtype == TT_F64 ? svd_launch<SvdParams>(ttsvd_kernel<double>, p, smem_of, s)
                                          : svd_launch<SvdParams>(ttsvd_kernel<float>, p, smem_of, s);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return TT_ERR_CUDA;
  }
  count_launch();
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

extern "C" int tt_dense_permute(const void* in_dev, int order, const int32_t* modes, const int32_t* axes, int dtype,
                                void* out_dev, tt_stream stream) {
  if (in_dev == nullptr || out_dev == nullptr || modes == nullptr || axes == nullptr) return TT_ERR_ARG;
  if (order < 1 || order > kMaxOrder) return TT_ERR_ARG;
  if (dtype != TT_F32 && dtype != TT_F64) return TT_ERR_DTYPE;
  if (in_dev == out_dev) return TT_ERR_ARG;
  bool seen[kMaxOrder] = {false};
  int64_t in_stride[kMaxOrder];
  int64_t numel = 1;
  for (int k = order - 1; k >= 0; --k) {
    if (modes[k] < 1) return TT_ERR_SHAPE;
    in_stride[k] = numel;
    numel *= modes[k];
    if (numel > (int64_t(1) << 40)) return TT_ERR_TOO_LARGE;
  }
  PermDims d;
  for (int t = 0; t < order; ++t) {
    const int a = axes[t];
    if (a < 0 || a >= order || seen[a]) return TT_ERR_ARG;
    seen[a] = true;
    d.dim[t] = modes[a];
    d.stride[t] = in_stride[a];
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int blocks = static_cast<int>(std::min<int64_t>(4 * 152, (numel + 255) / 256));
  if (dtype == TT_F64)
    dense_permute_kernel<double><<<blocks, 256, 0, s>>>(static_cast<const double*>(in_dev),
                                                        static_cast<double*>(out_dev), order, d, numel);
  else
    dense_permute_kernel<float><<<blocks, 256, 0, s>>>(static_cast<const float*>(in_dev), static_cast<float*>(out_dev),
                                                       order, d, numel);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}
