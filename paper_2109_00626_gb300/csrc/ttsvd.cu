// TT decomposition of a dense tensor (the TT-SVD of Section II, whose
// accuracy guarantee is ||X - TT(X)||_F <= eps ||X||_F), and the dense mode
// permutation that the dense-input contraction (Alg. 2: the paired modes of
// each operand brought to the front before decomposing) applies first.
//
// The decomposition walks the modes left to right.  At mode k the part of X
// not yet factored is a matrix C of (r_{k-1} I_k) rows and prod_{j>k} I_j
// columns.  Its SVD C = U S V^T is taken with a one-sided Jacobi method
// (Hestenes 1958): the p = min(rows, columns) vectors of the shorter side are
// made mutually orthogonal by plane rotations, swept in the round-robin
// order of the circle method (p / 2 disjoint pairs per round), each rotation
// also applied to an accumulated orthogonal p x p matrix.  The norms of the
// orthogonalised vectors are the singular values.  Ranks are kept by the
// truncation rule of the TT-SVD: the smallest r >= 1 whose dropped singular
// values have 2-norm <= eps ||X||_F / sqrt(N - 1), capped by an optional
// maximum rank.  Core k is U's first r columns (left-orthonormal cores), and
// S V^T's first r rows carry on to mode k + 1.
//
// One CTA of 1024 threads runs the whole decomposition (the steps depend on
// each other's ranks); the matrices live in the caller's workspace, and an SVD
// whose vectors and accumulated rotations fit in 200 KB is swept in shared
// memory.  Wide matrices (rows < columns) are
// orthogonalised by rows in place; tall ones are first transposed so their
// columns become contiguous rows.
#include <math.h>
#include <string.h>

#include "host_plan.h"

namespace ttc {

constexpr int kSvdThreads = 1024;
constexpr int kSvdWarps = kSvdThreads / 32;
constexpr int kSvdMaxP = 512;       // the shorter side of an unfolding
constexpr int kSvdMaxSweeps = 40;   // a bound on the Jacobi sweeps of one SVD

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

constexpr size_t kSvdSmemCap = 200 * 1024;

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block (every thread gets it).
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum_t(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < kSvdWarps; ++w) s += red[w];
  return s;
}

// dst (n x m) = src (m x n)^T through 32 x 33 shared-memory tiles.
template <typename T>
__device__ void transpose_rows(T* __restrict__ dst, const T* __restrict__ src, int m, int n, T* tile) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int b0 = 0; b0 < m; b0 += 32)
    for (int b1 = 0; b1 < n; b1 += 32) {
      const int r = b0 + ty, c = b1 + tx;
      if (r < m && c < n) tile[ty * 33 + tx] = src[static_cast<int64_t>(r) * n + c];
      __syncthreads();
      const int r2 = b1 + ty, c2 = b0 + tx;
      if (r2 < n && c2 < m) dst[static_cast<int64_t>(r2) * m + c2] = tile[tx * 33 + ty];
      __syncthreads();
    }
}

// Pair i of round t of the circle method over P (even) indices.
__device__ __forceinline__ void rr_pair(int P, int t, int i, int& a, int& b) {
  if (i == 0) {
    a = P - 1;
    b = t;
  } else {
    a = (t + i) % (P - 1);
    b = (t - i + P - 1) % (P - 1);
  }
}

// One-sided Jacobi on the p rows (length L) of W, rotations also applied to
// the rows of Qt (p x p).  Returns the number of sweeps taken.
template <typename T>
__device__ int jacobi_rows(T* __restrict__ W, T* __restrict__ Qt, int p, int L, int* s_rot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T tol = T(8) * (sizeof(T) == 8 ? T(1.1102230246251565e-16) : T(5.9604645e-08));
  const int P = (p + 1) & ~1;
  int sweep = 0;
  for (; sweep < kSvdMaxSweeps; ++sweep) {
    if (threadIdx.x == 0) *s_rot = 0;
    __syncthreads();
    for (int t = 0; t < P - 1; ++t) {
      for (int i = warp; i < P / 2; i += kSvdWarps) {
        int a, b;
        rr_pair(P, t, i, a, b);
        if (a >= p || b >= p) continue;  // the dummy index of an odd p
        T* wa = W + static_cast<int64_t>(a) * L;
        T* wb = W + static_cast<int64_t>(b) * L;
        T al = T(0), be = T(0), ga = T(0);
        for (int e = lane; e < L; e += 32) {
          const T u = wa[e], v = wb[e];
          al = fma(u, u, al);
          be = fma(v, v, be);
          ga = fma(u, v, ga);
        }
        al = warp_sum_t(al);
        be = warp_sum_t(be);
        ga = warp_sum_t(ga);
        if (ga == T(0) || al == T(0) || be == T(0) || fabs(ga) <= tol * sqrt(al) * sqrt(be)) continue;
        // rotation that zeroes the inner product of the two new rows:
        // t^2 + 2 zeta t - 1 = 0, the root of modulus <= 1
        const T zeta = (be - al) / (T(2) * ga);
        const T tn = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
        const T c = T(1) / sqrt(T(1) + tn * tn), s = c * tn;
        for (int e = lane; e < L; e += 32) {
          const T u = wa[e], v = wb[e];
          wa[e] = c * u - s * v;
          wb[e] = s * u + c * v;
        }
        T* qa = Qt + static_cast<int64_t>(a) * p;
        T* qb = Qt + static_cast<int64_t>(b) * p;
        for (int e = lane; e < p; e += 32) {
          const T u = qa[e], v = qb[e];
          qa[e] = c * u - s * v;
          qb[e] = s * u + c * v;
        }
        if (lane == 0) *s_rot = 1;
      }
      __syncthreads();
    }
    if (*s_rot == 0) break;
    __syncthreads();
  }
  return sweep;
}

template <typename T>
__global__ void __launch_bounds__(kSvdThreads, 1) ttsvd_kernel(const __grid_constant__ SvdParams p) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double red[kSvdWarps];
  __shared__ int s_rot, s_r;
  __shared__ T tile[32 * 33];
  const int tid = threadIdx.x;
  const T* x = static_cast<const T*>(p.x);
  T* cur = static_cast<T*>(p.buf0);
  T* oth = static_cast<T*>(p.buf1);
  T* Qt = static_cast<T*>(p.qt);
  const int N = p.order;

  // ||X||_F^2 (float64), and X copied into the first buffer
  double ss = 0.0;
  for (int64_t e = tid; e < p.numel; e += kSvdThreads) {
    const T v = x[e];
    cur[e] = v;
    ss += static_cast<double>(v) * static_cast<double>(v);
  }
  const double nrm2 = block_sum(ss, red);
  if (!isfinite(nrm2)) {
    if (tid == 0) atomicOr(p.status, TT_STATUS_NONFINITE);
    return;
  }
  const double delta2 = N > 1 ? p.eps * p.eps * nrm2 / (N - 1) : 0.0;
  if (tid == 0) p.ranks_out[0] = 1;

  int r_prev = 1;
  int64_t tail = p.numel;  // prod_{j >= k} I_j
  for (int k = 0; k + 1 < N; ++k) {
    tail /= p.modes[k];
    const int m = r_prev * p.modes[k];
    const int n = static_cast<int>(tail);
    const bool wide = m < n;
    const int pp = wide ? m : n, L = wide ? n : m;
    T* W = cur;
    if (!wide) {
      transpose_rows<T>(oth, cur, m, n, tile);
      W = oth;
    }
    // the Jacobi sweeps run in shared memory when the vectors and the
    // rotations fit (every round then costs shared-memory, not L2, latency)
    const int64_t wl = static_cast<int64_t>(pp) * L;
    const bool local = static_cast<size_t>(wl + static_cast<int64_t>(pp) * pp) * sizeof(T) <= p.smem_bytes;
    T* Wj = local ? reinterpret_cast<T*>(dsm) : W;
    T* Qj = local ? Wj + wl : Qt;
    if (local)
      for (int64_t e = tid; e < wl; e += kSvdThreads) Wj[e] = W[e];
    for (int e = tid; e < pp * pp; e += kSvdThreads) Qj[e] = (e / pp == e % pp) ? T(1) : T(0);
    __syncthreads();
    jacobi_rows<T>(Wj, Qj, pp, L, &s_rot);
    if (local) {
      for (int64_t e = tid; e < wl; e += kSvdThreads) W[e] = Wj[e];
      for (int e = tid; e < pp * pp; e += kSvdThreads) Qt[e] = Qj[e];
      __syncthreads();
    }
    // singular values: the row norms (float64 sums), warp per row
    const int lane = tid & 31, warp = tid >> 5;
    for (int i = warp; i < pp; i += kSvdWarps) {
      double s2 = 0.0;
      const T* w = W + static_cast<int64_t>(i) * L;
      for (int e = lane; e < L; e += 32) s2 += static_cast<double>(w[e]) * static_cast<double>(w[e]);
      s2 = warp_sum_t(s2);
      if (lane == 0) p.sig[i] = sqrt(s2);
    }
    __syncthreads();
    // order, largest first (ties by index): position of value i
    for (int i = tid; i < pp; i += kSvdThreads) {
      const double si = p.sig[i];
      int pos = 0;
      for (int j = 0; j < pp; ++j) {
        const double sj = p.sig[j];
        pos += (sj > si || (sj == si && j < i)) ? 1 : 0;
      }
      p.ord[pos] = i;
    }
    __syncthreads();
    // rank: the smallest r >= 1 whose dropped values have squared 2-norm <= delta^2
    if (tid == 0) {
      int r = pp;
      double dropped = 0.0;
      while (r > 1) {
        const double s = p.sig[p.ord[r - 1]];
        if (dropped + s * s > delta2) break;
        dropped += s * s;
        --r;
      }
      if (p.max_rank > 0 && r > p.max_rank) r = p.max_rank;
      s_r = r;
      p.ranks_out[k + 1] = r;
    }
    __syncthreads();
    const int r = s_r;
    T* core = static_cast<T*>(p.cores[k]);  // m x r
    if (wide) {
      // U = Q: core[i][t] = Qt[ord t][i]; S V^T = the rows of W in order
      for (int e = tid; e < m * r; e += kSvdThreads) {
        const int i = e / r, t = e - i * r;
        core[e] = Qt[static_cast<int64_t>(p.ord[t]) * pp + i];
      }
      for (int64_t e = tid; e < static_cast<int64_t>(r) * n; e += kSvdThreads) {
        const int t = static_cast<int>(e / n);
        const int64_t j = e - static_cast<int64_t>(t) * n;
        oth[e] = W[static_cast<int64_t>(p.ord[t]) * n + j];
      }
      __syncthreads();
      T* sw = cur;
      cur = oth;
      oth = sw;
    } else {
      // W = S U^T row by row: core[i][t] = W[ord t][i] / sigma; S V^T = sigma Qt rows
      for (int e = tid; e < m * r; e += kSvdThreads) {
        const int i = e / r, t = e - i * r;
        const int o = p.ord[t];
        const double s = p.sig[o];
        core[e] = s > 0.0 ? static_cast<T>(static_cast<double>(W[static_cast<int64_t>(o) * m + i]) / s) : T(0);
      }
      for (int e = tid; e < r * n; e += kSvdThreads) {
        const int t = e / n, j = e - t * n;
        const int o = p.ord[t];
        cur[e] = static_cast<T>(p.sig[o] * static_cast<double>(Qt[static_cast<int64_t>(o) * pp + j]));
      }
      __syncthreads();
    }
    r_prev = r;
  }
  // last core: the remaining r_{N-1} x I_N matrix
  T* last = static_cast<T*>(p.cores[N - 1]);
  for (int64_t e = tid; e < static_cast<int64_t>(r_prev) * p.modes[N - 1]; e += kSvdThreads) last[e] = cur[e];
  if (tid == 0) p.ranks_out[N] = 1;
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
  // shared memory for the largest SVD that fits (sizes bounded by the caps)
  size_t smem = 0;
  {
    int64_t tail = numel;
    for (int k = 0; k + 1 < order; ++k) {
      tail /= modes[k];
      const int64_t rows = static_cast<int64_t>(cap[k]) * modes[k];
      const int64_t ps = std::min<int64_t>(rows, tail);
      const size_t b = static_cast<size_t>(rows * tail + ps * ps) * eb;
      if (b <= kSvdSmemCap) smem = std::max(smem, b);
    }
  }
  p.smem_bytes = smem;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t err = dtype == TT_F64 ? cudaFuncSetAttribute(ttsvd_kernel<double>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                           static_cast<int>(smem))
                                    : cudaFuncSetAttribute(ttsvd_kernel<float>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                           static_cast<int>(smem));
  if (err != cudaSuccess) return TT_ERR_CUDA;
  if (dtype == TT_F64) ttsvd_kernel<double><<<1, kSvdThreads, smem, s>>>(p);
  else ttsvd_kernel<float><<<1, kSvdThreads, smem, s>>>(p);
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
