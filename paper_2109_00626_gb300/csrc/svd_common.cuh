// One-sided Jacobi SVD of a small matrix by one CTA of 1024 threads
// (Hestenes 1958), shared by the TT decomposition of a dense tensor and the
// rounding of a TT.  The p = min(rows, columns) vectors of the shorter side
// are made mutually orthogonal by plane rotations, swept in the round-robin
// order of the circle method (p / 2 disjoint pairs per round, a warp per
// pair), each rotation also applied to an accumulated orthogonal p x p
// matrix; their norms are the singular values.  svd_factor() then keeps the
// rank that the TT-SVD's truncation rule gives and writes the two factors.
#pragma once

#include <math.h>
#include <stdint.h>

#include "ttc_internal.h"

namespace ttc {

constexpr int kSvdThreads = 1024;
constexpr int kSvdWarps = kSvdThreads / 32;
constexpr int kSvdMaxP = 512;       // the shorter side of an unfolding
constexpr int kSvdMaxSweeps = 40;   // a bound on the Jacobi sweeps of one SVD
constexpr size_t kSvdSmemCap = 200 * 1024;  // shared memory for the sweeps of an SVD that fits

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
  // a pair counts as orthogonal once |<a, b>| <= 4 u sqrt(L) |a| |b|: the
  // rounding of an L-term dot product, below which rotations only chase noise
  const T tol = T(4) * (sizeof(T) == 8 ? T(1.1102230246251565e-16) : T(5.9604645e-08)) * sqrt(T(L > 1 ? L : 1));
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

// Per-CTA shared scalars of svd_factor and its dynamic shared memory.
template <typename T>
struct SvdShared {
  double* red;   // kSvdWarps
  int* s_rot;
  int* s_r;
  T* tile;       // 32 x 33
  unsigned char* dsm;
  size_t smem_bytes;
};

// SVD of the row-major m x n matrix M = U S V^T, truncated: the smallest
// r >= 1 whose dropped singular values have squared 2-norm <= delta2, then at
// most max_rank (0: no cap).  Writes U's first r columns to u_out (m x r,
// row-major) and the first r rows of S V^T to svt_out (r x n); returns r.
// M is overwritten; scratch holds m n entries (the transpose of a tall M),
// qt p^2, sig and ord p.  svt_out may alias M (not scratch), u_out neither.
template <typename T>
__device__ int svd_factor(T* M, T* scratch, T* qt, double* sig, int32_t* ord, int m, int n, double delta2,
                          int max_rank, T* u_out, T* svt_out, const SvdShared<T>& sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool wide = m < n;
  const int pp = wide ? m : n, L = wide ? n : m;
  T* W = M;
  if (!wide) {
    transpose_rows<T>(scratch, M, m, n, sh.tile);
    W = scratch;
  }
  // the sweeps run in shared memory when the vectors and the rotations fit
  const int64_t wl = static_cast<int64_t>(pp) * L;
  const bool local = static_cast<size_t>(wl + static_cast<int64_t>(pp) * pp) * sizeof(T) <= sh.smem_bytes;
  T* Wj = local ? reinterpret_cast<T*>(sh.dsm) : W;
  T* Qj = local ? Wj + wl : qt;
  if (local)
    for (int64_t e = tid; e < wl; e += kSvdThreads) Wj[e] = W[e];
  for (int e = tid; e < pp * pp; e += kSvdThreads) Qj[e] = (e / pp == e % pp) ? T(1) : T(0);
  __syncthreads();
  jacobi_rows<T>(Wj, Qj, pp, L, sh.s_rot);
  if (local) {
    for (int64_t e = tid; e < wl; e += kSvdThreads) W[e] = Wj[e];
    for (int e = tid; e < pp * pp; e += kSvdThreads) qt[e] = Qj[e];
    __syncthreads();
  }
  // singular values: the row norms (float64 sums), warp per row
  for (int i = warp; i < pp; i += kSvdWarps) {
    double s2 = 0.0;
    const T* w = W + static_cast<int64_t>(i) * L;
    for (int e = lane; e < L; e += 32) s2 += static_cast<double>(w[e]) * static_cast<double>(w[e]);
    s2 = warp_sum_t(s2);
    if (lane == 0) sig[i] = sqrt(s2);
  }
  __syncthreads();
  // order, largest first (ties by index): position of value i
  for (int i = tid; i < pp; i += kSvdThreads) {
    const double si = sig[i];
    int pos = 0;
    for (int j = 0; j < pp; ++j) {
      const double sj = sig[j];
      pos += (sj > si || (sj == si && j < i)) ? 1 : 0;
    }
    ord[pos] = i;
  }
  __syncthreads();
  if (tid == 0) {
    int r = pp;
    double dropped = 0.0;
    while (r > 1) {
      const double s = sig[ord[r - 1]];
      if (dropped + s * s > delta2) break;
      dropped += s * s;
      --r;
    }
    if (max_rank > 0 && r > max_rank) r = max_rank;
    *sh.s_r = r;
  }
  __syncthreads();
  const int r = *sh.s_r;
  if (wide) {
    // U = Q (u_out[i][t] = qt[ord t][i]); S V^T = the rows of W in order
    for (int64_t e = tid; e < static_cast<int64_t>(r) * n; e += kSvdThreads) {
      const int t = static_cast<int>(e / n);
      const int64_t j = e - static_cast<int64_t>(t) * n;
      svt_out[e] = W[static_cast<int64_t>(ord[t]) * n + j];
    }
    for (int e = tid; e < m * r; e += kSvdThreads) {
      const int i = e / r, t = e - i * r;
      u_out[e] = qt[static_cast<int64_t>(ord[t]) * pp + i];
    }
  } else {
    // W = S U^T row by row: u_out[i][t] = W[ord t][i] / sigma; S V^T = sigma qt rows
    for (int64_t e = tid; e < static_cast<int64_t>(m) * r; e += kSvdThreads) {
      const int64_t i = e / r;
      const int t = static_cast<int>(e - i * r);
      const int o = ord[t];
      const double s = sig[o];
      u_out[e] = s > 0.0 ? static_cast<T>(static_cast<double>(W[static_cast<int64_t>(o) * m + i]) / s) : T(0);
    }
    for (int e = tid; e < r * n; e += kSvdThreads) {
      const int t = e / n, j = e - t * n;
      const int o = ord[t];
      svt_out[e] = static_cast<T>(sig[o] * static_cast<double>(qt[static_cast<int64_t>(o) * pp + j]));
    }
  }
  __syncthreads();
  return r;
}

}  // namespace ttc
