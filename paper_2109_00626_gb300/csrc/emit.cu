// Chain-layout emission of a partial contraction (Algorithm 2 steps 5-6).
//
// The result TT is the free cores of X walked towards the contracted block
// (with their rank legs exchanged when walked backwards -- the paper's
// T[1;3]), the boundary core C = (boundary core of X) joined with K, then the
// free cores of Y.  The copies are pure data movement (HBM bound); C is one
// small product per mode index i.
#include <cuda_bf16.h>

#include "ttc_device.cuh"
#include "ttc_internal.h"

namespace ttc {

constexpr int kCopyChunk = 4096;  // elements per block
constexpr int kCopyThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kCopyThreads) copy_cores_kernel(const __grid_constant__ CopyParams p) {
  int t = 0;
  while (t + 1 < p.n_tasks && blockIdx.x >= p.block_start[t + 1]) ++t;
  const CopyTask tk = p.task[t];
  const int64_t n = static_cast<int64_t>(tk.r0) * tk.I * tk.r1;
  const int64_t beg = (blockIdx.x - p.block_start[t]) * static_cast<int64_t>(kCopyChunk);
  const int64_t end = min(n, beg + kCopyChunk);
  const T* __restrict__ src = static_cast<const T*>(tk.src);
  T* __restrict__ dst = static_cast<T*>(tk.dst);
  if (!tk.swap) {
    for (int64_t e = beg + threadIdx.x; e < end; e += kCopyThreads) dst[e] = src[e];
  } else {
    // dst is [r1][I][r0]; element e of dst = (c1, i, c0)
    for (int64_t e = beg + threadIdx.x; e < end; e += kCopyThreads) {
      const int64_t c0 = e % tk.r0;
      const int64_t rest = e / tk.r0;
      const int64_t i = rest % tk.I;
      const int64_t c1 = rest / tk.I;
      dst[e] = src[(c0 * tk.I + i) * tk.r1 + c1];
    }
  }
}

cudaError_t launch_copy(const CopyParams& p, int elem_bytes, cudaStream_t s) {
  const int64_t blocks = p.block_start[p.n_tasks];
  if (blocks <= 0) return cudaSuccess;
  count_launch();
  dim3 grid(static_cast<unsigned>(blocks));
  if (elem_bytes == 8) copy_cores_kernel<double><<<grid, kCopyThreads, 0, s>>>(p);
  else if (elem_bytes == 4) copy_cores_kernel<float><<<grid, kCopyThreads, 0, s>>>(p);
  else copy_cores_kernel<unsigned short><<<grid, kCopyThreads, 0, s>>>(p);
  return cudaGetLastError();
}

// C for one mode index i per block (blockIdx.x = i), one output element per
// thread iteration.
//   lead : C[u][i][y] = sum_a gx[a][i][u] K[a][y],  u < rb, a < ra
//   trail: C[u][i][y] = sum_b gx[u][i][b] K[b][y],  u < ra, b < rb
template <typename T>
__global__ void __launch_bounds__(256) emit_c_kernel(const __grid_constant__ EmitCParams p) {
  const int i = blockIdx.x;
  const T* __restrict__ gx = static_cast<const T*>(p.gx);
  const T* __restrict__ k = static_cast<const T*>(p.k);
  T* __restrict__ c = static_cast<T*>(p.c_out);
  const int nu = p.lead ? p.rb : p.ra;
  const int nk = p.lead ? p.ra : p.rb;
  const int64_t lg = p.k_log2 != nullptr ? *p.k_log2 : 0;
  const bool fold = p.z_log2_out == nullptr && lg != 0;
  int bad = 0;
  for (int idx = threadIdx.x; idx < nu * p.ry; idx += blockDim.x) {
    const int u = idx / p.ry, y = idx % p.ry;
    T s = T(0);
    if (p.lead) {
      for (int a = 0; a < nk; ++a)
        s = fma(gx[(static_cast<int64_t>(a) * p.I + i) * p.rb + u], k[static_cast<int64_t>(a) * p.ry + y], s);
    } else {
      const T* row = gx + (static_cast<int64_t>(u) * p.I + i) * p.rb;
      for (int b = 0; b < nk; ++b) s = fma(row[b], k[static_cast<int64_t>(b) * p.ry + y], s);
    }
    if (fold) {
      const T s0 = s;
      s = scale_pow2_sat<T>(s, lg);
      if (isfinite(s0) && !isfinite(s)) bad |= TT_STATUS_OVERFLOW;
    }
    if (!isfinite(s)) bad |= TT_STATUS_NONFINITE;
    c[(static_cast<int64_t>(u) * p.I + i) * p.ry + y] = s;
  }
  if (bad) set_status(p.status, bad);
  if (i == 0 && threadIdx.x == 0 && p.z_log2_out != nullptr) *p.z_log2_out = lg;
}

cudaError_t launch_emit_c_f32(const EmitCParams& p, cudaStream_t s) {
  count_launch();
  emit_c_kernel<float><<<p.I, 256, 0, s>>>(p);
  return cudaGetLastError();
}
cudaError_t launch_emit_c_f64(const EmitCParams& p, cudaStream_t s) {
  count_launch();
  emit_c_kernel<double><<<p.I, 256, 0, s>>>(p);
  return cudaGetLastError();
}

template <typename T>
__global__ void fill_identity_kernel(T* k, int64_t* k_log2) {
  k[0] = T(1);
  if (k_log2 != nullptr) *k_log2 = 0;
}

cudaError_t launch_fill_identity(void* k, int64_t* k_log2, int elem_bytes, cudaStream_t s) {
  count_launch();
  if (elem_bytes == 8) fill_identity_kernel<double><<<1, 1, 0, s>>>(static_cast<double*>(k), k_log2);
  else fill_identity_kernel<float><<<1, 1, 0, s>>>(static_cast<float*>(k), k_log2);
  return cudaGetLastError();
}

}  // namespace ttc
