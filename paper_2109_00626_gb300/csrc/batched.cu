// Persistent batched contraction: one launch works through thousands of
// independent pairs of uneven order, mode size and rank.
//
// The grid holds as many CTAs as fit on the GPU at once.  Each CTA takes the
// next pair from a global counter (pairs are pre-sorted longest-first, so the
// queue is an LPT schedule) and runs the whole environment sweep of that pair
// -- and, for a partial contraction, its chain emission -- with the per-CTA
// engine of pair_engine.cuh, following the evaluation order and panels the plan chose
// for each mode.  Nothing in
// the launch depends on the host: the counter is reset by a memset node, so
// the pair (memset, kernel) can be captured in a CUDA graph and replayed.
#include "pair_engine.cuh"

namespace ttc {

struct BatchKernelParams {
  const SweepParams* table;  // [n] per-pair sweep parameters
  const int32_t* order;      // [n] pair indices, longest first
  const int32_t* tile;       // [n] rank tile per pair: 0 -> 32, 1 -> 64, 2 -> 128
  int n;
  const CopyJob* jobs;       // free-core copies of the partial pairs
  int n_jobs;
  int* counter;              // [0] pair queue head, [1] copy queue head (zeroed before the launch)
  double* out;               // [n]
  int64_t* out_log2;         // [n] or NULL
  int32_t* status;
};

constexpr int kBatchThreads = eng::NTOT;

template <typename T>
__global__ void __launch_bounds__(eng::NTOT, 1) batched_kernel(const __grid_constant__ BatchKernelParams bp) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_idx;
  for (;;) {
    __syncthreads();  // every thread has read the previous s_idx
    if (threadIdx.x == 0) s_idx = atomicAdd(bp.counter, 1);
    __syncthreads();
    const int idx = s_idx;
    if (idx >= bp.n) break;
    const int pair = bp.order[idx];
    SweepOut o{bp.out + pair, bp.out_log2 != nullptr ? bp.out_log2 + pair : nullptr, bp.status};
    o.skip_copies = 1;
    eng::run_pair<T>(bp.table[pair], o, smem);
  }
}

// Free-core copies of the partial pairs (they depend on no sweep).  A grid of
// many small CTAs per SM keeps enough loads in flight to run at memory speed;
// jobs are dealt statically (job j to CTA j mod grid), so no scratch is used.
template <typename T>
__global__ void __launch_bounds__(256) copy_jobs_kernel(const CopyJob* __restrict__ jobs, int n_jobs) {
  __shared__ T tile[32 * 33];
  constexpr int U = 8;
  for (int jb = blockIdx.x; jb < n_jobs; jb += gridDim.x) {
    const CopyJob j = jobs[jb];
    const T* __restrict__ src = static_cast<const T*>(j.src);
    T* __restrict__ dst = static_cast<T*>(j.dst);
    if (!j.swap) {
      const int64_t run = static_cast<int64_t>(j.i1 - j.i0) * j.r1;
      const int64_t total = static_cast<int64_t>(j.r0) * run;
      for (int64_t e0 = threadIdx.x; e0 < total; e0 += static_cast<int64_t>(U) * blockDim.x) {
        T v[U];
        int64_t idx[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t e = e0 + static_cast<int64_t>(u) * blockDim.x;
          idx[u] = -1;
          if (e < total) {
            const int64_t c0 = e / run, off = e - c0 * run;
            idx[u] = (c0 * j.I + j.i0) * j.r1 + off;
            v[u] = ldg(src + idx[u]);
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (idx[u] >= 0) dst[idx[u]] = v[u];
      }
    } else {
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
      const int t0 = (j.r0 + 31) / 32, t1 = (j.r1 + 31) / 32;
      for (int i = j.i0; i < j.i1; ++i)
        for (int tt = 0; tt < t0 * t1; ++tt) {
          const int b0 = (tt / t1) * 32, b1 = (tt % t1) * 32;
          __syncthreads();
#pragma unroll
          for (int rr = warp; rr < 32; rr += 8) {
            const int c0 = b0 + rr, c1 = b1 + lane;
            if (c0 < j.r0 && c1 < j.r1) tile[rr * 33 + lane] = src[(static_cast<int64_t>(c0) * j.I + i) * j.r1 + c1];
          }
          __syncthreads();
#pragma unroll
          for (int rr = warp; rr < 32; rr += 8) {
            const int c1 = b1 + rr, c0 = b0 + lane;
            if (c0 < j.r0 && c1 < j.r1) dst[(static_cast<int64_t>(c1) * j.I + i) * j.r0 + c0] = tile[lane * 33 + rr];
          }
        }
    }
  }
}

template <typename T>
static cudaError_t launch_batched_impl(const BatchKernelParams& bp, int grid, cudaStream_t s) {
  const size_t smem = eng::smem_bytes<T>();
  cudaError_t err =
      cudaFuncSetAttribute(batched_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  if (grid <= 0) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batched_kernel<T>, kBatchThreads, smem);
    if (err != cudaSuccess) return err;
    grid = sms * std::max(per, 1);
  }
  grid = std::min(grid, std::max(bp.n, 1));
  count_launch();
  batched_kernel<T><<<grid, kBatchThreads, smem, s>>>(bp);
  err = cudaGetLastError();
  if (err != cudaSuccess || bp.n_jobs == 0) return err;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  count_launch();
  copy_jobs_kernel<T><<<std::min(bp.n_jobs, sms * 8), 256, 0, s>>>(bp.jobs, bp.n_jobs);
  return cudaGetLastError();
}

cudaError_t launch_batched(const void* table, const int32_t* order, const int32_t* tile, int n,
                           const CopyJob* jobs, int n_jobs, int* counters, double* out, int64_t* out_log2,
                           int32_t* status, int dtype, int grid, cudaStream_t s) {
  BatchKernelParams bp;
  bp.table = static_cast<const SweepParams*>(table);
  bp.order = order;
  bp.tile = tile;
  bp.n = n;
  bp.jobs = jobs;
  bp.n_jobs = n_jobs;
  bp.counter = counters;
  bp.out = out;
  bp.out_log2 = out_log2;
  bp.status = status;
  if (dtype == TT_F64) return launch_batched_impl<double>(bp, grid, s);
  return launch_batched_impl<float>(bp, grid, s);
}

}  // namespace ttc
