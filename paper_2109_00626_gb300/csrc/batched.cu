// Persistent batched contraction: one launch works through thousands of
// independent pairs of uneven order, mode size and rank.
//
// The grid holds as many CTAs as fit on the GPU at once.  Each CTA takes the
// next pair from a global counter (pairs are pre-sorted longest-first, so the
// queue is an LPT schedule) and runs the whole environment sweep of that pair
// -- and, for a partial contraction, its chain emission -- with the per-CTA
// engine of pair_engine.cuh, following the evaluation order and panels the
// plan chose for each mode.  The free-core copies of the partial pairs follow
// in a second kernel (copy_jobs.cuh), launched as a programmatic dependent so
// that it starts on the SMs the queue's tail leaves idle.  Nothing in the
// launch depends on the host: the counter is reset by a memset node, so the
// (memset, kernels) sequence can be captured in a CUDA graph and replayed.
#include "copy_jobs.cuh"
#include "pair_engine.cuh"

namespace ttc {

struct BatchKernelParams {
  const SweepParams* table;  // [n] per-pair sweep parameters
  const int32_t* order;      // [n] pair indices, longest first
  const int32_t* tile;       // [n] panel-budget level per pair (0, 1, 2: a quarter, half or all of the buffer)
  int n;
  const CopyJob* jobs;       // free-core copies of the partial pairs
  int n_jobs;
  int* counter;              // [0] pair queue head (zeroed before the launch)
  double* out;               // [n]
  int64_t* out_log2;         // [n] or NULL
  int32_t* status;
};

constexpr int kBatchThreads = eng::NTOT;

template <typename T>
__global__ void __launch_bounds__(eng::NTOT, 1) batched_kernel(const __grid_constant__ BatchKernelParams bp) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_idx;
  // The copy kernel that follows depends on none of this launch's work: let it
  // take each SM this launch leaves (it waits for this grid before it ends).
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
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

// Free-core copies of the partial pairs (they depend on no sweep): job j to
// CTA j mod grid (copy_jobs.cuh).
template <typename T>
__global__ void __launch_bounds__(kCopyThreads) copy_jobs_kernel(const CopyJob* __restrict__ jobs, int n_jobs) {
  extern __shared__ __align__(16) unsigned char copy_smem[];
  T* const buf0 = reinterpret_cast<T*>(copy_smem);
  copy_jobs_block<T>([&](int jb) { return jobs[jb]; }, blockIdx.x, n_jobs, gridDim.x, buf0, buf0 + copy_buf_elems<T>());
  // Launched as a programmatic dependent of the batched kernel: end only once
  // that grid has completed, so that stream order holds for later work.
  asm volatile("griddepcontrol.wait;" ::: "memory");
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
  const size_t csmem = copy_smem_bytes<T>();
  err = cudaFuncSetAttribute(copy_jobs_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(csmem));
  if (err != cudaSuccess) return err;
  int cper = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cper, copy_jobs_kernel<T>, kCopyThreads, csmem);
  if (err != cudaSuccess) return err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(std::min(bp.n_jobs, sms * std::max(cper, 1)));
  cfg.blockDim = dim3(kCopyThreads);
  cfg.dynamicSmemBytes = csmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;  // start on the SMs the sweeps leave
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, copy_jobs_kernel<T>, bp.jobs, bp.n_jobs);
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
