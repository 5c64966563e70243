// Persistent batched contraction: one launch works through thousands of
// independent pairs of uneven order, mode size and rank.
//
// The grid holds as many CTAs as fit on the GPU at once.  Each CTA takes the
// next pair from a global counter (pairs are pre-sorted longest-first, so the
// queue is an LPT schedule) and runs the whole environment sweep of that pair
// -- and, for a partial contraction, its chain emission -- with the shared
// sweep body, using the rank tile the plan chose for the pair.  Nothing in
// the launch depends on the host: the counter is reset by a memset node, so
// the pair (memset, kernel) can be captured in a CUDA graph and replayed.
#include "sweep_body.cuh"

namespace ttc {

struct BatchKernelParams {
  const SweepParams* table;  // [n] per-pair sweep parameters
  const int32_t* order;      // [n] pair indices, longest first
  const int32_t* tile;       // [n] rank tile per pair: 0 -> 32, 1 -> 64, 2 -> 128
  int n;
  int* counter;              // work queue head (zeroed before the launch)
  double* out;               // [n]
  int64_t* out_log2;         // [n] or NULL
  int32_t* status;
};

constexpr int kBatchThreads = SweepCfg<float, 128, false>::NT;
static_assert(SweepCfg<double, 64, false>::NT == kBatchThreads, "one block size for every tile");

template <typename T, int RM>
__device__ __forceinline__ void run_pair(const SweepParams& p, const SweepOut& o, unsigned char* smem) {
  SweepState<T, RM, false> st;
  if (sweep_body<T, RM, false>(p, o, smem, 1, 0, st)) sweep_tail<T, RM, false>(p, o, smem, 1, 0, st);
}

template <typename T>
struct BatchSmem {
  static constexpr size_t value =
      sizeof(T) == 4 ? SweepCfg<float, 128, false>::SMEM : SweepCfg<double, 64, false>::SMEM;
};

template <typename T>
__global__ void __launch_bounds__(512, 1) batched_kernel(const __grid_constant__ BatchKernelParams bp) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_idx;
  for (;;) {
    __syncthreads();  // every thread has read the previous s_idx
    if (threadIdx.x == 0) s_idx = atomicAdd(bp.counter, 1);
    __syncthreads();
    const int idx = s_idx;
    if (idx >= bp.n) break;
    const int pair = bp.order[idx];
    const SweepParams& p = bp.table[pair];
    const SweepOut o{bp.out + pair, bp.out_log2 != nullptr ? bp.out_log2 + pair : nullptr, bp.status};
    const int tile = bp.tile[pair];
    if constexpr (sizeof(T) == 4) {
      if (tile == 0) run_pair<T, 32>(p, o, smem);
      else if (tile == 1) run_pair<T, 64>(p, o, smem);
      else run_pair<T, 128>(p, o, smem);
    } else {
      if (tile == 0) run_pair<T, 32>(p, o, smem);
      else run_pair<T, 64>(p, o, smem);
    }
  }
}

template <typename T>
static cudaError_t launch_batched_impl(const BatchKernelParams& bp, int grid, cudaStream_t s) {
  const size_t smem = BatchSmem<T>::value;
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
  return cudaGetLastError();
}

cudaError_t launch_batched(const void* table, const int32_t* order, const int32_t* tile, int n, int* counter,
                           double* out, int64_t* out_log2, int32_t* status, int dtype, int grid, cudaStream_t s) {
  BatchKernelParams bp;
  bp.table = static_cast<const SweepParams*>(table);
  bp.order = order;
  bp.tile = tile;
  bp.n = n;
  bp.counter = counter;
  bp.out = out;
  bp.out_log2 = out_log2;
  bp.status = status;
  if (dtype == TT_F64) return launch_batched_impl<double>(bp, grid, s);
  return launch_batched_impl<float>(bp, grid, s);
}

}  // namespace ttc
