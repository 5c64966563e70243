// Single-contraction launches of the environment sweep (sweep_body.cuh): one
// thread-block cluster of up to 16 CTAs splits every contracted mode over its
// mode index; a cluster of one CTA runs the same body without the
// distributed-shared-memory reduction.
#include "sweep_body.cuh"

namespace ttc {

template <typename T, int RM>
__global__ void __launch_bounds__(256, 1) sweep_cluster_kernel(const __grid_constant__ SweepParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int C = static_cast<int>(cluster.num_blocks());
  const int crank = static_cast<int>(cluster.block_rank());
  SweepState<T, RM, true> st;
  const SweepOut o{p.z_out, p.z_out_log2, p.status};
  if (sweep_body<T, RM, true>(p, o, smem, C, crank, st)) {
    sweep_tail<T, RM, true>(p, o, smem, C, crank, st);
    cluster.sync();  // peers may still be reading this CTA's reduced rows
  }
}

template <typename T, int RM>
__global__ void __launch_bounds__(512, 1) sweep_cta_kernel(const __grid_constant__ SweepParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  SweepState<T, RM, false> st;
  const SweepOut o{p.z_out, p.z_out_log2, p.status};
  if (sweep_body<T, RM, false>(p, o, smem, 1, 0, st)) sweep_tail<T, RM, false>(p, o, smem, 1, 0, st);
}

template <typename T, int RM>
static cudaError_t prepare() {
  cudaError_t err = cudaFuncSetAttribute(sweep_cluster_kernel<T, RM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(SweepCfg<T, RM, true>::SMEM));
  if (err != cudaSuccess) return err;
  err = cudaFuncSetAttribute(sweep_cluster_kernel<T, RM>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (err != cudaSuccess) return err;
  return cudaFuncSetAttribute(sweep_cta_kernel<T, RM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(SweepCfg<T, RM, false>::SMEM));
}

template <typename T, int RM>
static cudaError_t launch_impl(const SweepParams& p, int C, cudaStream_t s) {
  cudaError_t err = prepare<T, RM>();
  if (err != cudaSuccess) return err;
  count_launch();
  if (C == 1) {
    sweep_cta_kernel<T, RM><<<1, SweepCfg<T, RM, false>::NT, SweepCfg<T, RM, false>::SMEM, s>>>(p);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(SweepCfg<T, RM, true>::NT, 1, 1);
  cfg.dynamicSmemBytes = SweepCfg<T, RM, true>::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, sweep_cluster_kernel<T, RM>, p);
}

template <typename T, int RM>
static int cluster_size_impl(int want) {
  if (prepare<T, RM>() != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  for (int C = want; C >= 2; C /= 2) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(SweepCfg<T, RM, true>::NT, 1, 1);
    cfg.dynamicSmemBytes = SweepCfg<T, RM, true>::SMEM;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, sweep_cluster_kernel<T, RM>, &cfg) == cudaSuccess && n >= 1) return C;
    cudaGetLastError();
  }
  return 1;
}

// Cached per (element size, rank tile, wanted size, device).
int sweep_cluster_size(int rmax, int elem_bytes, int want) {
  static int cache[2][3][17][8];  // 0 = unknown
  int dev = 0;
  cudaGetDevice(&dev);
  const int tile = rmax <= 32 ? 0 : (rmax <= 64 ? 1 : 2);
  const int d = elem_bytes == 8 ? 1 : 0;
  int* slot = (dev >= 0 && dev < 8 && want >= 1 && want <= 16) ? &cache[d][tile][want][dev] : nullptr;
  if (slot != nullptr && *slot > 0) return *slot;
  int c = 0;
  if (want <= 1) {
    c = 1;
  } else if (elem_bytes == 4) {
    c = tile == 0 ? cluster_size_impl<float, 32>(want)
                  : (tile == 1 ? cluster_size_impl<float, 64>(want) : cluster_size_impl<float, 128>(want));
  } else {
    c = tile == 0 ? cluster_size_impl<double, 32>(want) : cluster_size_impl<double, 64>(want);
  }
  if (slot != nullptr && c > 0) *slot = c;
  return c;
}

cudaError_t launch_sweep_f32(const SweepParams& p, int rmax, int C, cudaStream_t s) {
  if (rmax <= 32) return launch_impl<float, 32>(p, C, s);
  if (rmax <= 64) return launch_impl<float, 64>(p, C, s);
  if (rmax <= 128) return launch_impl<float, 128>(p, C, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_sweep_f64(const SweepParams& p, int rmax, int C, cudaStream_t s) {
  if (rmax <= 32) return launch_impl<double, 32>(p, C, s);
  if (rmax <= 64) return launch_impl<double, 64>(p, C, s);
  return cudaErrorInvalidValue;
}

}  // namespace ttc
