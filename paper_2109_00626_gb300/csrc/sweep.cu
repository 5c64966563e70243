// Single-contraction launches of the environment sweep (sweep_body.cuh): one
// thread-block cluster of up to 16 CTAs splits every contracted mode over its
// mode index; a cluster of one CTA runs the same body without the
// distributed-shared-memory reduction; a full contraction with a workspace
// runs as two clusters sweeping from both ends.
#include "sweep_body.cuh"

namespace ttc {

// A chain-layout partial contraction launched with two clusters gives the
// free-core copies (which depend on nothing) to the second one, so they run
// while the first sweeps.
template <typename T, int RM>
__global__ void __launch_bounds__(256, 1) sweep_cluster_kernel(const __grid_constant__ SweepParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int C = static_cast<int>(cluster.num_blocks());
  const int crank = static_cast<int>(cluster.block_rank());
  if (blockIdx.x >= static_cast<unsigned>(C)) {
    constexpr int NT = SweepCfg<T, RM, true>::NT;
    const int64_t g = static_cast<int64_t>(crank) * NT + threadIdx.x, gs = static_cast<int64_t>(C) * NT;
    for (int t = 0; t < p.emit.n_copies; ++t) {
      const CopyTask& tk = p.emit.copy[t];
      const T* __restrict__ src = static_cast<const T*>(tk.src);
      T* __restrict__ dst = static_cast<T*>(tk.dst);
      if (!tk.swap) copy_plain<T>(dst, src, static_cast<int64_t>(tk.r0) * tk.I * tk.r1, g, gs);
      else copy_swap_tiled<T, NT>(dst, src, tk.r0, tk.I, tk.r1, reinterpret_cast<T*>(smem), C, crank);
    }
    return;
  }
  SweepState<T, RM, true> st;
  SweepOut o{p.z_out, p.z_out_log2, p.status};
  o.skip_copies = gridDim.x > static_cast<unsigned>(C) ? 1 : 0;
  if (sweep_body<T, RM, true>(p, o, smem, C, crank, st)) {
    sweep_tail<T, RM, true>(p, o, smem, C, crank, st);
    cluster.sync();  // peers may still be reading this CTA's reduced rows
  }
}

// Full contraction from both ends: cluster 0 sweeps the leading modes left to
// right, cluster 1 the trailing ones right to left, each on its own SMs, and
// the two environments meet in the middle, z = sum_{a,b} E_L[a][b] F_R[a][b]
// (float64).  Each cluster writes its environment (mantissa and power-of-two
// scale) to the workspace; the one that finishes second (a counter in the
// workspace, zeroed before the launch) forms z.  No cluster waits for the
// other, so nothing depends on both being resident at once.
template <typename T, int RM>
__global__ void __launch_bounds__(256, 1) sweep_two_sided_kernel(const __grid_constant__ TwoSidedParams tp) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_last;
  __shared__ double s_red[8];
  cg::cluster_group cluster = cg::this_cluster();
  const int C = static_cast<int>(cluster.num_blocks());
  const int crank = static_cast<int>(cluster.block_rank());
  const int side = static_cast<int>(blockIdx.x) / C;
  const SweepParams& p = tp.half[side];
  SweepState<T, RM, true> st;
  const SweepOut o{nullptr, nullptr, tp.status};
  if (sweep_body<T, RM, true>(p, o, smem, C, crank, st)) {
    sweep_tail<T, RM, true>(p, o, smem, C, crank, st);
    cluster.sync();  // peers may still be reading this CTA's reduced rows
  }
  if (crank != 0) return;
  __threadfence();  // this cluster's environment and scale are visible before the count
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(tp.counter, 1);
  __syncthreads();
  if (s_last != 1) return;
  __threadfence();
  const T* el = static_cast<const T*>(tp.half[0].e_out);
  const T* er = static_cast<const T*>(tp.half[1].e_out);
  const int n = tp.rx * tp.ry;
  double part = 0.0;
  // eight pairs of loads in flight per thread before the first product
  const int nt = static_cast<int>(blockDim.x);
  for (int base = threadIdx.x; base < n; base += 8 * nt) {
    T a[8], b[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = base + u * nt;
      a[u] = i < n ? __ldcg(el + i) : T(0);
      b[u] = i < n ? __ldcg(er + i) : T(0);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) part = fma(static_cast<double>(a[u]), static_cast<double>(b[u]), part);
  }
  part = warp_sum(part);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) s_red[warp] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double z = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x) / 32; ++w) z += s_red[w];
    const int64_t log2s = __ldcg(tp.half[0].e_out_log2) + __ldcg(tp.half[1].e_out_log2);
    int st_bits = isfinite(z) ? 0 : TT_STATUS_NONFINITE;
    if (tp.z_out_log2 != nullptr) {
      *tp.z_out = z;
      *tp.z_out_log2 = log2s;
    } else {
      double v = z;
      if (z != 0.0 && isfinite(z)) {
        const int64_t tot = static_cast<int64_t>(exp2_of(z)) + log2s;
        if (tot > 1024) {
          v = z > 0 ? INFINITY : -INFINITY;
          st_bits |= TT_STATUS_OVERFLOW;
        } else if (tot < -1074) {
          v = 0.0;
        } else {
          v = ldexp(z, static_cast<int>(log2s));
        }
      }
      *tp.z_out = v;
    }
    set_status(tp.status, st_bits);
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
  err = cudaFuncSetAttribute(sweep_two_sided_kernel<T, RM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(SweepCfg<T, RM, true>::SMEM));
  if (err != cudaSuccess) return err;
  err = cudaFuncSetAttribute(sweep_two_sided_kernel<T, RM>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
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
  // a second cluster takes the free-core copies of a chain emission
  cfg.gridDim = dim3(p.emit.enabled && p.emit.n_copies > 0 ? 2 * C : C, 1, 1);
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
static cudaError_t launch_two_sided_impl(const TwoSidedParams& tp, int C, cudaStream_t s) {
  cudaError_t err = prepare<T, RM>();
  if (err != cudaSuccess) return err;
  count_launch();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * C, 1, 1);
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
  return cudaLaunchKernelEx(&cfg, sweep_two_sided_kernel<T, RM>, tp);
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

cudaError_t launch_two_sided(const TwoSidedParams& tp, int dtype, int rmax, int C, cudaStream_t s) {
  if (C < 2) return cudaErrorInvalidValue;  // the kernel reduces across a cluster
  if (dtype == TT_F64) {
    if (rmax <= 32) return launch_two_sided_impl<double, 32>(tp, C, s);
    if (rmax <= 64) return launch_two_sided_impl<double, 64>(tp, C, s);
    return cudaErrorInvalidValue;
  }
  if (rmax <= 32) return launch_two_sided_impl<float, 32>(tp, C, s);
  if (rmax <= 64) return launch_two_sided_impl<float, 64>(tp, C, s);
  if (rmax <= 128) return launch_two_sided_impl<float, 128>(tp, C, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_sweep_f64(const SweepParams& p, int rmax, int C, cudaStream_t s) {
  if (rmax <= 32) return launch_impl<double, 32>(p, C, s);
  if (rmax <= 64) return launch_impl<double, 64>(p, C, s);
  return cudaErrorInvalidValue;
}

}  // namespace ttc
