// Environment sweep over contracted modes on one thread-block cluster.
//
// One contracted mode folds the core pair into the running environment
// (the generalisation of Algorithm 2 step 4 / Example 1's K = A_x^T A_y):
//   E'[u][v] = sum_i  (A_i^T E B_i)[u][v]
// with A_i, B_i the i-th slices of the two cores (see SweepStep).  The sum
// over the mode index i is split across the CTAs of one cluster: CTA c owns
// slices i = c, c + C, ...  Each CTA computes, per slice, the two small
// products T = E B_i and P += A_i^T T out of shared memory with a
// register-blocked outer-product loop, then the cluster adds the partial P's
// through distributed shared memory (fixed order, so the result is
// deterministic) and every CTA receives the full E' for the next mode.
//
// Scaling: after each mode the largest |E'| is compared with 2^+-s; outside
// that band E' is multiplied by an exact power of two and the exponent is
// accumulated in an int64, so long sweeps cannot overflow or underflow.
//
// The last step of a full contraction (both right ranks 1) is summed in
// float64: t_i[p] = sum_q E[p][q] B_i[q] in the storage type, then
// z = sum_{i,p} A_i[p] t_i[p] in double, cluster-reduced in double.
#include <cooperative_groups.h>

#include "ttc_device.cuh"
#include "ttc_internal.h"

namespace cg = cooperative_groups;

namespace ttc {

constexpr int kNoExp = -(1 << 30);  // exponent marker of an all-zero environment

template <typename T, int RM>
struct SweepCfg {
  static constexpr int NT = 256;
  static constexpr int TM = RM / 16;               // thread tile is TM x TM
  static constexpr int LD = RM + 16 / sizeof(T);   // row stride (elements), 16-byte padded
  static constexpr int TILE = RM * LD;
  static constexpr size_t SMEM = 3 * TILE * sizeof(T) + 64 * sizeof(double);
};

// dst[r][c] (row stride LD) = slice i of a core.
//   transposed == 0: core is [rows][I][cols], dst[r][c] = core[r][i][c]
//   transposed == 1: core is [cols][I][rows], dst[r][c] = core[c][i][r]
template <typename T, int LD, int NT>
__device__ __forceinline__ void load_slice(T* __restrict__ dst, const T* __restrict__ core, int i,
                                           int I, int rows, int cols, int transposed) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NW = NT / 32;
  if (!transposed) {
    for (int r = warp; r < rows; r += NW) {
      const T* src = core + (static_cast<int64_t>(r) * I + i) * cols;
      for (int c = lane; c < cols; c += 32) dst[r * LD + c] = ldg(src + c);
    }
  } else {
    for (int c = warp; c < cols; c += NW) {
      const T* src = core + (static_cast<int64_t>(c) * I + i) * rows;
      for (int r = lane; r < rows; r += 32) dst[r * LD + c] = ldg(src + r);
    }
  }
}

template <typename T, int RM>
__global__ void __launch_bounds__(256, 1) sweep_cluster_kernel(const __grid_constant__ SweepParams p) {
  using Cfg = SweepCfg<T, RM>;
  constexpr int NT = Cfg::NT, TM = Cfg::TM, LD = Cfg::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Es = reinterpret_cast<T*>(smem_raw);      // E transposed: Es[q][p] = E[p][q]
  T* Ss = Es + Cfg::TILE;                      // slice buffer (B_i, then A_i)
  T* Ts = Ss + Cfg::TILE;                      // T = E B_i, later the partial P
  double* red = reinterpret_cast<double*>(Ts + Cfg::TILE);  // 64 doubles of scratch

  cg::cluster_group cluster = cg::this_cluster();
  const int C = static_cast<int>(cluster.num_blocks());
  const int crank = static_cast<int>(cluster.block_rank());
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  const int warp = tid >> 5, lane = tid & 31;

  int64_t log2s = 0;
  int bad = 0;

  // start environment
  {
    const int rx0 = p.step[0].rin_x, ry0 = p.step[0].rin_y;
    if (p.e_in == nullptr) {
      if (tid == 0) Es[0] = T(1);
    } else {
      const T* e = static_cast<const T*>(p.e_in);
      for (int idx = tid; idx < rx0 * ry0; idx += NT) {
        const int a = idx / ry0, b = idx % ry0;
        Es[b * LD + a] = e[idx];
      }
      if (p.e_in_log2 != nullptr) log2s = *p.e_in_log2;
    }
  }
  __syncthreads();

  for (int j = 0; j < p.n_steps; ++j) {
    const SweepStep st = p.step[j];
    const T* gx = static_cast<const T*>(st.gx);
    const T* gy = static_cast<const T*>(st.gy);
    const int I = st.I;

    if (p.final_scalar && j == p.n_steps - 1) {
      // ---- last mode of a full contraction: float64 sum ----
      T* bvec = Ss;       // B_i[q][0]
      T* avec = Ss + LD;  // A_i[p][0]
      double part = 0.0;
      for (int i = crank; i < I; i += C) {
        // rout = 1: B_i[q] = gy[q][i][0] (left) or gy[0][i][q] (right); same for A
        for (int q = tid; q < st.rin_y; q += NT)
          bvec[q] = p.transposed ? ldg(gy + static_cast<int64_t>(i) * st.rin_y + q)
                                 : ldg(gy + static_cast<int64_t>(q) * I + i);
        for (int a = tid; a < st.rin_x; a += NT)
          avec[a] = p.transposed ? ldg(gx + static_cast<int64_t>(i) * st.rin_x + a)
                                 : ldg(gx + static_cast<int64_t>(a) * I + i);
        __syncthreads();
        for (int a = tid; a < st.rin_x; a += NT) {
          T t = T(0);
          for (int q = 0; q < st.rin_y; ++q) t = fma(Es[q * LD + a], bvec[q], t);
          part = fma(static_cast<double>(avec[a]), static_cast<double>(t), part);
        }
        __syncthreads();
      }
      part = warp_sum(part);
      if (lane == 0) red[warp] = part;
      __syncthreads();
      if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < NT / 32; ++w) s += red[w];
        red[32] = s;
      }
      cluster.sync();
      if (crank == 0 && tid == 0) {
        double z = 0.0;
        for (int r = 0; r < C; ++r) z += *cluster.map_shared_rank(red + 32, r);
        int st_bits = (isfinite(z) && !bad) ? 0 : TT_STATUS_NONFINITE;
        if (p.z_out_log2 != nullptr) {
          *p.z_out = z;
          *p.z_out_log2 = log2s;
        } else {
          double v = z;
          if (z != 0.0 && isfinite(z)) {
            int ez = exp2_of(z);
            const int64_t tot = static_cast<int64_t>(ez) + log2s;
            if (tot > 1024) {
              v = z > 0 ? INFINITY : -INFINITY;
              st_bits |= TT_STATUS_OVERFLOW;
            } else if (tot < -1074) {
              v = 0.0;
            } else {
              v = ldexp(z, static_cast<int>(log2s));
            }
          }
          *p.z_out = v;
        }
        set_status(p.status, st_bits);
      }
      cluster.sync();  // keep peers' shared memory alive until CTA 0 has read it
      return;
    }

    // ---- one contracted mode: E' = sum_i A_i^T E B_i ----
    T acc[TM][TM];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TM; ++b) acc[a][b] = T(0);

    const int p0 = ty * TM, v0 = tx * TM;
    for (int i = crank; i < I; i += C) {
      load_slice<T, LD, NT>(Ss, gy, i, I, st.rin_y, st.rout_y, p.transposed);
      __syncthreads();
      T t[TM][TM];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TM; ++b) t[a][b] = T(0);
      if (p0 < st.rin_x && v0 < st.rout_y) {
#pragma unroll 4
        for (int q = 0; q < st.rin_y; ++q) {
          T av[TM], bv[TM];
          ld_vec<T, TM>(av, Es + q * LD + p0);
          ld_vec<T, TM>(bv, Ss + q * LD + v0);
#pragma unroll
          for (int a = 0; a < TM; ++a)
#pragma unroll
            for (int b = 0; b < TM; ++b) t[a][b] = fma(av[a], bv[b], t[a][b]);
        }
      }
      __syncthreads();
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TM; ++b) Ts[(p0 + a) * LD + v0 + b] = t[a][b];
      load_slice<T, LD, NT>(Ss, gx, i, I, st.rin_x, st.rout_x, p.transposed);
      __syncthreads();
      const int u0 = ty * TM;
      if (u0 < st.rout_x && v0 < st.rout_y) {
#pragma unroll 4
        for (int q = 0; q < st.rin_x; ++q) {
          T av[TM], bv[TM];
          ld_vec<T, TM>(av, Ss + q * LD + u0);
          ld_vec<T, TM>(bv, Ts + q * LD + v0);
#pragma unroll
          for (int a = 0; a < TM; ++a)
#pragma unroll
            for (int b = 0; b < TM; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
      }
      __syncthreads();
    }

    // ---- cluster reduction: E'[u][v] = sum over CTAs of P_c[u][v] ----
    {
      const int u0 = ty * TM;
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TM; ++b) Ts[(u0 + a) * LD + v0 + b] = acc[a][b];
    }
    cluster.sync();
    const int nu = st.rout_x, nv = st.rout_y;
    const int chunk = (nu + C - 1) / C;
    const int ub = min(nu, crank * chunk), ue = min(nu, ub + chunk);
    int lexp = kNoExp;  // largest binary exponent among the entries this CTA reduced
    int lbad = 0;
    for (int idx = tid; idx < (ue - ub) * nv; idx += NT) {
      const int u = ub + idx / nv, v = idx % nv;
      T s = T(0);
      for (int r = 0; r < C; ++r) s += *cluster.map_shared_rank(Ts + u * LD + v, r);
      for (int r = 0; r < C; ++r) *cluster.map_shared_rank(Es + v * LD + u, r) = s;
      if (!isfinite(s)) lbad = 1;
      else if (s != T(0)) lexp = max(lexp, exp2_of(static_cast<double>(s)));
    }
    lexp = __reduce_max_sync(0xffffffffu, lexp);
    lbad = __reduce_or_sync(0xffffffffu, lbad);
    int* ired = reinterpret_cast<int*>(red);
    if (lane == 0) {
      ired[warp] = lexp;
      ired[16 + warp] = lbad;
    }
    __syncthreads();
    if (tid == 0) {
      int m = kNoExp, bb = 0;
      for (int w = 0; w < NT / 32; ++w) {
        m = max(m, ired[w]);
        bb |= ired[16 + w];
      }
      for (int r = 0; r < C; ++r) {
        *cluster.map_shared_rank(ired + 32 + crank, r) = m;
        *cluster.map_shared_rank(ired + 64 + crank, r) = bb;
      }
    }
    cluster.sync();
    int gexp = kNoExp, gbad = 0;
    for (int r = 0; r < C; ++r) {
      gexp = max(gexp, ired[32 + r]);
      gbad |= ired[64 + r];
    }
    if (gbad) bad = 1;
    if (gexp != kNoExp && (gexp > p.renorm_bits || gexp < -p.renorm_bits)) {
      for (int idx = tid; idx < nu * nv; idx += NT) {
        const int u = idx / nv, v = idx % nv;
        Es[v * LD + u] = mul_pow2<T>(Es[v * LD + u], -gexp);
      }
      log2s += gexp;
    }
    __syncthreads();
  }

  // ---- environment output (partial contractions, backward seeds) ----
  if (crank == 0 && p.e_out != nullptr) {
    const SweepStep st = p.step[p.n_steps - 1];
    T* e = static_cast<T*>(p.e_out);
    for (int idx = tid; idx < st.rout_x * st.rout_y; idx += NT) {
      const int u = idx / st.rout_y, v = idx % st.rout_y;
      e[idx] = Es[v * LD + u];
    }
    if (tid == 0 && p.e_out_log2 != nullptr) *p.e_out_log2 = log2s;
  }
  if (tid == 0 && crank == 0) set_status(p.status, bad ? TT_STATUS_NONFINITE : 0);
  cluster.sync();
}

template <typename T, int RM>
static cudaError_t launch_impl(const SweepParams& p, int C, cudaStream_t s) {
  auto kern = sweep_cluster_kernel<T, RM>;
  const size_t smem = SweepCfg<T, RM>::SMEM;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  if (C > 8) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (err != cudaSuccess) return err;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(SweepCfg<T, RM>::NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, kern, p);
}

template <typename T, int RM>
static int cluster_size_impl(int want) {
  auto kern = sweep_cluster_kernel<T, RM>;
  const size_t smem = SweepCfg<T, RM>::SMEM;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
    return 0;
  cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  for (int C = want; C >= 1; C /= 2) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(SweepCfg<T, RM>::NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n >= 1) return C;
    cudaGetLastError();
  }
  return 0;
}

int sweep_cluster_size(int rmax, int elem_bytes, int want) {
  if (elem_bytes == 4) {
    if (rmax <= 32) return cluster_size_impl<float, 32>(want);
    if (rmax <= 64) return cluster_size_impl<float, 64>(want);
    return cluster_size_impl<float, 128>(want);
  }
  if (rmax <= 32) return cluster_size_impl<double, 32>(want);
  return cluster_size_impl<double, 64>(want);
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
