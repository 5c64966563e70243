// Adjoint of a full contraction whose second operand has every rank 1.  The
// sum of a TT's entries is its contraction with the all-ones rank-1 TT -- the
// usual way a partial contraction is reduced to a loss -- and with one operand
// of rank 1 the environments are vectors (y_k[i] = Gy_k[0][i][0]):
//   L_0 = 1,  L_{k+1}[a'] = sum_{a,i} L_k[a] y_k[i] Gx_k[a][i][a']
//   F_N = 1,  F_k[a]      = sum_{i,a'} Gx_k[a][i][a'] y_k[i] F_{k+1}[a']
// and, z being linear in each core (Eq. 9), the gradients are
//   dGx_k[a][i][a'] = g L_k[a] y_k[i] F_{k+1}[a']
//   dGy_k[0][i][0]  = g sum_{a,a'} L_k[a] Gx_k[a][i][a'] F_{k+1}[a'].
// One launch sweeps L and F at the same time (a cluster each), each mode a
// matrix-vector product over one core read once, and keeps every vector with
// a power-of-two scale (no checkpoints: the vectors are small); a second
// launch writes the gradients, one block per (k, i).
#include <cooperative_groups.h>

#include "ttc_device.cuh"
#include "ttc_internal.h"

namespace cg = cooperative_groups;

namespace ttc {

namespace {

constexpr int kR1Threads = 512;
constexpr int kR1Cluster = 8;  // CTAs per sweep direction
constexpr int kR1Warps = kR1Threads / 32;
constexpr int kNoExpR1 = -(1 << 30);

// Block-wide max of an exponent and OR of a flag (every thread gets both).
// One barrier: callers alternate `red` between two buffers, so the previous
// reduction's readers are past a later barrier before it is written again.
__device__ __forceinline__ void block_max_or_r1(int& e, int& bad, int* red) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  e = __reduce_max_sync(0xffffffffu, e);
  bad = __reduce_or_sync(0xffffffffu, bad);
  if (lane == 0) {
    red[warp] = e;
    red[kR1Warps + warp] = bad;
  }
  __syncthreads();
  e = kNoExpR1;
  bad = 0;
  for (int w = 0; w < kR1Warps; ++w) {
    e = max(e, red[w]);
    bad |= red[kR1Warps + w];
  }
}

// Cluster of kR1Cluster CTAs per direction (blocks [0, C): L, [C, 2C): F).
// Per mode each CTA forms part of the next vector from its share of the core
// (L: a share of the rows (a, i), summed into partial columns; F: a share of
// the rows a, each a full dot product), a cluster barrier makes the parts
// visible, and every CTA gathers the whole vector from its peers (in rank
// order: the same sum everywhere), so all CTAs take the same rescaling
// decision.  The parts alternate between two buffers by mode parity, so one
// barrier per mode suffices: a peer reads parts of mode k before it reaches
// the barrier of mode k + 1, and they are overwritten in mode k + 2.
template <typename T>
__global__ void __launch_bounds__(kR1Threads) r1_sweep_kernel(const __grid_constant__ AdjR1Params p) {
  extern __shared__ __align__(16) unsigned char r1_smem[];
  T* cur = reinterpret_cast<T*>(r1_smem);  // [kR1MaxRank] the current vector
  T* nxt = cur + kR1MaxRank;                // [kR1MaxRank] the next vector
  T* parts = nxt + kR1MaxRank;              // [2][kR1MaxRank] this CTA's part, by mode parity
  T* tmp = parts + 2 * kR1MaxRank;          // [16 / sizeof(T)][kR1Threads] per-thread partial columns
  __shared__ int red[2][2 * kR1Warps];  // block reductions, alternating by mode parity
  cg::cluster_group cluster = cg::this_cluster();
  const int C = static_cast<int>(cluster.num_blocks());
  const int crank = static_cast<int>(cluster.block_rank());
  const bool left = blockIdx.x < static_cast<unsigned>(C);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = p.n;
  int bad = 0;
  T* vecs = static_cast<T*>(left ? p.lvec : p.fvec);
  int64_t* scl = left ? p.llog : p.flog;
  int64_t lg = 0;
  if (tid == 0) cur[0] = T(1);
  if (crank == 0 && tid == 0) {
    vecs[static_cast<int64_t>(left ? 0 : n) * p.vstride] = T(1);
    scl[left ? 0 : n] = 0;
  }
  __syncthreads();
  for (int step = 0; step < n; ++step) {
    const int k = left ? step : n - 1 - step;
    const AdjStep& st = p.step[k];
    const T* gx = static_cast<const T*>(st.gx);
    const T* y = static_cast<const T*>(st.gy);
    const int R = st.rx, I = st.I, R2 = st.rx2;
    T* part = parts + (step & 1) * kR1MaxRank;
    int nout;  // length of the next vector
    if (left) {
      // L_{k+1}[a'] = sum over rows r = (a, i) of L_k[a] y_k[i] Gx_k[r][a'], rows
      // [r0, r1) here; 16-byte loads along a row when it allows
      nout = R2;
      const int rows = R * I, r0 = static_cast<int>(static_cast<int64_t>(rows) * crank / C),
                r1 = static_cast<int>(static_cast<int64_t>(rows) * (crank + 1) / C);
      constexpr int VW = 16 / static_cast<int>(sizeof(T));
      const bool vec = R2 % VW == 0 && (reinterpret_cast<uintptr_t>(gx) & 15) == 0;
      const int w = vec ? VW : 1;
      for (int c0 = 0; c0 < R2; c0 += kR1Threads * w) {
        if (c0 > 0) __syncthreads();  // the previous pass has read tmp
        const int nc = min(kR1Threads, (R2 - c0 + w - 1) / w);  // column units of this pass
        const int G = max(1, kR1Threads / nc);                   // row groups
        const int col = tid % nc, grp = tid / nc;
        T acc[VW];
#pragma unroll
        for (int q = 0; q < VW; ++q) acc[q] = T(0);
        if (grp < G) {
          int a = (r0 + grp) / I, i = (r0 + grp) - ((r0 + grp) / I) * I;
          const int da = G / I, di = G - da * I;
#pragma unroll 4
          for (int r = r0 + grp; r < r1; r += G) {
            const T wgt = cur[a] * ldg(y + i);
            const T* src = gx + static_cast<int64_t>(r) * R2 + c0 + col * w;
            if (vec) {
              T v[VW];
              ld_vec<T, VW>(v, src);
#pragma unroll
              for (int q = 0; q < VW; ++q) acc[q] = fma(wgt, v[q], acc[q]);
            } else {
              acc[0] = fma(wgt, ldg(src), acc[0]);
            }
            a += da;
            i += di;
            if (i >= I) {
              i -= I;
              ++a;
            }
          }
        }
        for (int q = 0; q < w; ++q) tmp[q * kR1Threads + tid] = acc[q];
        __syncthreads();
        for (int u = tid; u < nc * w; u += kR1Threads) {  // column unit u / w, lane u % w
          const int cu = u / w, q = u - cu * w;
          if (c0 + cu * w + q < R2) {
            T sum = T(0);
            for (int g = 0; g < G; ++g) sum += tmp[q * kR1Threads + g * nc + cu];
            part[c0 + cu * w + q] = sum;
          }
        }
      }
    } else {
      // F_k[a] = sum_{i,a'} Gx_k[a][i][a'] y_k[i] F_{k+1}[a'] for rows a in [a0, a1)
      nout = R;
      const int a0 = R * crank / C, a1 = R * (crank + 1) / C;
      for (int a = a0 + warp; a < a1; a += kR1Warps) {
        const T* row = gx + static_cast<int64_t>(a) * I * R2;
        T acc = T(0);
#pragma unroll 4
        for (int i = 0; i < I; ++i) {
          const T yi = ldg(y + i);
          for (int c = lane; c < R2; c += 32) acc = fma(ldg(row + static_cast<int64_t>(i) * R2 + c) * yi, cur[c], acc);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) part[a] = acc;
      }
    }
    cluster.sync();  // every CTA's part of this mode is visible (and this CTA's threads are in step)
    // gather the whole vector (each thread keeps its own entries in nxt) and
    // its largest binary exponent
    int e = kNoExpR1, lbad = 0;
    if (left) {
      for (int c = tid; c < nout; c += kR1Threads) {
        T sum = T(0);
        for (int r = 0; r < C; ++r) sum += *cluster.map_shared_rank(part + c, r);
        nxt[c] = sum;
        if (!isfinite(sum)) lbad = 1;
        else if (sum != T(0)) e = max(e, exp2_bits(sum));
      }
    } else {
      for (int a = tid; a < nout; a += kR1Threads) {
        // rows [R r / C, R (r + 1) / C) belong to rank r
        int o = min(C - 1, static_cast<int>((static_cast<int64_t>(a) * C + C - 1) / R));
        while (o > 0 && a < R * o / C) --o;
        while (o + 1 < C && a >= R * (o + 1) / C) ++o;
        const T v = *cluster.map_shared_rank(part + a, o);
        nxt[a] = v;
        if (!isfinite(v)) lbad = 1;
        else if (v != T(0)) e = max(e, exp2_bits(v));
      }
    }
    block_max_or_r1(e, lbad, red[step & 1]);
    if (lbad) bad = 1;
    const int sh = (e != kNoExpR1 && (e > p.renorm_bits || e < -p.renorm_bits)) ? e : 0;
    lg += sh;
    const int64_t vk = left ? k + 1 : k;
    for (int a = tid; a < nout; a += kR1Threads) {  // the same entries this thread gathered
      const T v = sh ? mul_pow2<T>(nxt[a], -sh) : nxt[a];
      cur[a] = v;
      if (crank == 0) vecs[vk * p.vstride + a] = v;
    }
    if (crank == 0 && tid == 0) scl[vk] = lg;
    __syncthreads();  // cur is complete before the next mode reads it
  }
  if (bad && tid == 0 && crank == 0) set_status(p.status, TT_STATUS_NONFINITE);
  cluster.sync();  // peers' parts stay readable until everyone is done
}

// One block per (i, k): dGx_k[:, i, :] and dGy_k[0][i][0].
template <typename T>
__global__ void __launch_bounds__(256) r1_grad_kernel(const __grid_constant__ AdjR1Params p) {
  __shared__ double red[8];
  const int k = blockIdx.y, i = blockIdx.x;
  const AdjStep& st = p.step[k];
  if (i >= st.I) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int R = st.rx, I = st.I, R2 = st.rx2;
  const T* lv = static_cast<const T*>(p.lvec) + static_cast<int64_t>(k) * p.vstride;
  const T* fv = static_cast<const T*>(p.fvec) + static_cast<int64_t>(k + 1) * p.vstride;
  const T* gx = static_cast<const T*>(st.gx);
  T* dgx = static_cast<T*>(st.dgx);
  const double gbar = p.cot != nullptr ? *p.cot : 1.0;
  int64_t esum = p.llog[k] + p.flog[k + 1];
  esum = esum < -4000 ? -4000 : (esum > 4000 ? 4000 : esum);
  const double fac = ldexp(gbar, static_cast<int>(esum));
  int ge = 0;
  const float fm = static_cast<float>(frexp(gbar, &ge));
  const int fe = ge + static_cast<int>(esum);
  const T yi = static_cast<const T*>(st.gy)[i];
  int sbits = 0;
  double dy = 0.0;
  for (int a = warp; a < R; a += 8) {
    const T la = lv[a];
    const T* grow = gx + (static_cast<int64_t>(a) * I + i) * R2;
    T* drow = dgx + (static_cast<int64_t>(a) * I + i) * R2;
    T s = T(0);
    for (int c = lane; c < R2; c += 32) {
      const T f = fv[c];
      s = fma(ldg(grow + c), f, s);
      T o;
      const T t = la * yi * f;
      if constexpr (sizeof(T) == 4) o = scale_pow2_sat<float>(t * fm, fe);
      else o = t * fac;
      if (!isfinite(o)) sbits |= isfinite(t) ? TT_STATUS_OVERFLOW : TT_STATUS_NONFINITE;
      drow[c] = o;
    }
    dy = fma(static_cast<double>(la), static_cast<double>(s), dy);
  }
  dy = warp_sum(dy);
  if (lane == 0) red[warp] = dy;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    // dGy_k[0][i][0] = g 2^esum s, rounded once to T
    const double v = ldexp(s * gbar, static_cast<int>(esum));
    const T o = static_cast<T>(v);
    if (!isfinite(o)) sbits |= isfinite(v) ? TT_STATUS_OVERFLOW : TT_STATUS_NONFINITE;
    static_cast<T*>(st.dgy)[i] = o;
  }
  if (sbits) set_status(p.status, sbits);
}

}  // namespace

cudaError_t launch_adjoint_r1(const AdjR1Params& p, int dtype, cudaStream_t s) {
  int imax = 1;
  for (int k = 0; k < p.n; ++k) imax = std::max(imax, p.step[k].I);
  const size_t esz = dtype == TT_F64 ? 8 : 4;
  const size_t smem = (4 * static_cast<size_t>(kR1MaxRank) + (16 / esz) * kR1Threads) * esz;
  const void* sweep = dtype == TT_F64 ? reinterpret_cast<const void*>(r1_sweep_kernel<double>)
                                      : reinterpret_cast<const void*>(r1_sweep_kernel<float>);
  cudaError_t err = cudaFuncSetAttribute(sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * kR1Cluster);
  cfg.blockDim = dim3(kR1Threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kR1Cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch(2);
  if (dtype == TT_F64) {
    err = cudaLaunchKernelEx(&cfg, r1_sweep_kernel<double>, p);
    if (err != cudaSuccess) return err;
    r1_grad_kernel<double><<<dim3(imax, p.n), 256, 0, s>>>(p);
  } else {
    err = cudaLaunchKernelEx(&cfg, r1_sweep_kernel<float>, p);
    if (err != cudaSuccess) return err;
    r1_grad_kernel<float><<<dim3(imax, p.n), 256, 0, s>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace ttc
