// Adjoint of the environment sweep: gradients of a contraction with respect
// to every core of both operands.
//
// For z = <L_seed | sweep over modes k0..k1-1 | F_seed> (a full contraction
// has both seeds [1]; a chain-layout partial contraction seeds one side with
// the cotangent of its K), z is linear in each core and, with L_k the left and
// F_{k+1} the right environments,
//   dGx_k[:, i, :] = L_k  Gy_k[:, i, :] F_{k+1}^T,
//   dGy_k[:, i, :] = L_k^T Gx_k[:, i, :] F_{k+1}.
// Per slice i this is evaluated as U = L Gy_i, dGx_i = U F^T, W = Gx_i F,
// dGy_i = L^T W, and the next right environment gets W Gy_i^T.
//
// Memory: the left environments are not all kept.  A forward sweep stores L
// every c modes (checkpoints, c = ceil(sqrt(n)) unless the caller picks one)
// in the workspace; the backward walk then goes segment by segment from the
// right, recomputing the c left environments of the segment from its
// checkpoint before walking it backwards.  Workspace is (ceil(n/c) + c)
// environments instead of n, for one extra forward sweep (c = 1 keeps all).
//
// Work split: like the forward sweep, the slices i of every mode are spread
// over the CTAs of one cluster and the environment sums are reduced through
// distributed shared memory.
#include <cooperative_groups.h>

#include "copy_jobs.cuh"
#include "ttc_device.cuh"
#include "ttc_internal.h"

namespace cg = cooperative_groups;

namespace ttc {

namespace {

constexpr int kNoExpA = -(1 << 30);

template <typename T, int RM>
struct AdjCfg {
  static constexpr int NT = 256;
  static constexpr int NW = NT / 32;
  static constexpr int TM = RM / 16;
  static constexpr int V = 16 / sizeof(T);
  static constexpr int LD = RM + V;
  static constexpr int TILE = RM * LD;
  // Ls, LT, F, FT, GyS, GyT, Gx, X1, W, Rs (half)
  static constexpr int NBUF_FULL = 9;
  static constexpr size_t SMEM = (NBUF_FULL * TILE + (RM / 2) * LD) * sizeof(T) + 128 * sizeof(int);
};

// acc[a][b] += sum_{k<K} A[k][m0+a] * B[k][n0+b]
template <typename T, int TM, int LD>
__device__ __forceinline__ void op_acc(T (&acc)[TM][TM], const T* __restrict__ A, const T* __restrict__ B, int K, int m0,
                                       int n0) {
#pragma unroll 16
  for (int k = 0; k < K; ++k) {
    T av[TM], bv[TM];
    ld_vec<T, TM>(av, A + k * LD + m0);
    ld_vec<T, TM>(bv, B + k * LD + n0);
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TM; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
  }
}

template <typename T, int TM>
__device__ __forceinline__ void zero(T (&acc)[TM][TM]) {
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TM; ++b) acc[a][b] = T(0);
}

// Slice i of a core into dst (row stride LD), asynchronously.
//   tr == 0: dst[r][c] = core[r][i][c]   (core [rows][I][cols])
//   tr == 1: dst[r][c] = core[c][i][r]   (core [cols][I][rows])
template <typename T, int LD, int NT>
__device__ __forceinline__ void slice_async(T* dst, const T* core, int i, int I, int rows, int cols, int tr) {
  constexpr int V = 16 / static_cast<int>(sizeof(T));
  if (!tr) {
    // rows of `cols` contiguous elements, I * cols apart: 16-byte copies when aligned
    const T* base = core + static_cast<int64_t>(i) * cols;
    const int64_t rs = static_cast<int64_t>(I) * cols;
    if (cols % V == 0 && rs % V == 0 && (reinterpret_cast<uintptr_t>(base) & 15) == 0) {
      const int cv = cols / V, tot = rows * cv;
      for (int e = threadIdx.x; e < tot; e += NT) {
        const int r = udiv16(e, cv), c = (e - r * cv) * V;
        cp_async16(dst + r * LD + c, base + r * rs + c);
      }
    } else {
      for (int e = threadIdx.x; e < rows * cols; e += NT) {
        const int r = udiv16(e, cols), c = e - r * cols;
        cp_async_elem(dst + r * LD + c, base + r * rs + c);
      }
    }
  } else {
    for (int e = threadIdx.x; e < rows * cols; e += NT) {
      const int c = udiv16(e, rows), r = e - c * rows;
      cp_async_elem(dst + r * LD + c, core + (static_cast<int64_t>(c) * I + i) * rows + r);
    }
  }
}

// Binary exponent of s folded into lexp (read from its bits); a non-finite s
// sets lbad.
template <typename T>
__device__ __forceinline__ void track_e(int& lexp, int& lbad, T s) {
  if (!isfinite(s)) lbad = 1;
  else if (s != T(0)) lexp = max(lexp, exp2_bits(s));
}

// Sum the thread tiles acc (tile at (u0, v0) of an nu x nv matrix) over the
// cluster; every CTA writes the sum into Dn[u][v] and Dt[v][u], rescaled by an
// exact power of two when its largest exponent leaves [-s, s].  Returns the
// exponent folded out (0 when none).  Ps / Rs: scratch tiles.
template <typename T, int RM>
__device__ int reduce_env(T (&acc)[RM / 16][RM / 16], int u0, int v0, int nu, int nv, T* Ps, T* Rs, T* Dn, T* Dt,
                          int* ired, int C, int crank, int renorm_bits, int& bad) {
  using Cfg = AdjCfg<T, RM>;
  constexpr int TM = Cfg::TM, LD = Cfg::LD, NT = Cfg::NT, NW = Cfg::NW;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __syncthreads();  // all readers of Dn / Dt / Ps are done
  if (C == 1) {
    int lexp = kNoExpA, lbad = 0;
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TM; ++b)
        if (u0 + a < nu && v0 + b < nv) track_e(lexp, lbad, acc[a][b]);
    lexp = __reduce_max_sync(0xffffffffu, lexp);
    lbad = __reduce_or_sync(0xffffffffu, lbad);
    if (lane == 0) {
      ired[warp] = lexp;
      ired[16 + warp] = lbad;
    }
    __syncthreads();
    int g = kNoExpA, gb = 0;
    for (int w = 0; w < NW; ++w) {
      g = max(g, ired[w]);
      gb |= ired[16 + w];
    }
    if (gb) bad = 1;
    const int sh = (g != kNoExpA && (g > renorm_bits || g < -renorm_bits)) ? g : 0;
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TM; ++b) {
        const T v = sh ? mul_pow2<T>(acc[a][b], -sh) : acc[a][b];
        Dn[(u0 + a) * LD + v0 + b] = v;
        Dt[(v0 + b) * LD + u0 + a] = v;
      }
    __syncthreads();
    return sh;
  }
  // Two cluster barriers per reduction: (1) every partial is in its owner's
  // reach, (2) every reduced chunk is.  The exponent is then taken by each CTA
  // over the whole matrix it has pulled (the same data everywhere, so the same
  // shift).  No third barrier is needed before Ps / Rs are written again: a
  // CTA writes Ps only after barrier (2), which every peer passes after its
  // last read of Ps, and writes Rs only after barrier (1) of the next
  // reduction, which every peer passes after its last read of Rs.
  cg::cluster_group cluster = cg::this_cluster();
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TM; ++b) Ps[(u0 + a) * LD + v0 + b] = acc[a][b];
  cluster.sync();
  const int chunk = (nu + C - 1) / C;
  const int ub = min(nu, crank * chunk), ue = min(nu, ub + chunk);
  for (int idx = tid; idx < (ue - ub) * nv; idx += NT) {
    const int q = udiv16(idx, nv), u = ub + q, v = idx - q * nv;
    T part[16];
#pragma unroll
    for (int r = 0; r < 16; ++r)
      if (r < C) part[r] = *cluster.map_shared_rank(Ps + u * LD + v, r);
    T s = T(0);
#pragma unroll
    for (int r = 0; r < 16; ++r)
      if (r < C) s += part[r];
    Rs[(u - ub) * LD + v] = s;
  }
  cluster.sync();
  // every CTA reads the reduced rows from their owners (16-byte remote loads,
  // four per thread in flight) into Dn / Dt
  int lexp = kNoExpA, lbad = 0;
  constexpr int V = 16 / static_cast<int>(sizeof(T));
  if (nv % V == 0) {
    const int nvv = nv / V, tot = nu * nvv;
    for (int b0 = tid; b0 < tot; b0 += 4 * NT) {
      uint4 q[4];
      int uu[4], vv[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int idx = b0 + j * NT;
        uu[j] = -1;
        if (idx < tot) {
          const int u = udiv16(idx, nvv), v = (idx - u * nvv) * V;
          const int owner = udiv16(u, chunk);
          q[j] = *reinterpret_cast<const uint4*>(cluster.map_shared_rank(Rs + (u - owner * chunk) * LD + v, owner));
          uu[j] = u;
          vv[j] = v;
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (uu[j] >= 0) {
          T e[V];
          memcpy(e, &q[j], sizeof(e));
#pragma unroll
          for (int t = 0; t < V; ++t) {
            track_e(lexp, lbad, e[t]);
            Dn[uu[j] * LD + vv[j] + t] = e[t];
            Dt[(vv[j] + t) * LD + uu[j]] = e[t];
          }
        }
    }
  } else {
    for (int idx = tid; idx < nu * nv; idx += NT) {
      const int u = udiv16(idx, nv), v = idx - u * nv;
      const int owner = udiv16(u, chunk);
      const T e = *cluster.map_shared_rank(Rs + (u - owner * chunk) * LD + v, owner);
      track_e(lexp, lbad, e);
      Dn[u * LD + v] = e;
      Dt[v * LD + u] = e;
    }
  }
  lexp = __reduce_max_sync(0xffffffffu, lexp);
  lbad = __reduce_or_sync(0xffffffffu, lbad);
  if (lane == 0) {
    ired[warp] = lexp;
    ired[16 + warp] = lbad;
  }
  __syncthreads();
  int g = kNoExpA, gb = 0;
  for (int w = 0; w < NW; ++w) {
    g = max(g, ired[w]);
    gb |= ired[16 + w];
  }
  if (gb) bad = 1;
  const int sh = (g != kNoExpA && (g > renorm_bits || g < -renorm_bits)) ? g : 0;
  if (sh) {  // rare: rescale both copies in place
    for (int idx = tid; idx < nu * nv; idx += NT) {
      const int u = udiv16(idx, nv), v = idx - u * nv;
      Dn[u * LD + v] = mul_pow2<T>(Dn[u * LD + v], -sh);
      Dt[v * LD + u] = mul_pow2<T>(Dt[v * LD + u], -sh);
    }
  }
  __syncthreads();
  return sh;
}

// Load an environment (row-major [nu][nv] in global memory; the sum of
// `parts` consecutive such matrices, added in order) into Dn / Dt.
template <typename T, int LD, int NT>
__device__ void load_env(const T* src, int nu, int nv, T* Dn, T* Dt, int parts = 1) {
  for (int idx = threadIdx.x; idx < nu * nv; idx += NT) {
    const int u = idx / nv, v = idx - u * nv;
    T e = src[idx];
    for (int g = 1; g < parts; ++g) e += src[static_cast<int64_t>(g) * nu * nv + idx];
    Dn[u * LD + v] = e;
    Dt[v * LD + u] = e;
  }
}

template <typename T, int LD, int NT>
__device__ void store_env(T* dst, int nu, int nv, const T* Dn) {
  for (int idx = threadIdx.x; idx < nu * nv; idx += NT) {
    const int u = idx / nv, v = idx - u * nv;
    dst[idx] = Dn[u * LD + v];
  }
}

}  // namespace

// A gradient entry t times the scale fac = fm * 2^fe: in float64 for double
// cores, in float (mantissa product, then an exact power of two, saturated)
// for float cores.  Overflow of a finite value sets TT_STATUS_OVERFLOW, a
// non-finite t TT_STATUS_NONFINITE.
template <typename T>
__device__ __forceinline__ T grad_out(T t, double fac, float fm, int fe, int& sbits) {
  T o;
  if constexpr (sizeof(T) == 4) {
    o = scale_pow2_sat<float>(t * fm, fe);
  } else {
    o = t * fac;
  }
  if (!isfinite(o)) sbits |= isfinite(t) ? TT_STATUS_OVERFLOW : TT_STATUS_NONFINITE;
  return o;
}

template <typename T, int RM>
__global__ void __launch_bounds__(256, 1) adjoint_kernel(const __grid_constant__ AdjointParams p) {
  using Cfg = AdjCfg<T, RM>;
  constexpr int NT = Cfg::NT, TM = Cfg::TM, LD = Cfg::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ls = reinterpret_cast<T*>(smem_raw);  // L[a][b]
  T* LT = Ls + Cfg::TILE;                  // L[b][a]
  T* Fs = LT + Cfg::TILE;                  // F[a'][b']
  T* FT = Fs + Cfg::TILE;                  // F[b'][a']
  T* GyS = FT + Cfg::TILE;                 // Gy_i[b][b']
  T* GyT = GyS + Cfg::TILE;                // Gy_i[b'][b]
  T* Gx = GyT + Cfg::TILE;                 // Gx_i[a][a'] (forward) or [a'][a] (backward)
  T* X1 = Gx + Cfg::TILE;                  // U^T, W^T, partial sums
  T* Wn = X1 + Cfg::TILE;                  // W[a][b'] / T[a][b']
  T* Rs = Wn + Cfg::TILE;                  // reduced rows (RM/2 x LD)
  int* ired = reinterpret_cast<int*>(Rs + (RM / 2) * LD);

  const bool cl = p.cluster > 1;
  int C = 1, crank = 0;
  if (cl) {
    cg::cluster_group cluster = cg::this_cluster();
    C = static_cast<int>(cluster.num_blocks());
    crank = static_cast<int>(cluster.block_rank());
  }
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  const int u0 = ty * TM, v0 = tx * TM;
  const int n = p.n;
  const int c = p.stride;
  int bad = 0, sbits = 0;
  T* ckpt = static_cast<T*>(p.ckpt);
  T* seg = static_cast<T*>(p.seg);
  const int64_t env_elems = p.env_elems;

  // One forward step L_{k+1} = sum_i Gx_i^T (L_k Gy_i); L in Ls/LT, result back in Ls/LT.
  auto forward = [&](int k, int64_t& lg) {
    const AdjStep& st = p.step[k];
    T pacc[TM][TM];
    zero<T, TM>(pacc);
    for (int i = crank; i < st.I; i += C) {
      __syncthreads();
      slice_async<T, LD, NT>(GyS, static_cast<const T*>(st.gy), i, st.I, st.ry, st.ry2, 0);
      slice_async<T, LD, NT>(Gx, static_cast<const T*>(st.gx), i, st.I, st.rx, st.rx2, 0);
      cp_async_commit();
      cp_async_wait<0>();
      __syncthreads();
      T t[TM][TM];
      zero<T, TM>(t);
      if (u0 < st.rx && v0 < st.ry2) op_acc<T, TM, LD>(t, LT, GyS, st.ry, u0, v0);  // T[a][b'] = L Gy_i
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TM; ++b) Wn[(u0 + a) * LD + v0 + b] = t[a][b];
      __syncthreads();
      if (u0 < st.rx2 && v0 < st.ry2) op_acc<T, TM, LD>(pacc, Gx, Wn, st.rx, u0, v0);  // P[a'][b'] += Gx_i^T T
    }
    lg += reduce_env<T, RM>(pacc, u0, v0, st.rx2, st.ry2, X1, Rs, Ls, LT, ired, C, crank, p.renorm_bits, bad);
  };

  // ---- phase 1: forward sweep storing checkpoints L_{jc} ----
  int64_t lg = 0;
  {
    const int rx0 = p.step[0].rx, ry0 = p.step[0].ry;
    if (p.l_seed != nullptr) {
      load_env<T, LD, NT>(static_cast<const T*>(p.l_seed), rx0, ry0, Ls, LT, p.seed_parts);
      if (p.l_seed_log2 != nullptr) lg = *p.l_seed_log2;
    } else if (tid == 0) {
      Ls[0] = T(1);
      LT[0] = T(1);
    }
    __syncthreads();
  }
  const int nseg = (n + c - 1) / c;
  const int last_ck = (nseg - 1) * c;
  // (skipped when the forward sweep of the contraction already stored them)
  for (int k = 0; k <= last_ck && !p.ckpt_given; ++k) {
    if (k % c == 0 && crank == 0) {
      store_env<T, LD, NT>(ckpt + (k / c) * env_elems, p.step[k].rx, p.step[k].ry, Ls);
      if (tid == 0) p.ckpt_log2[k / c] = lg;
    }
    if (k < last_ck) forward(k, lg);
  }
  __threadfence();
  if (cl) cg::this_cluster().sync();
  else __syncthreads();

  // ---- phase 2: backward walk, segment by segment from the right ----
  int64_t fl = 0;
  {
    const int rxn = p.step[n - 1].rx2, ryn = p.step[n - 1].ry2;
    if (p.f_seed != nullptr) {
      load_env<T, LD, NT>(static_cast<const T*>(p.f_seed), rxn, ryn, Fs, FT, p.seed_parts);
      if (p.f_seed_log2 != nullptr) fl = *p.f_seed_log2;
    } else if (tid == 0) {
      Fs[0] = T(1);
      FT[0] = T(1);
    }
  }
  const double gbar = p.cot != nullptr ? *p.cot : 1.0;
  for (int g = nseg - 1; g >= 0; --g) {
    const int k0 = g * c, k1 = min(n, k0 + c);
    // recompute L_{k0..k1-1} from the checkpoint into the segment buffer
    __syncthreads();
    load_env<T, LD, NT>(ckpt + g * env_elems, p.step[k0].rx, p.step[k0].ry, Ls, LT);
    int64_t l = p.ckpt_log2[g];
    __syncthreads();
    if (crank == 0) {
      store_env<T, LD, NT>(seg, p.step[k0].rx, p.step[k0].ry, Ls);
      if (tid == 0) p.seg_log2[0] = l;
    }
    for (int k = k0; k + 1 < k1; ++k) {
      forward(k, l);
      if (crank == 0) {
        store_env<T, LD, NT>(seg + (k + 1 - k0) * env_elems, p.step[k + 1].rx, p.step[k + 1].ry, Ls);
        if (tid == 0) p.seg_log2[k + 1 - k0] = l;
      }
    }
    __threadfence();
    if (cl) cg::this_cluster().sync();
    else __syncthreads();
    // walk the segment backwards
    for (int k = k1 - 1; k >= k0; --k) {
      const AdjStep& st = p.step[k];
      __syncthreads();
      load_env<T, LD, NT>(seg + (k - k0) * env_elems, st.rx, st.ry, Ls, LT);
      const int64_t lk = p.seg_log2[k - k0];
      // gradient scale: gbar * 2^(lk + fl)
      int64_t esum = lk + fl;
      esum = esum < -4000 ? -4000 : (esum > 4000 ? 4000 : esum);
      const double fac = ldexp(gbar, static_cast<int>(esum));
      // float gradients are scaled in float: fac = fm * 2^fe with fm the
      // float-rounded mantissa of gbar (the float64 pipe is a small fraction
      // of the float32 one here)
      int ge = 0;
      const float fm = static_cast<float>(frexp(gbar, &ge));
      const int fe = ge + static_cast<int>(esum);
      T facc[TM][TM];
      zero<T, TM>(facc);
      T* dgx = static_cast<T*>(st.dgx);
      T* dgy = static_cast<T*>(st.dgy);
      for (int i = crank; i < st.I; i += C) {
        __syncthreads();
        slice_async<T, LD, NT>(GyS, static_cast<const T*>(st.gy), i, st.I, st.ry, st.ry2, 0);   // [b][b']
        slice_async<T, LD, NT>(GyT, static_cast<const T*>(st.gy), i, st.I, st.ry2, st.ry, 1);   // [b'][b]
        slice_async<T, LD, NT>(Gx, static_cast<const T*>(st.gx), i, st.I, st.rx2, st.rx, 1);    // [a'][a]
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
        T t[TM][TM];
        // U[a][b'] = L Gy_i  -> X1 as U^T[b'][a]
        zero<T, TM>(t);
        if (u0 < st.rx && v0 < st.ry2) op_acc<T, TM, LD>(t, LT, GyS, st.ry, u0, v0);
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
          for (int b = 0; b < TM; ++b) X1[(v0 + b) * LD + u0 + a] = t[a][b];
        __syncthreads();
        // dGx[a][a'] = U F^T : A = U^T[b'][a], B = F^T[b'][a']
        zero<T, TM>(t);
        if (u0 < st.rx && v0 < st.rx2) op_acc<T, TM, LD>(t, X1, FT, st.ry2, u0, v0);
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
          for (int b = 0; b < TM; ++b)
            if (u0 + a < st.rx && v0 + b < st.rx2) {
              dgx[(static_cast<int64_t>(u0 + a) * st.I + i) * st.rx2 + v0 + b] = grad_out<T>(t[a][b], fac, fm, fe, sbits);
            }
        // W[a][b'] = Gx_i F : A = Gx^T[a'][a], B = F[a'][b']
        zero<T, TM>(t);
        if (u0 < st.rx && v0 < st.ry2) op_acc<T, TM, LD>(t, Gx, Fs, st.rx2, u0, v0);
        __syncthreads();  // X1 (U^T) is read by everyone before it becomes W^T
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
          for (int b = 0; b < TM; ++b) {
            Wn[(u0 + a) * LD + v0 + b] = t[a][b];
            X1[(v0 + b) * LD + u0 + a] = t[a][b];
          }
        __syncthreads();
        // dGy[b][b'] = L^T W : A = L[a][b], B = W[a][b']
        zero<T, TM>(t);
        if (u0 < st.ry && v0 < st.ry2) op_acc<T, TM, LD>(t, Ls, Wn, st.rx, u0, v0);
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
          for (int b = 0; b < TM; ++b)
            if (u0 + a < st.ry && v0 + b < st.ry2) {
              dgy[(static_cast<int64_t>(u0 + a) * st.I + i) * st.ry2 + v0 + b] = grad_out<T>(t[a][b], fac, fm, fe, sbits);
            }
        // F_k[a][b] += W Gy_i^T : A = W^T[b'][a], B = Gy^T[b'][b]
        if (u0 < st.rx && v0 < st.ry) op_acc<T, TM, LD>(facc, X1, GyT, st.ry2, u0, v0);
      }
      if (k > 0 || p.need_f0) fl += reduce_env<T, RM>(facc, u0, v0, st.rx, st.ry, X1, Rs, Fs, FT, ired, C, crank,
                                                      p.renorm_bits, bad);
    }
  }
  if (sbits) set_status(p.status, sbits);
  if (bad && tid == 0 && crank == 0) set_status(p.status, TT_STATUS_NONFINITE);
  if (cl) cg::this_cluster().sync();
}

// ---------------------------------------------------------------------------
// Chain-layout partial contraction: cotangents of the emitted cores -> the
// gradient of the boundary core, the cotangent dK of the environment K, and
// the gradients of the free cores (plain or leg-swapped copies).
//   lead : C[u][i][y] = sum_a Gx[a][i][u] K[a][y]
//          dGx[a][i][u] = sum_y K[a][y] dC[u][i][y],  dK[a][y] = sum_{u,i} Gx[a][i][u] dC[u][i][y]
//   trail: C[u][i][y] = sum_b Gx[u][i][b] K[b][y]
//          dGx[u][i][b] = sum_y dC[u][i][y] K[b][y],  dK[b][y] = sum_{u,i} Gx[u][i][b] dC[u][i][y]
// Both gradients are small products, run as shared-memory tiled GEMMs with
// register tiles (ranks <= 128): blocks 0..I-1 compute the gradient slice i
// (K times the slice of dC), the next blocks compute dK in 32-row tiles (a
// sum over every (i, u) pair, its operand chunks double-buffered with
// cp.async), and the remaining blocks run the copies as jobs (copy_jobs.cuh).
// ---------------------------------------------------------------------------
namespace chainadj {
constexpr int LDS = 132;  // staged row stride (elements): up to 128 columns
constexpr int kRowsPerKBlock = 32;
template <typename T>
struct Ch {
  static constexpr int KCH = sizeof(T) == 4 ? 32 : 16;  // one (As, Bs) set: 2 * KCH * 132 * sizeof(T) = 33.8 KB
  static constexpr int SET = 2 * KCH * LDS;               // elements of one set
  static constexpr int NSET = 4;                          // dK operand ring: three sets in flight
  static constexpr size_t SMEM =
      NSET * SET * sizeof(T) > copy_smem_bytes<T>() ? NSET * SET * sizeof(T) : copy_smem_bytes<T>();
};

// acc[a][b] += sum_{k<K} As[k][m0+a] * Bs[k][n0+b]
template <typename T>
__device__ __forceinline__ void tile44(T (&acc)[4][4], const T* As, const T* Bs, int K, int m0, int n0) {
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    T av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = As[k * LDS + m0 + a];
#pragma unroll
    for (int b = 0; b < 4; ++b) bv[b] = Bs[k * LDS + n0 + b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
  }
}
// acc[a][b] += sum_{k<K} As[k][m0+a] * Bs[k][n0+b], a 4 x TW tile
template <typename T, int TW>
__device__ __forceinline__ void tile4w(T (&acc)[4][TW], const T* As, const T* Bs, int K, int m0, int n0) {
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    T av[4], bv[TW];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = As[k * LDS + m0 + a];
#pragma unroll
    for (int b = 0; b < TW; ++b) bv[b] = Bs[k * LDS + n0 + b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < TW; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
  }
}

// dK rows [r0, r0 + M), M <= 32, over slice group grp: partial sum
//   dK_grp[r][y] = sum_{i in group, u} A[(i,u)][r] dC[u][i][y]
//   lead : A = Gx[r][i][u] (u < rb);  trail: A = Gx[u][i][r] (u < ra)
// (the adjoint adds the dk_parts partials as it loads its seed).
// Thread tiles 4 x TW: with TW = 2 and ry <= 64, 8 x 32 tiles keep all 256
// threads busy; the (i, u-chunk) operand pairs stream through a ring of NSET
// cp.async sets, NSET - 1 of them in flight.
template <typename T, int TW>
__device__ void dk_block(const ChainAdjParams& p, int r0, int grp, T* sm) {
  constexpr int KCH = Ch<T>::KCH, SET = Ch<T>::SET, NSET = Ch<T>::NSET;
  const int tid = threadIdx.x;
  const T* gx = static_cast<const T*>(p.gx);
  const T* dc = static_cast<const T*>(p.dc);
  const int I = p.I, rb = p.rb, ry = p.ry;
  const int nk = p.lead ? p.ra : p.rb;
  const int M = min(kRowsPerKBlock, nk - r0), N = ry;
  const int nu = p.lead ? rb : p.ra;
  const int i_lo = grp * I / p.dk_parts, i_hi = (grp + 1) * I / p.dk_parts;  // this group's slices
  const int nuc = (nu + KCH - 1) / KCH, nit = (i_hi - i_lo) * nuc;
  const int ncb = (N + TW - 1) / TW;  // <= 32
  const bool on = tid < 8 * ncb;
  const int m0 = (tid / ncb) * 4, n0 = (tid % ncb) * TW;
  T acc[4][TW];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < TW; ++b) acc[a][b] = T(0);
  auto issue = [&](int it) {  // one commit group per call, empty past the end
    if (it >= nit) {
      cp_async_commit();
      return;
    }
    T* As = sm + (it % NSET) * SET;
    T* Bs = As + KCH * LDS;
    const int q = it / nuc, i = i_lo + q, u0 = (it - q * nuc) * KCH, kc = min(KCH, nu - u0);
    for (int e = tid; e < kc * M; e += blockDim.x) {
      if (p.lead) {
        const int r = udiv16(e, kc), uu = e - r * kc;  // contiguous in u
        cp_async_elem(As + uu * LDS + r, gx + (static_cast<int64_t>(r0 + r) * I + i) * rb + u0 + uu);
      } else {
        const int uu = udiv16(e, M), r = e - uu * M;  // contiguous in r
        cp_async_elem(As + uu * LDS + r, gx + (static_cast<int64_t>(u0 + uu) * I + i) * rb + r0 + r);
      }
    }
    for (int e = tid; e < kc * N; e += blockDim.x) {
      const int uu = udiv16(e, N), y = e - uu * N;  // contiguous in y
      cp_async_elem(Bs + uu * LDS + y, dc + (static_cast<int64_t>(u0 + uu) * I + i) * ry + y);
    }
    cp_async_commit();
  };
  for (int it = 0; it < NSET - 1; ++it) issue(it);
  for (int it = 0; it < nit; ++it) {
    // set (it + NSET - 1) % NSET was read in iteration it - 1, before its closing barrier
    issue(it + NSET - 1);
    cp_async_wait<NSET - 1>();  // the group of iteration it is complete
    __syncthreads();
    const int q = it / nuc, kc = min(KCH, nu - (it - q * nuc) * KCH);
    const T* As = sm + (it % NSET) * SET;
    if (on) tile4w<T, TW>(acc, As, As + KCH * LDS, kc, m0, n0);
    __syncthreads();
  }
  if (on) {
    T* dk = static_cast<T*>(p.dk) + static_cast<int64_t>(grp) * nk * ry;  // this group's partial sum
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < TW; ++b)
        if (m0 + a < M && n0 + b < N) dk[(r0 + m0 + a) * ry + n0 + b] = acc[a][b];
  }
}
}  // namespace chainadj

template <typename T>
__global__ void __launch_bounds__(256) chain_adjoint_kernel(const __grid_constant__ ChainAdjParams p) {
  using namespace chainadj;
  constexpr int KCH = Ch<T>::KCH;
  extern __shared__ __align__(16) unsigned char chain_smem[];
  T* const As = reinterpret_cast<T*>(chain_smem);
  T* const Bs = As + KCH * LDS;
  const int tid = threadIdx.x;
  const T* k = static_cast<const T*>(p.k);
  const T* dc = static_cast<const T*>(p.dc);
  const int ra = p.ra, rb = p.rb, I = p.I, ry = p.ry;
  const int nk = p.lead ? ra : rb;  // rows of K
  const int nkb = (nk + kRowsPerKBlock - 1) / kRowsPerKBlock * (p.dk != nullptr ? p.dk_parts : 1);
  int bits = 0;
  if (static_cast<int>(blockIdx.x) < I) {
    // ---- gradient slice i: out[m][n] = sum_y A[y][m] B[y][n] ----
    //   lead : m = a < ra, n = u < rb, A[y][a] = K[a][y],         B[y][u] = dC[u][i][y]
    //   trail: m = u < ra, n = b < rb, A[y][u] = dC[u][i][y],     B[y][b] = K[b][y]
    const int i = blockIdx.x;
    const int64_t klg = p.k_log2 != nullptr ? *p.k_log2 : 0;
    const int M = ra, N = rb;
    const int ncb = (N + 3) / 4, ntiles = ((M + 3) / 4) * ncb;
    T acc[4][4][4];
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[t][a][b] = T(0);
    for (int y0 = 0; y0 < ry; y0 += KCH) {
      const int kc = min(KCH, ry - y0);
      __syncthreads();
      // stage: consecutive threads read consecutive y of one row
      for (int e = tid; e < kc * M; e += blockDim.x) {
        const int r = e / kc, yy = e - r * kc;
        As[yy * LDS + r] = p.lead ? k[r * ry + y0 + yy] : dc[(static_cast<int64_t>(r) * I + i) * ry + y0 + yy];
      }
      for (int e = tid; e < kc * N; e += blockDim.x) {
        const int c = e / kc, yy = e - c * kc;
        Bs[yy * LDS + c] = p.lead ? dc[(static_cast<int64_t>(c) * I + i) * ry + y0 + yy] : k[c * ry + y0 + yy];
      }
      __syncthreads();
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int tt = tid + t * 256;
        if (tt < ntiles) tile44<T>(acc[t], As, Bs, kc, (tt / ncb) * 4, (tt % ncb) * 4);
      }
    }
    T* dg = static_cast<T*>(p.dgx);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int tt = tid + t * 256;
      if (tt >= ntiles) continue;
      const int m0 = (tt / ncb) * 4, n0 = (tt % ncb) * 4;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int m = m0 + a, n = n0 + b;
          if (m >= M || n >= N) continue;
          const T sv = acc[t][a][b];
          const T o = scale_pow2_sat<T>(sv, klg);
          if (!isfinite(o)) bits |= isfinite(sv) ? TT_STATUS_OVERFLOW : TT_STATUS_NONFINITE;
          dg[(static_cast<int64_t>(m) * I + i) * rb + n] = o;
        }
    }
  } else if (static_cast<int>(blockIdx.x) < I + nkb) {
    if (p.dk != nullptr) {
      const int nrb = (nk + kRowsPerKBlock - 1) / kRowsPerKBlock, b = blockIdx.x - I;
      const int grp = b / nrb, r0 = (b - grp * nrb) * kRowsPerKBlock;
      dk_block<T, 2>(p, r0, grp, As);  // ry <= 64 whenever there is a dK (checked at launch)
    }
  } else {
    // the copies, as jobs of at most kCopyJobBytes dealt over the copy blocks
    const int first = blockIdx.x - (I + nkb), step = gridDim.x - (I + nkb);
    auto job_of = [&](int jb) {
      int t = 0;
      CopyCut cut = copy_cut(p.copy[0].r0, p.copy[0].I, p.copy[0].r1, static_cast<int>(sizeof(T)));
      while (jb >= cut.n_i * cut.n_a && t + 1 < p.n_copies) {
        jb -= cut.n_i * cut.n_a;
        ++t;
        cut = copy_cut(p.copy[t].r0, p.copy[t].I, p.copy[t].r1, static_cast<int>(sizeof(T)));
      }
      return copy_job_at(p.copy[t], cut, jb);
    };
    T* const buf0 = reinterpret_cast<T*>(chain_smem);
    copy_jobs_block<T>(job_of, first, p.n_copy_jobs, step, buf0, buf0 + copy_buf_elems<T>());
  }
  if (bits) set_status(p.status, bits);
}

template <typename T, int RM>
static cudaError_t adjoint_launch_impl(const AdjointParams& p, cudaStream_t s) {
  const size_t smem = AdjCfg<T, RM>::SMEM;
  cudaError_t err =
      cudaFuncSetAttribute(adjoint_kernel<T, RM>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  err = cudaFuncSetAttribute(adjoint_kernel<T, RM>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (err != cudaSuccess) return err;
  int C = p.cluster;
  // the largest cluster (<= requested) that can be resident
  for (; C >= 2; C /= 2) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nact = 0;
    if (cudaOccupancyMaxActiveClusters(&nact, adjoint_kernel<T, RM>, &cfg) == cudaSuccess && nact >= 1) break;
    cudaGetLastError();
  }
  AdjointParams q = p;
  q.cluster = C < 1 ? 1 : C;
  count_launch();
  if (q.cluster == 1) {
    adjoint_kernel<T, RM><<<1, 256, smem, s>>>(q);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(q.cluster, 1, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = q.cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, adjoint_kernel<T, RM>, q);
}

cudaError_t launch_adjoint(const AdjointParams& p, int dtype, int rmax, cudaStream_t s) {
  if (dtype == TT_F64) {
    if (rmax <= 16) return adjoint_launch_impl<double, 16>(p, s);
    return adjoint_launch_impl<double, 32>(p, s);
  }
  if (rmax <= 32) return adjoint_launch_impl<float, 32>(p, s);
  return adjoint_launch_impl<float, 64>(p, s);
}

cudaError_t launch_chain_adjoint(const ChainAdjParams& p, int dtype, cudaStream_t s) {
  if (p.ra > 128 || p.rb > 128 || p.ry > 128) return cudaErrorInvalidValue;  // staged tiles hold 128 columns
  // a dK exists only for a non-empty contracted block, whose ranks are capped
  // at 64 (F32) / 32 (F64) by the adjoint: the dK tiles cover ry <= 64
  if (p.dk != nullptr && p.ry > 64) return cudaErrorInvalidValue;
  const int nk = p.lead ? p.ra : p.rb;
  const int eb = dtype == TT_F64 ? 8 : 4;
  ChainAdjParams q = p;
  q.n_copy_jobs = 0;
  for (int t = 0; t < p.n_copies; ++t) {
    if (p.copy[t].r1 > kCopyJobBytes / eb) return cudaErrorInvalidValue;  // a copy slice row must fit a job
    const CopyCut cut = copy_cut(p.copy[t].r0, p.copy[t].I, p.copy[t].r1, eb);
    q.n_copy_jobs += cut.n_i * cut.n_a;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int copy_blocks = std::min(q.n_copy_jobs, 2 * std::max(sms, 1));
  if (p.dk != nullptr && (p.dk_parts < 1 || p.dk_parts > std::min(p.I, kDkGroups))) return cudaErrorInvalidValue;
  const int nkb = (nk + chainadj::kRowsPerKBlock - 1) / chainadj::kRowsPerKBlock * (p.dk != nullptr ? p.dk_parts : 1);
  const int grid = p.I + nkb + copy_blocks;
  const size_t smem = dtype == TT_F64 ? chainadj::Ch<double>::SMEM : chainadj::Ch<float>::SMEM;
  cudaError_t err = dtype == TT_F64 ? cudaFuncSetAttribute(chain_adjoint_kernel<double>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                           static_cast<int>(smem))
                                    : cudaFuncSetAttribute(chain_adjoint_kernel<float>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                           static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  count_launch();
  if (dtype == TT_F64) chain_adjoint_kernel<double><<<grid, 256, smem, s>>>(q);
  else chain_adjoint_kernel<float><<<grid, 256, smem, s>>>(q);
  return cudaGetLastError();
}

}  // namespace ttc
