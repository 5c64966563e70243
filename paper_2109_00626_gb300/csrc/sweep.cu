// Environment sweep over contracted modes on one thread-block cluster, with
// the chain-layout emission of a partial contraction fused behind it.
//
// One contracted mode folds the core pair into the running environment
// (the generalisation of Algorithm 2 step 4 / Example 1's K = A_x^T A_y):
//   E'[u][v] = sum_i  (A_i^T E B_i)[u][v]
// with A_i, B_i the i-th slices of the two cores (see SweepStep).  The sum
// over the mode index i is split across the CTAs of one cluster: CTA c owns
// slices i = c, c + C, ...  Per slice a CTA computes T = E B_i and
// P += A_i^T T out of shared memory with a register-blocked outer-product
// loop.  Core slices stream in with cp.async, up to three loads ahead of the
// one being consumed (the loads do not depend on E, so the next mode's slices
// land while the cluster is still reducing the current one).  The cluster
// then adds the partial P's through distributed shared memory: CTA c sums its
// share of rows over all peers (fixed order: deterministic), and every CTA
// pulls the reduced rows back into its own copy of E'.
//
// Scaling: after each mode the largest binary exponent of E' is compared with
// +-s; outside that band E' is multiplied by an exact power of two and the
// exponent is accumulated in an int64, so long sweeps neither overflow nor
// underflow.
//
// The last step of a full contraction (both right ranks 1) is summed in
// float64: t_i[p] = sum_q E[p][q] B_i[q] in the storage type, then
// z = sum_{i,p} A_i[p] t_i[p] in double, cluster-reduced in double.
//
// Partial contractions (Algorithm 2 steps 5-6, chain layout) continue in the
// same launch: K = E is joined into the boundary core of X, slice by slice
// across the cluster, and the free cores are copied (leg-swapped where the
// chain walks X backwards), so one launch performs the whole operation.
#include <cooperative_groups.h>

#include "ttc_device.cuh"
#include "ttc_internal.h"

namespace cg = cooperative_groups;

namespace ttc {

constexpr int kNoExp = -(1 << 30);  // exponent marker of an all-zero environment

template <typename T, int RM>
struct SweepCfg {
  static constexpr int NT = 256;
  static constexpr int NW = NT / 32;
  static constexpr int TM = RM / 16;               // thread tile is TM x TM
  static constexpr int V = 16 / sizeof(T);         // elements per 16-byte vector
  static constexpr int LD = RM + V;                // row stride (elements), 16-byte padded
  static constexpr int TILE = RM * LD;
  static constexpr size_t TB = TILE * sizeof(T);
  static constexpr size_t kBudget = 232448 - 1024;
  // slice buffers: 4 (A and B double-buffered) when they fit, else 2, else 1
  // (then the reduction buffer shares the single slice buffer)
  static constexpr int NBUF = (7 * TB <= kBudget) ? 4 : ((5 * TB <= kBudget) ? 2 : 1);
  static constexpr int NFIX = NBUF == 1 ? 2 : 3;   // Es, Ts (+ Rs)
  static constexpr size_t SMEM = (NFIX + NBUF) * TB + 128 * sizeof(int);
};

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static __device__ __forceinline__ float get(const float4& v, int j) {
    return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
  }
  static __device__ __forceinline__ float4 add(float4 a, float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
  }
  static __device__ __forceinline__ float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
};
template <>
struct Vec16<double> {
  using type = double2;
  static __device__ __forceinline__ double get(const double2& v, int j) { return j == 0 ? v.x : v.y; }
  static __device__ __forceinline__ double2 add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
  static __device__ __forceinline__ double2 zero() { return make_double2(0.0, 0.0); }
};

// Asynchronously copy slice i of a core into dst[r][c] (row stride LD).
//   transposed == 0: core is [rows][I][cols], dst[r][c] = core[r][i][c]
//   transposed == 1: core is [cols][I][rows], dst[r][c] = core[c][i][r]
template <typename T, int LD, int NT>
__device__ __forceinline__ void load_slice_async(T* __restrict__ dst, const T* __restrict__ core, int i, int I,
                                                 int rows, int cols, int transposed) {
  if (!transposed) {
    constexpr int V = 16 / sizeof(T);
    if ((cols % V) == 0 && (reinterpret_cast<uintptr_t>(core) & 15) == 0) {
      const int cv = cols / V;
      for (int idx = threadIdx.x; idx < rows * cv; idx += NT) {
        const int r = idx / cv, c = (idx - r * cv) * V;
        cp_async16(dst + r * LD + c, core + (static_cast<int64_t>(r) * I + i) * cols + c);
      }
    } else {
      for (int idx = threadIdx.x; idx < rows * cols; idx += NT) {
        const int r = idx / cols, c = idx - r * cols;
        cp_async_elem(dst + r * LD + c, core + (static_cast<int64_t>(r) * I + i) * cols + c);
      }
    }
  } else {
    for (int idx = threadIdx.x; idx < rows * cols; idx += NT) {
      const int c = idx / rows, r = idx - c * rows;
      cp_async_elem(dst + r * LD + c, core + (static_cast<int64_t>(c) * I + i) * rows + r);
    }
  }
}

// acc[a][b] += sum_{k<K} A[k][m0+a] * B[k][n0+b]   (A, B row stride LD)
template <typename T, int TM, int LD>
__device__ __forceinline__ void outer_product(T (&acc)[TM][TM], const T* __restrict__ A, const T* __restrict__ B,
                                              int K, int m0, int n0) {
#pragma unroll 2
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

template <typename T>
__device__ __forceinline__ void track(int& lexp, int& lbad, T s) {
  if (!isfinite(s)) lbad = 1;
  else if (s != T(0)) lexp = max(lexp, exp2_of(static_cast<double>(s)));
}

// Block-wide max exponent / or of bad flags; every thread gets the result.
template <int NW>
__device__ __forceinline__ void block_exp(int& lexp, int& lbad, int* ired) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  lexp = __reduce_max_sync(0xffffffffu, lexp);
  lbad = __reduce_or_sync(0xffffffffu, lbad);
  if (lane == 0) {
    ired[warp] = lexp;
    ired[16 + warp] = lbad;
  }
  __syncthreads();
  int m = kNoExp, b = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    m = max(m, ired[w]);
    b |= ired[16 + w];
  }
  lexp = m;
  lbad = b;
}

// Position in the stream of slice loads of one CTA: job (mode j, slice i),
// operand which = 0 (B_i) or 1 (A_i).
struct LoadIt {
  int j, i, which;
  bool valid;
};

__device__ __forceinline__ void it_settle(LoadIt& it, const SweepParams& p, int n_pipe, int crank) {
  while (it.j < n_pipe && it.i >= p.step[it.j].I) {
    ++it.j;
    it.i = crank;
  }
  it.valid = it.j < n_pipe;
}
__device__ __forceinline__ void it_first(LoadIt& it, const SweepParams& p, int n_pipe, int crank) {
  it.j = 0;
  it.i = crank;
  it.which = 0;
  it_settle(it, p, n_pipe, crank);
}
__device__ __forceinline__ void it_next(LoadIt& it, const SweepParams& p, int n_pipe, int crank, int C) {
  if (it.which == 0) {
    it.which = 1;
    return;
  }
  it.which = 0;
  it.i += C;
  it_settle(it, p, n_pipe, crank);
}

template <typename T, int RM>
__global__ void __launch_bounds__(256, 1) sweep_cluster_kernel(const __grid_constant__ SweepParams p) {
  using Cfg = SweepCfg<T, RM>;
  using VT = typename Vec16<T>::type;
  constexpr int NT = Cfg::NT, NW = Cfg::NW, TM = Cfg::TM, LD = Cfg::LD, V = Cfg::V, NBUF = Cfg::NBUF;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Es = reinterpret_cast<T*>(smem_raw);  // E transposed: Es[q][p] = E[p][q]
  T* Ts = Es + Cfg::TILE;                  // T = E B_i; the partial P at a mode's end
  T* Rs = Ts + Cfg::TILE;                  // reduced rows (this is buf[0] when NBUF == 1)
  T* buf0 = Es + Cfg::NFIX * Cfg::TILE;
  int* ired = reinterpret_cast<int*>(buf0 + NBUF * Cfg::TILE);

  cg::cluster_group cluster = cg::this_cluster();
  const int C = static_cast<int>(cluster.num_blocks());
  const int crank = static_cast<int>(cluster.block_rank());
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  const int warp = tid >> 5, lane = tid & 31;
  const int n_pipe = p.final_scalar ? p.n_steps - 1 : p.n_steps;

  int64_t log2s = 0;
  int bad = 0;

  // ---- start environment ----
  if (p.e_in == nullptr) {
    if (tid == 0) Es[0] = T(1);
  } else {
    const T* e = static_cast<const T*>(p.e_in);
    for (int idx = tid; idx < p.rx0 * p.ry0; idx += NT) {
      const int a = idx / p.ry0, b = idx - a * p.ry0;
      Es[b * LD + a] = e[idx];
    }
    if (p.e_in_log2 != nullptr) log2s = *p.e_in_log2;
  }

  // ---- slice-load pipeline ----
  LoadIt prod, cons;
  it_first(prod, p, n_pipe, crank);
  it_first(cons, p, n_pipe, crank);
  int Lp = 0, Lc = 0;
  auto produce = [&]() {
    if (prod.valid) {
      const SweepStep& st = p.step[prod.j];
      T* dst = buf0 + (Lp % NBUF) * Cfg::TILE;
      if (prod.which == 0)
        load_slice_async<T, LD, NT>(dst, static_cast<const T*>(st.gy), prod.i, st.I, st.rin_y, st.rout_y,
                                    p.transposed);
      else
        load_slice_async<T, LD, NT>(dst, static_cast<const T*>(st.gx), prod.i, st.I, st.rin_x, st.rout_x,
                                    p.transposed);
      ++Lp;
      it_next(prod, p, n_pipe, crank, C);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int s = 0; s < NBUF - 1; ++s) produce();
  __syncthreads();

  for (int j = 0; j < n_pipe; ++j) {
    const SweepStep st = p.step[j];
    T acc[TM][TM];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TM; ++b) acc[a][b] = T(0);
    const int p0 = ty * TM, v0 = tx * TM;

    while (cons.valid && cons.j == j) {
      // T = E B_i
      produce();
      cp_async_wait<NBUF - 1>();
      __syncthreads();
      const T* Bs = buf0 + (Lc % NBUF) * Cfg::TILE;
      ++Lc;
      {
        T t[TM][TM];
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
          for (int b = 0; b < TM; ++b) t[a][b] = T(0);
        if (p0 < st.rin_x && v0 < st.rout_y) outer_product<T, TM, LD>(t, Es, Bs, st.rin_y, p0, v0);
#pragma unroll
        for (int a = 0; a < TM; ++a) {
          T* row = Ts + (p0 + a) * LD + v0;
#pragma unroll
          for (int b = 0; b < TM; ++b) row[b] = t[a][b];
        }
      }
      __syncthreads();
      it_next(cons, p, n_pipe, crank, C);
      // P += A_i^T T
      produce();
      cp_async_wait<NBUF - 1>();
      __syncthreads();
      const T* As = buf0 + (Lc % NBUF) * Cfg::TILE;
      ++Lc;
      if (p0 < st.rout_x && v0 < st.rout_y) outer_product<T, TM, LD>(acc, As, Ts, st.rin_x, p0, v0);
      __syncthreads();
      it_next(cons, p, n_pipe, crank, C);
    }

    const int nu = st.rout_x, nv = st.rout_y;
    if (C == 1) {
      int lexp = kNoExp, lbad = 0;
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TM; ++b)
          if (p0 + a < nu && v0 + b < nv) track(lexp, lbad, acc[a][b]);
      block_exp<NW>(lexp, lbad, ired);
      if (lbad) bad = 1;
      const bool rescale = lexp != kNoExp && (lexp > p.renorm_bits || lexp < -p.renorm_bits);
      if (rescale) log2s += lexp;
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TM; ++b)
          Es[(v0 + b) * LD + p0 + a] = rescale ? mul_pow2<T>(acc[a][b], -lexp) : acc[a][b];
      __syncthreads();
      continue;
    }

    // ---- cluster reduction: E'[u][v] = sum over CTAs of P_c[u][v] ----
#pragma unroll
    for (int a = 0; a < TM; ++a) {
      T* row = Ts + (p0 + a) * LD + v0;
#pragma unroll
      for (int b = 0; b < TM; ++b) row[b] = acc[a][b];
    }
    cluster.sync();
    const int nvv = (nv + V - 1) / V;
    const int chunk = (nu + C - 1) / C;
    const int ub = min(nu, crank * chunk), ue = min(nu, ub + chunk);
    int lexp = kNoExp, lbad = 0;
    for (int idx = tid; idx < (ue - ub) * nvv; idx += NT) {
      const int u = ub + idx / nvv, c = (idx % nvv) * V;
      VT s = Vec16<T>::zero();
      for (int r = 0; r < C; ++r)
        s = Vec16<T>::add(s, *reinterpret_cast<const VT*>(cluster.map_shared_rank(Ts + u * LD + c, r)));
      *reinterpret_cast<VT*>(Rs + u * LD + c) = s;
#pragma unroll
      for (int q = 0; q < V; ++q)
        if (c + q < nv) track(lexp, lbad, Vec16<T>::get(s, q));
    }
    lexp = __reduce_max_sync(0xffffffffu, lexp);
    lbad = __reduce_or_sync(0xffffffffu, lbad);
    if (lane == 0) {
      ired[warp] = lexp;
      ired[16 + warp] = lbad;
    }
    __syncthreads();
    if (tid == 0) {
      int m = kNoExp, bb = 0;
      for (int w = 0; w < NW; ++w) {
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
    const bool rescale = gexp != kNoExp && (gexp > p.renorm_bits || gexp < -p.renorm_bits);
    if (rescale) log2s += gexp;
    for (int idx = tid; idx < nu * nvv; idx += NT) {
      const int u = idx / nvv, c = (idx % nvv) * V;
      const int owner = u / chunk;
      const VT v = *reinterpret_cast<const VT*>(cluster.map_shared_rank(Rs + u * LD + c, owner));
#pragma unroll
      for (int q = 0; q < V; ++q) {
        const T e = Vec16<T>::get(v, q);
        Es[(c + q) * LD + u] = rescale ? mul_pow2<T>(e, -gexp) : e;
      }
    }
    if (NBUF == 1) cluster.sync();  // peers finished reading Rs (= slice buffer) before it is reused
    __syncthreads();
  }

  // ---- last mode of a full contraction: float64 sum ----
  if (p.final_scalar) {
    const SweepStep st = p.step[p.n_steps - 1];
    const T* gx = static_cast<const T*>(st.gx);
    const T* gy = static_cast<const T*>(st.gy);
    const int I = st.I;
    T* bvec = buf0;       // B_i[q][0]
    T* avec = buf0 + LD;  // A_i[p][0]
    double part = 0.0;
    for (int i = crank; i < I; i += C) {
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
    double* dred = reinterpret_cast<double*>(ired + 96);  // 16 doubles (ired has 128 ints)
    if (lane == 0) dred[warp] = part;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < NW; ++w) s += dred[w];
      dred[8] = s;
    }
    cluster.sync();
    if (crank == 0 && tid == 0) {
      double z = 0.0;
      for (int r = 0; r < C; ++r) z += *cluster.map_shared_rank(dred + 8, r);
      int st_bits = (isfinite(z) && !bad) ? 0 : TT_STATUS_NONFINITE;
      if (p.z_out_log2 != nullptr) {
        *p.z_out = z;
        *p.z_out_log2 = log2s;
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
        *p.z_out = v;
      }
      set_status(p.status, st_bits);
    }
    cluster.sync();  // keep peers' shared memory alive until CTA 0 has read it
    return;
  }

  // ---- environment output ----
  const int kx = p.n_steps > 0 ? p.step[p.n_steps - 1].rout_x : p.rx0;
  const int ky = p.n_steps > 0 ? p.step[p.n_steps - 1].rout_y : p.ry0;
  if (crank == 0 && p.e_out != nullptr) {
    T* e = static_cast<T*>(p.e_out);
    for (int idx = tid; idx < kx * ky; idx += NT) {
      const int u = idx / ky, v = idx - u * ky;
      e[idx] = Es[v * LD + u];
    }
    if (tid == 0 && p.e_out_log2 != nullptr) *p.e_out_log2 = log2s;
  }

  // ---- chain emission: C = boundary core joined with K, then the copies ----
  if (p.emit.enabled) {
    const EmitParams& em = p.emit;
    // K row-major into Ts: Ts[a][y] = K[a][y] = Es[y][a]
    for (int idx = tid; idx < kx * ky; idx += NT) {
      const int a = idx / ky, y = idx - a * ky;
      Ts[a * LD + y] = Es[y * LD + a];
    }
    const T* gx = static_cast<const T*>(em.gx);
    T* cout = static_cast<T*>(em.c_out);
    const int nu = em.lead ? em.rb : em.ra;
    const bool fold = em.z_log2_out == nullptr && log2s != 0;
    int ebits = 0;
    const int u0 = ty * TM, y0 = tx * TM;
    for (int i = crank; i < em.I; i += C) {
      __syncthreads();
      if (em.lead) load_slice_async<T, LD, NT>(buf0, gx, i, em.I, em.ra, em.rb, 0);
      else load_slice_async<T, LD, NT>(buf0, gx, i, em.I, em.rb, em.ra, 1);
      cp_async_commit();
      cp_async_wait<0>();
      __syncthreads();
      T acc[TM][TM];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TM; ++b) acc[a][b] = T(0);
      if (u0 < nu && y0 < em.ry) outer_product<T, TM, LD>(acc, buf0, Ts, kx, u0, y0);
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TM; ++b) {
          const int u = u0 + a, y = y0 + b;
          if (u < nu && y < em.ry) {
            T s = acc[a][b];
            if (fold) {
              const T s0 = s;
              s = scale_pow2_sat<T>(s, log2s);
              if (isfinite(s0) && !isfinite(s)) ebits |= TT_STATUS_OVERFLOW;
            }
            if (!isfinite(s)) ebits |= TT_STATUS_NONFINITE;
            cout[(static_cast<int64_t>(u) * em.I + i) * em.ry + y] = s;
          }
        }
    }
    if (ebits) set_status(p.status, ebits);
    if (crank == 0 && tid == 0 && em.z_log2_out != nullptr) *em.z_log2_out = log2s;
    // free cores: plain or leg-swapped copies, grid-stride over the cluster
    const int64_t g = static_cast<int64_t>(crank) * NT + tid, gs = static_cast<int64_t>(C) * NT;
    for (int t = 0; t < em.n_copies; ++t) {
      const CopyTask tk = em.copy[t];
      const T* __restrict__ src = static_cast<const T*>(tk.src);
      T* __restrict__ dst = static_cast<T*>(tk.dst);
      const int64_t n = static_cast<int64_t>(tk.r0) * tk.I * tk.r1;
      if (!tk.swap) {
        for (int64_t e = g; e < n; e += gs) dst[e] = ldg(src + e);
      } else {
        // dst is [r1][I][r0]; element e of dst = (c1, i, c0)
        for (int64_t e = g; e < n; e += gs) {
          const int64_t c0 = e % tk.r0, rest = e / tk.r0;
          const int64_t ii = rest % tk.I, c1 = rest / tk.I;
          dst[e] = ldg(src + (c0 * tk.I + ii) * tk.r1 + c1);
        }
      }
    }
  }
  if (tid == 0 && crank == 0 && bad) set_status(p.status, TT_STATUS_NONFINITE);
  cluster.sync();
}

template <typename T, int RM>
static cudaError_t prepare(int C) {
  auto kern = sweep_cluster_kernel<T, RM>;
  cudaError_t err =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(SweepCfg<T, RM>::SMEM));
  if (err != cudaSuccess) return err;
  if (C > 8) err = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return err;
}

template <typename T, int RM>
static cudaError_t launch_impl(const SweepParams& p, int C, cudaStream_t s) {
  cudaError_t err = prepare<T, RM>(C);
  if (err != cudaSuccess) return err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(SweepCfg<T, RM>::NT, 1, 1);
  cfg.dynamicSmemBytes = SweepCfg<T, RM>::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, sweep_cluster_kernel<T, RM>, p);
}

template <typename T, int RM>
static int cluster_size_impl(int want) {
  if (prepare<T, RM>(16) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  for (int C = want; C >= 1; C /= 2) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(SweepCfg<T, RM>::NT, 1, 1);
    cfg.dynamicSmemBytes = SweepCfg<T, RM>::SMEM;
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
  return 0;
}

// Cached per (rank tile, element size, wanted size) for the current device.
int sweep_cluster_size(int rmax, int elem_bytes, int want) {
  static int cache[2][4][17][8];  // [f64?][tile][want][device] ; 0 = unknown
  int dev = 0;
  cudaGetDevice(&dev);
  const int tile = rmax <= 32 ? 0 : (rmax <= 64 ? 1 : 2);
  const int d = elem_bytes == 8 ? 1 : 0;
  int* slot = (dev < 8 && want <= 16) ? &cache[d][tile][want][dev] : nullptr;
  if (slot != nullptr && *slot > 0) return *slot;
  int c = 0;
  if (elem_bytes == 4) {
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
