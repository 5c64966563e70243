// Environment sweep over contracted modes, as a device body shared by the
// single-contraction cluster kernel and the batched persistent kernel.
//
// One contracted mode folds the core pair into the running environment
// (the generalisation of Algorithm 2 step 4 / Example 1's K = A_x^T A_y):
//   E'[u][v] = sum_i  (A_i^T E B_i)[u][v]
// with A_i, B_i the i-th slices of the two cores (see SweepStep).  The sum
// over the mode index i is split across the CTAs of a cluster: CTA c owns
// slices i = c, c + C, ...  Per slice a CTA computes T = E B_i and
// P += A_i^T T out of shared memory with a register-blocked outer-product
// loop.  Core slices stream in 32-row chunks through a ring of NST stages
// filled by cp.async, NST-2 to NST-1 chunks ahead of the one being consumed
// (a chunk's copies are issued after the products of the chunk before); the
// loads do not depend on E, so the next mode's chunks land while the cluster
// is still reducing the current mode.  The cluster adds the partial P's through
// distributed shared memory: CTA c sums its share of rows over all peers
// (fixed order: deterministic), and every CTA gets the reduced rows back into
// its own copy of E'.  For float32 tiles up to rank 64 both exchanges are
// pushes: bulk asynchronous copies from a CTA's shared memory into its peers'
// (partial sums into receive slots, reduced rows straight into the peers'
// transposed environments), completed on an mbarrier of the receiver
// (bounded waits), so no cluster-wide barrier is taken per mode.  Other tiles
// pull from the peers' shared memory between two cluster barriers.
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
// chain walks X backwards).
#pragma once

#include <cooperative_groups.h>

#include <type_traits>

#include "tc_common.cuh"
#include "ttc_device.cuh"
#include "ttc_internal.h"

namespace ttc {

namespace cg = cooperative_groups;

constexpr int kNoExp = -(1 << 30);  // exponent marker of an all-zero environment
constexpr int KC = 32;               // rows per pipeline chunk (ranks above 64)

// Shared-memory plan of the sweep for element type T and rank tile RM.
//   CL: cluster mode (a reduction buffer of RM/2 rows is needed)
template <typename T, int RM, bool CL>
struct SweepCfg {
  // a CTA of a cluster runs 256 threads; a CTA working alone runs 512, so a
  // single SM still has 16 warps to hide the latency of its small GEMMs
  static constexpr int NT = CL ? 256 : 512;
  static constexpr int NW = NT / 32;
  static constexpr int IRED = 192;                 // ints of reduction scratch
  static constexpr int TM = RM / 16;               // thread tile of the chain emission (TM x TM)
  // sweep GEMMs: 4x4 sub-tiles dealt round-robin, at most NS per thread
  static constexpr int NS = ((RM / 4) * (RM / 4) + NT - 1) / NT;
  static constexpr int V = 16 / sizeof(T);         // elements per 16-byte vector
  static constexpr int LD = RM + V;                // row stride (elements), 16-byte padded
  static constexpr int TILE = RM * LD;
  static constexpr int RS_ROWS = CL ? RM / 2 : 0;  // a CTA of a cluster (C >= 2) reduces <= RM/2 rows
  // rows per pipeline chunk: a whole slice of a rank-64 core in one chunk
  static constexpr int KC = RM <= 64 ? 64 : ttc::KC;
  static constexpr int STAGE = KC * LD;
  static constexpr size_t kBudget = 232448 - 1024;
  // Push exchange (float, ranks <= 64, cluster): partial rows go to their
  // owner and reduced rows to every peer by bulk copies into receive buffers
  static constexpr bool PUSH = CL && sizeof(T) == 4 && RM <= 64;
  static constexpr int RB_ROWS = RM + 16;            // C slots of ceil(RM / C) rows
  static constexpr size_t XB = PUSH ? (RB_ROWS * LD * sizeof(T) + 16 * 16 + 16 + 16) : 0;
  static constexpr size_t FIXED = (2 * TILE + RS_ROWS * LD) * sizeof(T) + IRED * sizeof(int) +
                                  kMaxOrder * sizeof(SweepStep) + XB;
  static constexpr int NST_FIT = static_cast<int>((kBudget - FIXED) / (STAGE * sizeof(T)));
  static constexpr int NST = NST_FIT >= 4 ? 4 : NST_FIT;
  static_assert(NST >= 2, "sweep tile does not fit in shared memory");
  static constexpr size_t SMEM = FIXED + static_cast<size_t>(NST) * STAGE * sizeof(T);
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

// Asynchronously copy rows [r0, r0 + nr) of slice i of a core into dst[r - r0][c]
// (row stride LD).
//   transposed == 0: core is [rows][I][cols], dst[r][c] = core[r][i][c]
//   transposed == 1: core is [cols][I][rows], dst[r][c] = core[c][i][r]
template <typename T, int LD, int NT>
__device__ __forceinline__ void load_rows_async(T* __restrict__ dst, const T* __restrict__ core, int i, int I,
                                                int rows, int cols, int transposed, int r0, int nr) {
  constexpr int NW = NT / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (!transposed) {
    constexpr int V = 16 / sizeof(T);
    if ((cols % V) == 0 && (reinterpret_cast<uintptr_t>(core) & 15) == 0) {
      const int cv = cols / V;
      for (int idx = threadIdx.x; idx < nr * cv; idx += NT) {
        const int r = idx / cv, c = (idx - r * cv) * V;
        cp_async16(dst + r * LD + c, core + (static_cast<int64_t>(r0 + r) * I + i) * cols + c);
      }
    } else {
      // one warp per row, lanes along the row: coalesced, no division
      for (int r = warp; r < nr; r += NW) {
        const T* src = core + (static_cast<int64_t>(r0 + r) * I + i) * cols;
        for (int c = lane; c < cols; c += 32) cp_async_elem(dst + r * LD + c, src + c);
      }
    }
  } else {
    // one warp per source row (a column of dst), lanes along it
    for (int c = warp; c < cols; c += NW) {
      const T* src = core + (static_cast<int64_t>(c) * I + i) * rows + r0;
      for (int r = lane; r < nr; r += 32) cp_async_elem(dst + r * LD + c, src + r);
    }
  }
}

// dst[e] = src[e] for e = g, g + gs, ... < n, four loads in flight per thread.
template <typename T>
__device__ __forceinline__ void copy_plain(T* __restrict__ dst, const T* __restrict__ src, int64_t n, int64_t g,
                                           int64_t gs) {
  int64_t e = g;
  for (; e + 3 * gs < n; e += 4 * gs) {
    const T a0 = ldg(src + e), a1 = ldg(src + e + gs), a2 = ldg(src + e + 2 * gs), a3 = ldg(src + e + 3 * gs);
    dst[e] = a0;
    dst[e + gs] = a1;
    dst[e + 2 * gs] = a2;
    dst[e + 3 * gs] = a3;
  }
  for (; e < n; e += gs) dst[e] = ldg(src + e);
}

// dst[c1][i][c0] = src[c0][i][c1] for one core ([r0][I][r1] -> [r1][I][r0]),
// through 32 x 32 shared-memory tiles so both the reads and the writes are
// coalesced.  Tiles are dealt to the CTAs of the cluster.
template <typename T, int NT>
__device__ void copy_swap_tiled(T* __restrict__ dst, const T* __restrict__ src, int r0, int I, int r1, T* tile,
                                int C, int crank) {
  constexpr int NW = NT / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t0 = (r0 + 31) / 32, t1 = (r1 + 31) / 32;
  const int ntiles = I * t0 * t1;
  for (int job = crank; job < ntiles; job += C) {
    const int i = job / (t0 * t1);
    const int rem = job - i * t0 * t1;
    const int b0 = (rem / t1) * 32, b1 = (rem % t1) * 32;
    __syncthreads();
    for (int rr = warp; rr < 32; rr += NW) {
      const int c0 = b0 + rr, c1 = b1 + lane;
      if (c0 < r0 && c1 < r1) tile[rr * 33 + lane] = src[(static_cast<int64_t>(c0) * I + i) * r1 + c1];
    }
    __syncthreads();
    for (int rr = warp; rr < 32; rr += NW) {
      const int c1 = b1 + rr, c0 = b0 + lane;
      if (c0 < r0 && c1 < r1) dst[(static_cast<int64_t>(c1) * I + i) * r0 + c0] = tile[lane * 33 + rr];
    }
  }
}

// acc[a][b] += sum_{k<K} A[k][m0+a] * B[k][n0+b]   (A, B row stride LD)
template <typename T, int TM, int LD>
__device__ __forceinline__ void outer_product(T (&acc)[TM][TM], const T* __restrict__ A, const T* __restrict__ B,
                                              int K, int m0, int n0) {
#pragma unroll 4
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

// Sub-tile j of the calling thread in an M x N output covered by 4x4
// sub-tiles in row-major order: consecutive threads take consecutive column
// blocks, so their 16-byte operand reads are contiguous (no bank conflicts)
// and every thread has work whatever the ranks of the mode.
struct Sub {
  int m0, n0;
  bool on;
};
template <int NT>
__device__ __forceinline__ Sub sub_tile(int j, int M, int N) {
  const int ncb = (N + 3) >> 2;
  const int s = static_cast<int>(threadIdx.x) + j * NT;
  Sub t;
  t.on = s < ((M + 3) >> 2) * ncb;
  const int r = s / ncb;
  t.m0 = r * 4;
  t.n0 = (s - r * ncb) * 4;
  return t;
}

template <typename T>
__device__ __forceinline__ void track(int& lexp, int& lbad, T s) {
  if (!isfinite(s)) lbad = 1;
  else if (s != T(0)) lexp = max(lexp, exp2_bits(s));
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

// Position in the stream of chunk loads of one CTA: job (mode j, slice i),
// operand which = 0 (B_i, rin_y rows) or 1 (A_i, rin_x rows), chunk c of nch.
struct ChunkIt {
  int j, i, which, c, nch;
  bool valid;
};

template <int KCV>
__device__ __forceinline__ int nchunks(int rows) {
  return (rows + KCV - 1) / KCV;
}

template <int KCV>
__device__ __forceinline__ void it_settle(ChunkIt& it, const SweepStep* steps, int n_pipe, int crank) {
  while (it.j < n_pipe && it.i >= steps[it.j].I) {
    ++it.j;
    it.i = crank;
  }
  it.valid = it.j < n_pipe;
  if (it.valid) it.nch = nchunks<KCV>(steps[it.j].rin_y);
}
template <int KCV>
__device__ __forceinline__ void it_first(ChunkIt& it, const SweepStep* steps, int n_pipe, int crank) {
  it.j = 0;
  it.i = crank;
  it.which = 0;
  it.c = 0;
  it_settle<KCV>(it, steps, n_pipe, crank);
}
template <int KCV>
__device__ __forceinline__ void it_next(ChunkIt& it, const SweepStep* steps, int n_pipe, int crank, int C) {
  if (++it.c < it.nch) return;
  it.c = 0;
  if (it.which == 0) {
    it.which = 1;
    it.nch = nchunks<KCV>(steps[it.j].rin_x);
    return;
  }
  it.which = 0;
  it.i += C;
  it_settle<KCV>(it, steps, n_pipe, crank);
}

// A chain emission whose K fits one pipeline chunk gets its first boundary-core
// slice loaded during the last mode of the sweep (sweep_body issues it,
// sweep_tail only waits for it).
template <int KCV>
__device__ __forceinline__ bool emit_prefetched(const SweepParams& p, int crank) {
  return p.emit.enabled && !p.final_scalar && p.n_steps > 0 && p.step[p.n_steps - 1].rout_x <= KCV &&
         crank < p.emit.I;
}

// Where results and device status go (per call; the batched kernel points
// these at its per-pair slots).
struct SweepOut {
  double* z_out;
  int64_t* z_out_log2;
  int32_t* status;
  int skip_copies = 0;  // the free-core copies are done elsewhere (batched launch)
};

// Result of a sweep that is not a full contraction: E (in Es, transposed) and
// its scale; the caller continues with the environment output / emission.
template <typename T, int RM, bool CL>
struct SweepState {
  int64_t log2s;
  int bad;
};

// The sweep itself.  Returns false when it handled a final scalar (full
// contraction) and nothing is left to do.
template <typename T, int RM, bool CL>
__device__ __forceinline__ bool sweep_body(const SweepParams& p, const SweepOut& o, unsigned char* smem, int C,
                                           int crank, SweepState<T, RM, CL>& out) {
  using Cfg = SweepCfg<T, RM, CL>;
  using VT = typename Vec16<T>::type;
  constexpr int NT = Cfg::NT, NW = Cfg::NW, LD = Cfg::LD, V = Cfg::V, NST = Cfg::NST;
  T* Es = reinterpret_cast<T*>(smem);  // E transposed: Es[q][p] = E[p][q]
  T* Ts = Es + Cfg::TILE;              // T = E B_i; the partial P at a mode's end
  T* Rs = Ts + Cfg::TILE;              // reduced rows of this CTA (cluster mode)
  T* stage0 = Rs + Cfg::RS_ROWS * LD;
  int* ired = reinterpret_cast<int*>(stage0 + NST * Cfg::STAGE);
  SweepStep* sst = reinterpret_cast<SweepStep*>(ired + Cfg::IRED);  // step table cached on chip
  // push-exchange buffers (16-byte aligned: the step table is 48 * 64 bytes)
  T* Rb = reinterpret_cast<T*>(sst + kMaxOrder);   // receive slots [C][chunk][LD]
  int* grec = reinterpret_cast<int*>(Rb + Cfg::RB_ROWS * LD);  // 16 records of 16 bytes: (exponent, bad)
  int* srec = grec + 64;                            // this CTA's record
  uint64_t* xbar = reinterpret_cast<uint64_t*>(srec + 4);  // [0] partial rows in, [1] reduced rows in
  int xph = 0;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int n_pipe = p.final_scalar ? p.n_steps - 1 : p.n_steps;
  const bool emit_prefetch = emit_prefetched<Cfg::KC>(p, crank);

  int64_t log2s = 0;
  int bad = 0;

  // ---- start environment: [1] (the trains start and end with rank 1), or
  //      a given one (the sum of its parts, added in order) ----
  if (p.e_seed != nullptr) {
    const int ry0 = p.ry0;
    sum_parts<T, NT>(static_cast<const T*>(p.e_seed), p.rx0 * ry0, p.e_seed_parts > 1 ? p.e_seed_parts : 1,
                     [&](int idx, T e) {
                       const int u = idx / ry0, v = idx - u * ry0;
                       Es[v * LD + u] = e;
                     });
    if (p.e_seed_log2 != nullptr) log2s = *p.e_seed_log2;
  } else if (tid == 0) {
    Es[0] = T(1);
  }

  for (int q = tid; q < p.n_steps; q += NT) sst[q] = p.step[q];
  if constexpr (Cfg::PUSH) {
    if (tid == 0) {
      tc::mbar_init(&xbar[0], 1);
      tc::mbar_init(&xbar[1], 1);
      tc::mbar_init_fence();
      ired[Cfg::IRED - 1] = 0;  // abort flag of the bounded waits
    }
    cg::this_cluster().sync();  // barriers exist before any peer pushes
  }
  __syncthreads();

  // ---- chunk pipeline ----
  ChunkIt prod, cons;
  it_first<Cfg::KC>(prod, sst, n_pipe, crank);
  it_first<Cfg::KC>(cons, sst, n_pipe, crank);
  int Lp = 0, Lc = 0;
  auto produce = [&]() {
    if (prod.valid) {
      const SweepStep& st = sst[prod.j];
      T* dst = stage0 + (Lp % NST) * Cfg::STAGE;
      const int rows = prod.which == 0 ? st.rin_y : st.rin_x;
      const int cols = prod.which == 0 ? st.rout_y : st.rout_x;
      const T* core = static_cast<const T*>(prod.which == 0 ? st.gy : st.gx);
      const int r0 = prod.c * Cfg::KC;
      load_rows_async<T, LD, NT>(dst, core, prod.i, st.I, rows, cols, prod.which == 0 ? p.transposed_y : p.transposed,
                                 r0, min(Cfg::KC, rows - r0));
      ++Lp;
      it_next<Cfg::KC>(prod, sst, n_pipe, crank, C);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int s = 0; s < NST - 1; ++s) produce();
  __syncthreads();

  // One contracted mode; NSE = sub-tiles per thread this mode needs (the
  // largest tile runs the one-sub-tile code whenever the ranks allow).
  auto mode = [&](const int j, auto nse_tag) {
    constexpr int NSE = decltype(nse_tag)::value;
    const SweepStep st = sst[j];
    T acc[NSE][4][4];
#pragma unroll
    for (int u = 0; u < NSE; ++u)
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[u][a][b] = T(0);

    while (cons.valid && cons.j == j) {
      // ---- T = E B_i over chunks of q ----
      T t[NSE][4][4];
#pragma unroll
      for (int u = 0; u < NSE; ++u)
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) t[u][a][b] = T(0);
      while (true) {
        cp_async_wait<NST - 2>();
        __syncthreads();
        const T* Bs = stage0 + (Lc % NST) * Cfg::STAGE;
        ++Lc;
        const int q0 = cons.c * Cfg::KC, kc = min(Cfg::KC, st.rin_y - q0);
#pragma unroll
        for (int u = 0; u < NSE; ++u) {
          const Sub sb = sub_tile<NT>(u, st.rin_x, st.rout_y);
          if (sb.on) outer_product<T, 4, LD>(t[u], Es + q0 * LD, Bs, kc, sb.m0, sb.n0);
        }
        produce();  // refills the stage the barrier above freed, overlapping other warps' products
        const bool last = cons.c + 1 == cons.nch;
        it_next<Cfg::KC>(cons, sst, n_pipe, crank, C);
        if (last) break;
      }
#pragma unroll
      for (int u = 0; u < NSE; ++u) {
        const Sub sb = sub_tile<NT>(u, st.rin_x, st.rout_y);
        if (sb.on) {
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            T* row = Ts + (sb.m0 + a) * LD + sb.n0;
            if constexpr (sizeof(T) == 4) {
              *reinterpret_cast<float4*>(row) = make_float4(t[u][a][0], t[u][a][1], t[u][a][2], t[u][a][3]);
            } else {
              *reinterpret_cast<double2*>(row) = make_double2(t[u][a][0], t[u][a][1]);
              *reinterpret_cast<double2*>(row + 2) = make_double2(t[u][a][2], t[u][a][3]);
            }
          }
        }
      }
      // ---- P += A_i^T T over chunks of p ----
      while (true) {
        cp_async_wait<NST - 2>();
        __syncthreads();
        const T* As = stage0 + (Lc % NST) * Cfg::STAGE;
        ++Lc;
        const int r0 = cons.c * Cfg::KC, kc = min(Cfg::KC, st.rin_x - r0);
#pragma unroll
        for (int u = 0; u < NSE; ++u) {
          const Sub sb = sub_tile<NT>(u, st.rout_x, st.rout_y);
          if (sb.on) outer_product<T, 4, LD>(acc[u], As, Ts + r0 * LD, kc, sb.m0, sb.n0);
        }
        produce();
        const bool last = cons.c + 1 == cons.nch;
        it_next<Cfg::KC>(cons, sst, n_pipe, crank, C);
        if (last) break;
      }
    }
    __syncthreads();  // every thread is done reading Es / Ts of this mode
    if (j == n_pipe - 1 && emit_prefetch) {
      // the first slice of the boundary core this CTA joins with K after the
      // sweep (every chunk of the ring has been consumed, so stage 0 is free):
      // its load overlaps the cluster exchange of the last mode
      const EmitParams& em = p.emit;
      const T* gx = static_cast<const T*>(em.gx);
      if (em.lead) load_rows_async<T, LD, NT>(stage0, gx, crank, em.I, em.ra, em.rb, 0, 0, st.rout_x);
      else load_rows_async<T, LD, NT>(stage0, gx, crank, em.I, em.rb, em.ra, 1, 0, st.rout_x);
      cp_async_commit();
    }

    const int nu = st.rout_x, nv = st.rout_y;
    if (!CL || C == 1) {
      int lexp = kNoExp, lbad = 0;
#pragma unroll
      for (int u = 0; u < NSE; ++u) {
        const Sub sb = sub_tile<NT>(u, nu, nv);
        if (sb.on) {
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
              if (sb.m0 + a < nu && sb.n0 + b < nv) track(lexp, lbad, acc[u][a][b]);
        }
      }
      block_exp<NW>(lexp, lbad, ired);
      if (lbad) bad = 1;
      const bool rescale = lexp != kNoExp && (lexp > p.renorm_bits || lexp < -p.renorm_bits);
      if (rescale) log2s += lexp;
#pragma unroll
      for (int u = 0; u < NSE; ++u) {
        const Sub sb = sub_tile<NT>(u, nu, nv);
        if (sb.on) {
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
              Es[(sb.n0 + b) * LD + sb.m0 + a] = rescale ? mul_pow2<T>(acc[u][a][b], -lexp) : acc[u][a][b];
        }
      }
      __syncthreads();
      return;
    }

    if constexpr (CL) {
      cg::cluster_group cluster = cg::this_cluster();
      // ---- cluster reduction: E'[u][v] = sum over CTAs of P_c[u][v] ----
      if constexpr (Cfg::PUSH) {
        // Push exchange.  Partial sums are staged transposed (Ts[v][u]) and
        // owned by blocks of v, so an owner's reduced block is whole rows of
        // every CTA's transposed environment Es[v][u]: it is pushed straight
        // into the peers' Es.  One lane per peer issues the bulk copies.
#pragma unroll
        for (int u = 0; u < NSE; ++u) {
          const Sub sb = sub_tile<NT>(u, nu, nv);
          if (sb.on) {
#pragma unroll
            for (int b = 0; b < 4; ++b)
              *reinterpret_cast<float4*>(Ts + (sb.n0 + b) * LD + sb.m0) =
                  make_float4(acc[u][0][b], acc[u][1][b], acc[u][2][b], acc[u][3][b]);
          }
        }
        const int chunk = (nv + C - 1) / C;
        const uint32_t rowb = LD * sizeof(T);
        const int my0 = min(nv, crank * chunk), my_rows = min(nv, my0 + chunk) - my0;
        volatile int* abort = ired + Cfg::IRED - 1;
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) tc::mbar_expect_tx(&xbar[0], static_cast<uint32_t>(C * my_rows) * rowb);
        if (tid < C) {
          const int o = tid;
          const int r0o = min(nv, o * chunk), ro = min(nv, r0o + chunk) - r0o;
          if (ro > 0)
            tc::bulk_s2c(tc::mapa(tc::su32(Rb + crank * chunk * LD), o), Ts + r0o * LD, ro * rowb,
                         tc::mapa(tc::su32(&xbar[0]), o));
        }
        if (!tc::mbar_wait(&xbar[0], xph & 1, abort)) {
          bad = 1;
          set_status(o.status, TT_STATUS_TIMEOUT);
        }
        // owner sum over the C peers: four threads per 4-column vector, C/4 peers each
        const int nuv = (nu + 3) / 4;
        float lmax = 0.f;
        int lbad = 0;
        const int sub = tid & 3;
        const int nbase = my_rows * nuv, niter = (nbase + NT / 4 - 1) / (NT / 4);  // same for every thread
        for (int it = 0; it < niter; ++it) {
          const int base = (tid >> 2) + it * (NT / 4);
          const bool act = base < nbase;
          const int v = act ? base / nuv : 0, c = act ? (base - v * nuv) * 4 : 0;
          float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
          for (int r = sub; act && r < C; r += 4) {
            const float4 x = *reinterpret_cast<const float4*>(Rb + (r * chunk + v) * LD + c);
            sum.x += x.x;
            sum.y += x.y;
            sum.z += x.z;
            sum.w += x.w;
          }
#pragma unroll
          for (int off = 1; off < 4; off <<= 1) {
            sum.x += __shfl_xor_sync(0xffffffffu, sum.x, off);
            sum.y += __shfl_xor_sync(0xffffffffu, sum.y, off);
            sum.z += __shfl_xor_sync(0xffffffffu, sum.z, off);
            sum.w += __shfl_xor_sync(0xffffffffu, sum.w, off);
          }
          if (act && sub == 0) {
            *reinterpret_cast<float4*>(Rs + v * LD + c) = sum;
            const float e4[4] = {sum.x, sum.y, sum.z, sum.w};
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (c + q < nu) {
                if (isfinite(e4[q])) lmax = fmaxf(lmax, fabsf(e4[q]));
                else lbad = 1;
              }
          }
        }
        // binary exponent e of the largest entry, 2^(e-1) <= max < 2^e (0 -> none)
        int lexp = lmax > 0.f ? static_cast<int>((__float_as_uint(lmax) >> 23) & 0xff) - 126 : kNoExp;
        block_exp<NW>(lexp, lbad, ired);
        if (tid == 0) {
          srec[0] = lexp;
          srec[1] = lbad;
          tc::mbar_expect_tx(&xbar[1], static_cast<uint32_t>(nv) * rowb + 16u * C);
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (tid < C) {
          const int o = tid;
          if (my_rows > 0)
            tc::bulk_s2c(tc::mapa(tc::su32(Es + my0 * LD), o), Rs, my_rows * rowb, tc::mapa(tc::su32(&xbar[1]), o));
          tc::bulk_s2c(tc::mapa(tc::su32(grec + 4 * crank), o), srec, 16, tc::mapa(tc::su32(&xbar[1]), o));
        }
        if (!tc::mbar_wait(&xbar[1], xph & 1, abort)) {
          bad = 1;
          set_status(o.status, TT_STATUS_TIMEOUT);
        }
        ++xph;
        int gexp = kNoExp, gbad = 0;
        for (int r = 0; r < C; ++r) {
          gexp = max(gexp, grec[4 * r]);
          gbad |= grec[4 * r + 1];
        }
        if (gbad) bad = 1;
        if (gexp != kNoExp && (gexp > p.renorm_bits || gexp < -p.renorm_bits)) {
          log2s += gexp;
          for (int idx = tid; idx < nv * nu; idx += NT) {
            const int v = idx / nu, u = idx - v * nu;
            Es[v * LD + u] = mul_pow2<T>(Es[v * LD + u], -gexp);
          }
        }
        __syncthreads();
        return;
      } else {
#pragma unroll
        for (int u = 0; u < NSE; ++u) {
          const Sub sb = sub_tile<NT>(u, nu, nv);
          if (sb.on) {
#pragma unroll
            for (int a = 0; a < 4; ++a) {
              T* row = Ts + (sb.m0 + a) * LD + sb.n0;
#pragma unroll
              for (int b = 0; b < 4; ++b) row[b] = acc[u][a][b];
            }
          }
        }
        cluster.sync();
        const int nvv = (nv + V - 1) / V;
        const int chunk = (nu + C - 1) / C;
        const int ub = min(nu, crank * chunk), ue = min(nu, ub + chunk);
        int lexp = kNoExp, lbad = 0;
        for (int idx = tid; idx < (ue - ub) * nvv; idx += NT) {
          const int u = ub + idx / nvv, c = (idx % nvv) * V;
          VT part[16];
#pragma unroll
          for (int r = 0; r < 16; ++r)
            if (r < C) part[r] = *reinterpret_cast<const VT*>(cluster.map_shared_rank(Ts + u * LD + c, r));
          VT s = Vec16<T>::zero();
#pragma unroll
          for (int r = 0; r < 16; ++r)
            if (r < C) s = Vec16<T>::add(s, part[r]);
          *reinterpret_cast<VT*>(Rs + (u - ub) * LD + c) = s;
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
        if (tid < C) {
          int m = kNoExp, bb = 0;
          for (int w = 0; w < NW; ++w) {
            m = max(m, ired[w]);
            bb |= ired[16 + w];
          }
          *cluster.map_shared_rank(ired + 32 + crank, tid) = m;
          *cluster.map_shared_rank(ired + 64 + crank, tid) = bb;
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
          const VT v =
              *reinterpret_cast<const VT*>(cluster.map_shared_rank(Rs + (u - owner * chunk) * LD + c, owner));
#pragma unroll
          for (int q = 0; q < V; ++q) {
            const T e = Vec16<T>::get(v, q);
            Es[(c + q) * LD + u] = rescale ? mul_pow2<T>(e, -gexp) : e;
          }
        }
        __syncthreads();
      }  // pull exchange
    }

  };
  for (int j = 0; j < n_pipe; ++j) {
    if (p.ckpt != nullptr && j % p.ckpt_stride == 0 && j / p.ckpt_stride < p.ckpt_n) {
      // checkpoint: the environment before mode j (read before this mode's
      // products; nothing writes Es until its exchange).  Every CTA holds
      // all of E: each stores a 1/C share, so no CTA lags the exchange.
      const int g = j / p.ckpt_stride;
      const int rxk = j == 0 ? p.rx0 : sst[j - 1].rout_x, ryk = j == 0 ? p.ry0 : sst[j - 1].rout_y;
      T* dst = static_cast<T*>(p.ckpt) + g * p.ckpt_elems;
      for (int idx = crank * NT + tid; idx < rxk * ryk; idx += NT * C) {
        const int u = idx / ryk, v = idx - u * ryk;
        dst[idx] = Es[v * LD + u];
      }
      if (tid == 0 && crank == 0) p.ckpt_log2[g] = log2s;
    }
    const SweepStep& sj = sst[j];
    const int need1 = ((sj.rin_x + 3) >> 2) * ((sj.rout_y + 3) >> 2);
    const int need2 = ((sj.rout_x + 3) >> 2) * ((sj.rout_y + 3) >> 2);
    if (Cfg::NS > 1 && need1 <= NT && need2 <= NT) mode(j, std::integral_constant<int, 1>{});
    else mode(j, std::integral_constant<int, Cfg::NS>{});
  }

  // ---- last mode of a full contraction: float64 sum ----
  if (p.final_scalar) {
    const SweepStep st = p.step[p.n_steps - 1];
    const T* gx = static_cast<const T*>(st.gx);
    const T* gy = static_cast<const T*>(st.gy);
    const int I = st.I;
    T* bvec = Ts;       // B_i[q][0]
    T* avec = Ts + LD;  // A_i[p][0]
    double part = 0.0;
    for (int i = crank; i < I; i += C) {
      for (int q = tid; q < st.rin_y; q += NT)
        bvec[q] = p.transposed_y ? ldg(gy + static_cast<int64_t>(i) * st.rin_y + q)
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
    double* dred = reinterpret_cast<double*>(ired + 128);  // 32 doubles: per-warp sums, total in [16]
    if (lane == 0) dred[warp] = part;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < NW; ++w) s += dred[w];
      dred[16] = s;
    }
    double z = 0.0;
    if constexpr (CL) {
      cg::cluster_group cluster = cg::this_cluster();
      cluster.sync();
      if (crank == 0 && tid == 0)
        for (int r = 0; r < C; ++r) z += *cluster.map_shared_rank(dred + 16, r);
    } else {
      __syncthreads();
      z = dred[16];
    }
    if (crank == 0 && tid == 0) {
      int st_bits = (isfinite(z) && !bad) ? 0 : TT_STATUS_NONFINITE;
      if (o.z_out_log2 != nullptr) {
        *o.z_out = z;
        *o.z_out_log2 = log2s;
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
        *o.z_out = v;
      }
      set_status(o.status, st_bits);
    }
    if constexpr (CL) cg::this_cluster().sync();  // peers' shared memory stays alive until CTA 0 has read it
    return false;
  }
  out.log2s = log2s;
  out.bad = bad;
  return true;
}

// Environment output and chain emission after a sweep (see EmitParams).
template <typename T, int RM, bool CL>
__device__ __forceinline__ void sweep_tail(const SweepParams& p, const SweepOut& o, unsigned char* smem, int C,
                                           int crank, const SweepState<T, RM, CL>& s) {
  using Cfg = SweepCfg<T, RM, CL>;
  constexpr int NT = Cfg::NT, LD = Cfg::LD;
  T* Es = reinterpret_cast<T*>(smem);
  T* Ts = Es + Cfg::TILE;
  T* stage0 = Ts + Cfg::TILE + Cfg::RS_ROWS * LD;
  const int tid = threadIdx.x;
  const int64_t log2s = s.log2s;

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
    const bool pre = emit_prefetched<Cfg::KC>(p, crank);
    int ebits = 0;
    constexpr int NS = Cfg::NS;
    for (int i = crank; i < em.I; i += C) {
      T acc[NS][4][4];
#pragma unroll
      for (int u = 0; u < NS; ++u)
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[u][a][b] = T(0);
      for (int r0 = 0; r0 < kx; r0 += Cfg::KC) {
        const int kc = min(Cfg::KC, kx - r0);
        __syncthreads();
        if (!(pre && i == crank)) {  // else the sweep's last mode already issued this load
          if (em.lead) load_rows_async<T, LD, NT>(stage0, gx, i, em.I, em.ra, em.rb, 0, r0, kc);
          else load_rows_async<T, LD, NT>(stage0, gx, i, em.I, em.rb, em.ra, 1, r0, kc);
          cp_async_commit();
        }
        cp_async_wait<0>();
        __syncthreads();
#pragma unroll
        for (int u = 0; u < NS; ++u) {
          const Sub sb = sub_tile<NT>(u, nu, em.ry);
          if (sb.on) outer_product<T, 4, LD>(acc[u], stage0, Ts + r0 * LD, kc, sb.m0, sb.n0);
        }
      }
#pragma unroll
      for (int u = 0; u < NS; ++u) {
        const Sub sb = sub_tile<NT>(u, nu, em.ry);
        if (!sb.on) continue;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int uu = sb.m0 + a, y = sb.n0 + b;
            if (uu < nu && y < em.ry) {
              T v = acc[u][a][b];
              if (fold) {
                const T v0 = v;
                v = scale_pow2_sat<T>(v, log2s);
                if (isfinite(v0) && !isfinite(v)) ebits |= TT_STATUS_OVERFLOW;
              }
              if (!isfinite(v)) ebits |= TT_STATUS_NONFINITE;
              cout[(static_cast<int64_t>(uu) * em.I + i) * em.ry + y] = v;
            }
          }
      }
    }
    if (ebits) set_status(o.status, ebits);
    if (crank == 0 && tid == 0 && em.z_log2_out != nullptr) *em.z_log2_out = log2s;
    // free cores: plain copies grid-stride over the cluster, leg-swapped ones
    // through shared-memory tiles
    const int64_t g = static_cast<int64_t>(crank) * NT + tid, gs = static_cast<int64_t>(C) * NT;
    for (int t = 0; t < (o.skip_copies ? 0 : em.n_copies); ++t) {
      const CopyTask& tk = em.copy[t];
      const T* __restrict__ src = static_cast<const T*>(tk.src);
      T* __restrict__ dst = static_cast<T*>(tk.dst);
      if (!tk.swap) {
        copy_plain<T>(dst, src, static_cast<int64_t>(tk.r0) * tk.I * tk.r1, g, gs);
      } else {
        copy_swap_tiled<T, NT>(dst, src, tk.r0, tk.I, tk.r1, stage0, C, crank);
      }
    }
  }
  if (tid == 0 && crank == 0 && s.bad) set_status(o.status, TT_STATUS_NONFINITE);
}

}  // namespace ttc
