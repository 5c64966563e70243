// Per-CTA environment sweep of one contraction, the body of the batched
// persistent launch (batched.cu).
//
// A contracted mode folds its core pair into the running environment
// (Algorithm 2 step 4 / Example 1's K = A_x^T A_y, generalised to many modes):
//   E'[u][v] = sum_i (A_i^T E B_i)[u][v],
// A_i, B_i the i-th slices of the two cores (SweepStep).  The engine evaluates
// it as two products, in whichever order is cheaper for the mode's ranks
// (the host picks `ord`):
//   ord 0:  T_i = E B_i,        E'  += A_i^T T_i
//   ord 1:  T_i = E^T A_i,      E'^T += B_i^T T_i
// Both are one code path: GEMM1  T_j[m][n] = sum_k Ein[m][k] F_j[k][n]  and
// GEMM2  P[u][n] += sum_m S_j[m][u] T_j[m][n], with (Ein, F, S) = (E, B, A) or
// (E^T, A, B).
//
// Ragged ranks leave most threads of a one-slice product idle, so g slices
// form a panel: GEMM1 of a panel is one product with g*n columns (the slices
// of a core row are contiguous in memory), and GEMM2 splits the panel's slices
// over `rep` replica groups of threads, each with its own partial P, summed
// when the mode ends.  Each product deals 4x4 output tiles round-robin over
// the threads (one or two per thread); operands are read from shared memory
// as 16-byte vectors.
//
// Operand rows stream through a ring of NST stages filled with cp.async by
// every thread; a chunk's copies are issued right after the products of the
// chunk before it, so one warp's copy set-up overlaps the other warps'
// multiply-adds, and the loads run ahead across panel and mode boundaries
// (they do not depend on E).  Each thread owns one column of a panel and
// walks its rows, so the copy loops hold no division.  E stays in shared
// memory for the whole pair, stored in the layout the next product reads
// (k-major: Ein_s[k][m]).
//
// Scaling: after each mode the largest magnitude of E' is compared with
// 2^(+-s); outside that band E' is multiplied by an exact power of two and the
// exponent accumulated in an int64.  The last mode of a full contraction
// (right ranks 1) forms t[p][i] = sum_q E[p][q] B_i[q] in the storage type and
// sums z = sum_{p,i} A_i[p] t[p][i] in float64.  A partial contraction ends
// with the chain emission C = A_i^T K of Algorithm 2 steps 5-6, streamed like
// a GEMM2 with K in place of T.
#pragma once

#include "sweep_body.cuh"
#include "ttc_device.cuh"
#include "ttc_internal.h"

namespace ttc {
namespace eng {

constexpr int NT = kEngThreads;  // threads of the CTA
constexpr int NW = NT / 32;
constexpr int NTOT = NT;
constexpr int NST = 4;  // pipeline stages
constexpr int kNoExpE = -(1 << 30);

template <typename T>
struct Smem {
  using L = EngLimits<T>;
  static constexpr size_t EIN = static_cast<size_t>(L::RM) * L::LDE * sizeof(T);
  static constexpr size_t TB = static_cast<size_t>(L::TBUF) * sizeof(T);
  static constexpr size_t ST = static_cast<size_t>(NST) * L::STAGE * sizeof(T);
};

// Thread tilings of a product: one or two 4x4 tiles per thread.
enum { kTile4x1 = 0, kTile4x2 = 1 };

// One phase of the pipeline: a contracted mode (kind 0), the last mode of a
// full contraction (kind 1) or the chain emission (kind 2).
struct Geo {
  const void* F;  // GEMM1 right operand core (kind 0, 1)
  const void* S;  // GEMM2 left operand core (kind 0, 2; kind 1: A of the float64 sum)
  int kind, ord;
  int I, g;        // slices and slices per panel
  int m, k, n, u;  // product sizes (see the file comment)
  int n_pad, u_pad;
  int ftrans, strans;  // 1: the core is stored [cols][I][rows] (right-to-left sweep)
  int kcF, kcS;        // rows per chunk (powers of two)
  int LWF, LWS;        // stage row strides
  int nchF, nchS;      // chunks per panel
  int rep;             // GEMM2 replica groups
  int tile;            // kTile*
};

constexpr size_t kGeoBytes = ((sizeof(Geo) * (kMaxOrder + 1)) + 15) / 16 * 16;
constexpr size_t kRedBytes = 64 * sizeof(double);

__host__ __device__ constexpr int r4(int v) { return (v + 3) & ~3; }
__host__ __device__ constexpr int r8(int v) { return (v + 7) & ~7; }
template <int S>
__device__ __forceinline__ int rpad(int v) {
  return (v + S - 1) / S * S;
}
__device__ __forceinline__ int pow2_floor_d(int v) { return v <= 1 ? 1 : (1 << (31 - __clz(v))); }

// acc[a][b] += sum_{r<K} A[r*lda + a] * B[r*ldb + b]
template <typename T, int SM, int SN>
__device__ __forceinline__ void opk(T (&acc)[SM][SN], const T* __restrict__ A, int lda, const T* __restrict__ B,
                                    int ldb, int K) {
#pragma unroll(SM == 8 ? 2 : 4)
  for (int r = 0; r < K; ++r) {
    T av[SM], bv[SN];
    ld_vec<T, SM>(av, A + r * lda);
    ld_vec<T, SN>(bv, B + r * ldb);
#pragma unroll
    for (int a = 0; a < SM; ++a)
#pragma unroll
      for (int b = 0; b < SN; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
  }
}

template <typename T, int SM, int SN>
__device__ __forceinline__ void zero_acc(T (&acc)[SM][SN]) {
#pragma unroll
  for (int a = 0; a < SM; ++a)
#pragma unroll
    for (int b = 0; b < SN; ++b) acc[a][b] = T(0);
}

// Row-major SM x SN tile of acc into dst (row stride ld), 16-byte stores.
template <typename T, int SM, int SN>
__device__ __forceinline__ void store_tile(T* __restrict__ dst, int ld, const T (&acc)[SM][SN]) {
  constexpr int V = 16 / sizeof(T);
#pragma unroll
  for (int a = 0; a < SM; ++a)
#pragma unroll
    for (int b = 0; b < SN; b += V) {
      if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(dst + a * ld + b) = make_float4(acc[a][b], acc[a][b + 1], acc[a][b + 2], acc[a][b + 3]);
      } else {
        *reinterpret_cast<double2*>(dst + a * ld + b) = make_double2(acc[a][b], acc[a][b + 1]);
      }
    }
}

// Tile t of a rows x cols output covered by SM x SN tiles.  Tiles are taken
// in strips 8 tiles wide (row by row inside a strip, the last strip narrower),
// so the 32 tiles of a warp form a 4 x 8 block wherever the output allows: a
// k-step then reads 4 distinct A vectors and 8 distinct B vectors (two
// shared-memory wavefronts) instead of one row of 32 B vectors.  No tile is
// padding.
struct Sub {
  int r0, c0;
  bool on;
};
template <int SM, int SN>
__device__ __forceinline__ Sub sub_at(int t, int rows, int cols) {
  const int nrb = rpad<SM>(rows) / SM, ncb = rpad<SN>(cols) / SN;
  const int nfull = ncb >> 3;              // strips of 8 tile columns
  const int in_full = nfull * nrb * 8;     // tiles in full strips
  Sub s;
  s.on = t < nrb * ncb;
  int rb, cb;
  if (t < in_full) {
    const int q = udiv16(t, nrb * 8), rem = t - q * nrb * 8;
    rb = rem >> 3;
    cb = q * 8 + (rem & 7);
  } else {
    const int wl = max(1, ncb - nfull * 8), rem = t - in_full;  // last, narrower strip
    rb = udiv16(rem, wl);
    cb = nfull * 8 + rem - rb * wl;
  }
  s.r0 = rb * SM;
  s.c0 = cb * SN;
  return s;
}

// Copy rows [r0, r0 + kcur) of slices [i0, i0 + gc) of a core into a stage:
// dst[r * LW + j * ncol_pad + c] = slice (i0 + j), row (r0 + r), column c.
//   trans == 0: core [rows][I][ncol];  trans == 1: core [ncol][I][rows].
// kc (a power of two <= 32) is the chunk capacity; kcur <= kc rows are valid.
// A loaded element feeds only m (or n) multiply-adds, so the copy loops are
// kept to a few instructions per element: each thread owns one column of the
// panel (consecutive threads, consecutive addresses) and walks rows by
// pointer increments; the index splits happen once per chunk.
template <typename T>
__device__ __forceinline__ void load_chunk(T* __restrict__ dst, int LW, const T* __restrict__ core, int I, int rows,
                                           int ncol, int ncol_pad, int trans, int r0, int kc, int kcur, int i0,
                                           int gc) {
  constexpr int V = 16 / sizeof(T);
  const int tid = threadIdx.x;
  if (!trans) {
    const int64_t gstride = static_cast<int64_t>(I) * ncol;  // one core row
    const T* src0 = core + (static_cast<int64_t>(r0) * I + i0) * ncol;
    const bool vec = ncol == ncol_pad && (ncol % V) == 0 && (reinterpret_cast<uintptr_t>(core) & 15) == 0;
    const int unit = vec ? V : 1;
    const int w = gc * ncol / unit;  // columns of the panel, in copy units (<= NT)
    const int rstep = udiv16(NT, w);
    const int rt = udiv16(tid, w);
    if (rt >= min(rstep, kcur)) return;
    const int col = (tid - rt * w) * unit;  // element column within the panel row
    const int j = udiv16(col, ncol), c = col - j * ncol;
    T* d = dst + rt * LW + j * ncol_pad + c;
    const T* g = src0 + rt * gstride + col;
    const int dstep = rstep * LW;
    const int64_t gstep = rstep * gstride;
    if (vec) {
      for (int r = rt; r < kcur; r += rstep, d += dstep, g += gstep) cp_async16(d, g);
    } else {
      for (int r = rt; r < kcur; r += rstep, d += dstep, g += gstep) cp_async_elem(d, g);
    }
  } else {
    // kc contiguous source elements per (slice, column): lanes take kc rows of 32/kc columns
    const int lk = 31 - __clz(kc);
    const int lane = tid & 31, warp = tid >> 5;
    const int sub = lane >> lk, r = lane & (kc - 1);
    const int cstep = NW * (32 >> lk);
    const int ncolumns = gc * ncol;
    if (r >= kcur) return;
    int cb = warp * (32 >> lk) + sub;
    int j = udiv16(cb, ncol), c = cb - j * ncol;
    const T* g0 = core + static_cast<int64_t>(i0) * rows + r0 + r;
    T* d0 = dst + r * LW;
    const int64_t crow = static_cast<int64_t>(I) * rows;  // one source column
    for (; cb < ncolumns; cb += cstep) {
      cp_async_elem(d0 + j * ncol_pad + c, g0 + c * crow + static_cast<int64_t>(j) * rows);
      if (cstep < ncol) {  // at most one wrap per step
        c += cstep;
        if (c >= ncol) {
          c -= ncol;
          ++j;
        }
      } else {
        j = udiv16(cb + cstep, ncol);
        c = cb + cstep - j * ncol;
      }
    }
  }
}

// Position in the stream of chunks: phase gi, panel starting at slice i0,
// operand which (0 = F, 1 = S), chunk c.
struct It {
  int gi, i0, which, c;
  bool valid;
};

__device__ __forceinline__ void settle(It& it, const Geo* geo, int ng) {
  for (;;) {
    if (it.gi >= ng) {
      it.valid = false;
      return;
    }
    const Geo& G = geo[it.gi];
    if (it.i0 >= G.I) {
      ++it.gi;
      it.i0 = 0;
      it.which = 0;
      it.c = 0;
      continue;
    }
    const int nch = it.which == 0 ? G.nchF : G.nchS;
    if (it.c < nch) {
      it.valid = true;
      return;
    }
    it.c = 0;
    if (it.which == 0) {
      it.which = 1;
      continue;
    }
    it.which = 0;
    it.i0 += G.g;
  }
}

// Layout of E in Ein_s that phase G reads: 0 -> Ein_s[y][x] (E^T rows),
// 1 -> Ein_s[x][y] (E rows).  ord 0 reads Ein = E (k = y index), ord 1 reads
// Ein = E^T (k = x index); the float64 last mode uses ord 0, the emission K rows.
__device__ __forceinline__ int layout_of(const Geo& G) { return G.kind == 0 ? G.ord : (G.kind == 1 ? 0 : 1); }

template <typename T>
constexpr size_t smem_bytes() {
  return Smem<T>::EIN + Smem<T>::TB + Smem<T>::ST + kGeoBytes + kRedBytes;
}

// Barrier of the CTA's threads (all of them compute and copy).
__device__ __forceinline__ void cbar() { __syncthreads(); }

// The chunk ring: produce() issues the next chunk's copies (one commit group
// per call, empty when the schedule is done); next() waits for the oldest
// outstanding chunk and returns its stage; release() refills the ring.
template <typename T>
struct Pipe {
  T* st0;
  const Geo* geo;
  int ng;
  It prod;
  int Lp, Lc;

  __device__ __forceinline__ void produce() {
    if (prod.valid) {
      using L = EngLimits<T>;
      const Geo& G = geo[prod.gi];
      T* dst = st0 + (Lp % NST) * L::STAGE;
      const int gc = min(G.g, G.I - prod.i0);
      if (prod.which == 0) {
        const int r0 = prod.c * G.kcF;
        load_chunk<T>(dst, G.LWF, static_cast<const T*>(G.F), G.I, G.k, G.n, G.n_pad, G.ftrans, r0, G.kcF,
                      min(G.kcF, G.k - r0), prod.i0, gc);
      } else {
        const int r0 = prod.c * G.kcS;
        load_chunk<T>(dst, G.LWS, static_cast<const T*>(G.S), G.I, G.m, G.u, G.u_pad, G.strans, r0, G.kcS,
                      min(G.kcS, G.m - r0), prod.i0, gc);
      }
      ++Lp;
      ++prod.c;
      settle(prod, geo, ng);
    }
    cp_async_commit();
  }
  // Wait for the next chunk and return its stage.  The barrier also frees
  // the stage of the chunk consumed before it, which release() reuses.
  __device__ __forceinline__ const T* next() {
    cp_async_wait<NST - 2>();
    __syncthreads();
    const T* b = st0 + (Lc % NST) * EngLimits<T>::STAGE;
    ++Lc;
    return b;
  }
  __device__ __forceinline__ void release() { produce(); }
};

// Block-wide max of e and or of b; every thread gets the result.
__device__ __forceinline__ void block_max_or(int& e, int& b, int* red) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  e = __reduce_max_sync(0xffffffffu, e);
  b = __reduce_or_sync(0xffffffffu, b);
  cbar();  // red may still be read from the previous use
  if (lane == 0) {
    red[warp] = e;
    red[32 + warp] = b;
  }
  cbar();
  e = kNoExpE;
  b = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    e = max(e, red[w]);
    b |= red[32 + w];
  }
}

__device__ __forceinline__ double block_sum_d(double v, double* red) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  v = warp_sum(v);
  cbar();
  if (lane == 0) red[warp] = v;
  cbar();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < NW; ++w) s += red[w];
  return s;
}

// The whole sweep of one pair; every thread of the CTA (compute warps and
// the producer warp) calls it.
template <typename T>
__device__ void run_pair(const SweepParams& p, const SweepOut& o, unsigned char* smem) {
  using L = EngLimits<T>;
  constexpr int LDE = L::LDE;
  T* Ein = reinterpret_cast<T*>(smem);
  T* Tb = reinterpret_cast<T*>(smem + Smem<T>::EIN);
  T* st0 = reinterpret_cast<T*>(smem + Smem<T>::EIN + Smem<T>::TB);
  Geo* geo = reinterpret_cast<Geo*>(smem + Smem<T>::EIN + Smem<T>::TB + Smem<T>::ST);
  double* redd = reinterpret_cast<double*>(smem + Smem<T>::EIN + Smem<T>::TB + Smem<T>::ST + kGeoBytes);
  int* redi = reinterpret_cast<int*>(redd);
  const int tid = threadIdx.x;

  // ---- phases ----
  const int n_modes = p.final_scalar ? p.n_steps - 1 : p.n_steps;
  const int ng = n_modes + (p.final_scalar ? 1 : 0) + (p.emit.enabled ? 1 : 0);
  for (int q = tid; q < ng; q += NTOT) {
    Geo G;
    G.rep = 1;
    G.tile = kTile4x1;
    if (q < n_modes) {
      const SweepStep& st = p.step[q];
      G.kind = 0;
      G.ord = st.ord;
      G.I = st.I;
      if (st.ord == 0) {
        G.F = st.gy;
        G.S = st.gx;
        G.m = st.rin_x;
        G.k = st.rin_y;
        G.n = st.rout_y;
        G.u = st.rout_x;
      } else {
        G.F = st.gx;
        G.S = st.gy;
        G.m = st.rin_y;
        G.k = st.rin_x;
        G.n = st.rout_x;
        G.u = st.rout_y;
      }
      G.ftrans = G.strans = p.transposed;
      // the planner's g, held within the stage width and the T panel
      // (r8(m) * r8(g n_pad) <= TILES)
      const int n4 = r4(G.n), u4 = r4(G.u);
      const int gw = max(1, L::WMAX / max(n4, u4));
      const int gt = max(1, ((L::TILES / r8(G.m)) & ~7) / n4);
      G.g = max(1, min(min(st.g, G.I), min(gw, gt)));
      const int tiles1 = (r4(G.m) / 4) * (r4(G.g * n4) / 4);
      const int tiles2 = (u4 / 4) * (n4 / 4);
      int rep = min(G.g, NT / 32);  // replica groups of whole warps
      rep = min(rep, max(1, NT / tiles2));
      rep = min(rep, max(1, L::TBUF / (r8(G.u) * r8(G.n))));
      if (st.rcap > 0) rep = min(rep, st.rcap);  // autotuned cap
      G.rep = pow2_floor_d(rep);
      const int ntr = NT / G.rep;
      // tiles1 <= r8(m) r8(W) / 16 <= 2 NT and tiles2 <= 2 NT / rep by the limits above
      G.tile = (tiles1 <= NT && tiles2 <= ntr) || sizeof(T) == 8 ? kTile4x1 : kTile4x2;
    } else if (p.final_scalar && q == n_modes) {
      // t[p][i] = sum_q E[p][q] Gy[q][i] (Gy read as a [k][I][1] core with
      // its slices side by side), z = sum A[p][i] t[p][i]
      const SweepStep& st = p.step[p.n_steps - 1];
      G.kind = 1;
      G.ord = 0;
      G.I = st.I;
      G.F = st.gy;
      G.S = st.gx;
      G.m = st.rin_x;
      G.k = st.rin_y;
      G.n = 1;
      G.u = 1;
      G.ftrans = G.strans = 0;
      // one 4x4 tile per thread (r4(m) * g <= 16 NT) and a T panel within
      // the buffer; g a multiple of 4 unless it is I itself
      G.g = max(1, min(G.I, min(min(((16 * NT) / r4(G.m)) & ~3, (L::TBUF / r4(G.m)) & ~3), L::WMAX)));
    } else {
      const EmitParams& em = p.emit;
      G.kind = 2;
      G.ord = 1;
      G.I = em.I;
      G.F = nullptr;
      G.S = em.gx;
      // lead: A_i[a][u] = gx[a][i][u] (rows ra); trail: A_i[b][u] = gx[u][i][b] (rows rb)
      G.m = em.lead ? em.ra : em.rb;
      G.u = em.lead ? em.rb : em.ra;
      G.k = 0;
      G.n = em.ry;
      G.ftrans = 0;
      G.strans = em.lead ? 0 : 1;
      const int tilesE = (r4(G.u) / 4) * (r4(G.n) / 4);  // <= 2 NT
      constexpr int kSub = sizeof(T) == 4 ? 2 : 1;
      G.g = max(1, min(G.I, min((kSub * NT) / tilesE, L::WMAX / r4(G.u))));
      G.tile = G.g * tilesE <= NT ? kTile4x1 : kTile4x2;
    }
    G.n_pad = G.kind == 1 ? 1 : r4(G.n);
    G.u_pad = r4(G.u);
    G.LWF = r4(G.g * G.n_pad) + L::V;
    G.LWS = G.g * G.u_pad + L::V;
    G.kcF = pow2_floor_d(min(32, L::STAGE / G.LWF));
    G.kcS = pow2_floor_d(min(32, L::STAGE / G.LWS));
    G.nchF = G.kind == 2 ? 0 : (G.k + G.kcF - 1) / G.kcF;
    G.nchS = G.kind == 1 ? 0 : (G.m + G.kcS - 1) / G.kcS;
    geo[q] = G;
  }
  __syncthreads();  // the phase table is complete

  // ---- start environment: [1] (either layout) ----
  int64_t log2s = 0;
  int bad = 0;
  if (tid == 0) Ein[0] = T(1);

  Pipe<T> pipe;
  pipe.st0 = st0;
  pipe.geo = geo;
  pipe.ng = ng;
  pipe.prod = It{0, 0, 0, 0, false};
  settle(pipe.prod, geo, ng);
  pipe.Lp = 0;
  pipe.Lc = 0;
#pragma unroll
  for (int s = 0; s < NST - 1; ++s) pipe.produce();

  // ---- one contracted mode: NS tiles of SM x SM per thread ----
  auto mode = [&](const Geo& G, const int next_layout, auto sm_tag, auto ns_tag) {
    constexpr int SM = decltype(sm_tag)::value, SN = SM;
    constexpr int NS = decltype(ns_tag)::value;
    const int lgr = 31 - __clz(NT / G.rep);  // threads per replica group = 2^lgr
    const int rid = tid >> lgr, lt = tid - (rid << lgr);
    Sub s2[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) s2[s] = sub_at<SM, SN>(lt + (s << lgr), G.u, G.n);
    T acc2[NS][SM][SN];
#pragma unroll
    for (int s = 0; s < NS; ++s) zero_acc(acc2[s]);

    for (int i0 = 0; i0 < G.I; i0 += G.g) {
      const int gc = min(G.g, G.I - i0);
      const int W = gc * G.n_pad;  // T panel columns
      const int LT = r8(W);        // T panel row stride
      Sub s1[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) s1[s] = sub_at<SM, SN>(tid + s * NT, G.m, W);
      // GEMM1: T[m][c] = sum_k Ein_s[k][m] F[k][c]
      T acc1[NS][SM][SN];
#pragma unroll
      for (int s = 0; s < NS; ++s) zero_acc(acc1[s]);
      for (int c = 0; c < G.nchF; ++c) {
        const T* Fs = pipe.next();
        const int k0 = c * G.kcF, kcur = min(G.kcF, G.k - k0);
#pragma unroll
        for (int s = 0; s < NS; ++s)
          if (s1[s].on) opk<T, SM, SN>(acc1[s], Ein + k0 * LDE + s1[s].r0, LDE, Fs + s1[s].c0, G.LWF, kcur);
        pipe.release();
      }
      cbar();  // every thread is done reading T (previous panel)
#pragma unroll
      for (int s = 0; s < NS; ++s)
        if (s1[s].on) store_tile(Tb + s1[s].r0 * LT + s1[s].c0, LT, acc1[s]);
      cbar();  // T complete
      // GEMM2: P[u][n] += sum_m S_j[m][u] T_j[m][n] over this replica's slices
      for (int c = 0; c < G.nchS; ++c) {
        const T* Ss = pipe.next();
        const int r0 = c * G.kcS, kcur = min(G.kcS, G.m - r0);
        for (int j = rid; j < gc; j += G.rep) {
#pragma unroll
          for (int s = 0; s < NS; ++s)
            if (s2[s].on)
              opk<T, SM, SN>(acc2[s], Ss + j * G.u_pad + s2[s].r0, G.LWS, Tb + r0 * LT + j * G.n_pad + s2[s].c0, LT,
                             kcur);
        }
        pipe.release();
      }
    }
    // ---- replica partials -> E' in the layout the next phase reads ----
    cbar();  // T and Ein are no longer read
    const int NP8 = r8(G.n), UN = r8(G.u) * NP8;
#pragma unroll
    for (int s = 0; s < NS; ++s)
      if (s2[s].on) store_tile(Tb + rid * UN + s2[s].r0 * NP8 + s2[s].c0, NP8, acc2[s]);
    cbar();
    T lmax = T(0);
    int lbad = 0;
    const int n4 = G.n_pad / 4;
    for (int e = tid; e < G.u * n4; e += NT) {
      const int uu = udiv16(e, n4), c4 = (e - uu * n4) * 4;
      T sv[4];
      ld_vec<T, 4>(sv, Tb + uu * NP8 + c4);
      for (int r = 1; r < G.rep; ++r) {
        T t4[4];
        ld_vec<T, 4>(t4, Tb + r * UN + uu * NP8 + c4);
#pragma unroll
        for (int b = 0; b < 4; ++b) sv[b] += t4[b];
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int nn = c4 + b;
        if (nn < G.n) {
          const T v = sv[b];
          if (isfinite(v)) lmax = fmax(lmax, fabs(v));
          else lbad = 1;
          // (x, y) index of E'
          const int x = G.ord == 0 ? uu : nn, y = G.ord == 0 ? nn : uu;
          Ein[next_layout == 0 ? y * LDE + x : x * LDE + y] = v;
        }
      }
    }
    // largest entry in [2^(e-1), 2^e): rescale when e leaves [-s, s]
    int lexp = lmax > T(0) ? exp2_bits(lmax) : kNoExpE;
    block_max_or(lexp, lbad, redi);
    if (lbad) bad = 1;
    if (lexp != kNoExpE && (lexp > p.renorm_bits || lexp < -p.renorm_bits)) {
      log2s += lexp;
      const int nx = G.ord == 0 ? G.u : G.n, ny = G.ord == 0 ? G.n : G.u;
      for (int e = tid; e < nx * ny; e += NT) {
        const int x = udiv16(e, ny), y = e - x * ny;
        T& r = Ein[next_layout == 0 ? y * LDE + x : x * LDE + y];
        r = mul_pow2<T>(r, -lexp);
      }
    }
    cbar();
  };

  // ---- last mode of a full contraction, float64 sum ----
  auto final_mode = [&](const Geo& G) {
    const T* ax = static_cast<const T*>(G.S);  // Gx_last [m][I][1]
    double part = 0.0;
    for (int i0 = 0; i0 < G.I; i0 += G.g) {
      const int gc = min(G.g, G.I - i0);
      const int W = r4(gc);
      const Sub sb = sub_at<4, 4>(tid, G.m, W);
      T acc[4][4];
      zero_acc(acc);
      for (int c = 0; c < G.nchF; ++c) {
        const T* Fs = pipe.next();
        const int k0 = c * G.kcF, kcur = min(G.kcF, G.k - k0);
        if (sb.on) opk<T, 4, 4>(acc, Ein + k0 * LDE + sb.r0, LDE, Fs + sb.c0, G.LWF, kcur);
        pipe.release();
      }
      cbar();  // every thread is done reading T (previous panel)
      if (sb.on) store_tile(Tb + sb.r0 * W + sb.c0, W, acc);
      cbar();
      for (int e = tid; e < G.m * gc; e += NT) {
        const int pp = udiv16(e, gc), j = e - pp * gc;
        part = fma(static_cast<double>(ldg(ax + static_cast<int64_t>(pp) * G.I + i0 + j)),
                   static_cast<double>(Tb[pp * W + j]), part);
      }
    }
    const double z = block_sum_d(part, redd);
    if (tid == 0) {
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
  };

  // ---- chain emission: C[u][i][y] = sum_a A_i[a][u] K[a][y] ----
  auto emission = [&](const Geo& G, auto sm_tag, auto ns_tag) {
    constexpr int SM = decltype(sm_tag)::value, SN = SM;
    constexpr int NS = decltype(ns_tag)::value;
    const EmitParams& em = p.emit;
    T* cout = static_cast<T*>(em.c_out);
    const bool fold = em.z_log2_out == nullptr && log2s != 0;
    const int tilesE = (rpad<SM>(G.u) / SM) * (rpad<SN>(G.n) / SN);
    int ebits = 0;
    for (int i0 = 0; i0 < G.I; i0 += G.g) {
      const int gc = min(G.g, G.I - i0);
      int js[NS];
      Sub sb[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        const int t = tid + s * NT;
        js[s] = udiv16(t, tilesE);
        sb[s] = sub_at<SM, SN>(t - js[s] * tilesE, G.u, G.n);
        sb[s].on = t < gc * tilesE;
      }
      T acc[NS][SM][SN];
#pragma unroll
      for (int s = 0; s < NS; ++s) zero_acc(acc[s]);
      for (int c = 0; c < G.nchS; ++c) {
        const T* Ss = pipe.next();
        const int r0 = c * G.kcS, kcur = min(G.kcS, G.m - r0);
#pragma unroll
        for (int s = 0; s < NS; ++s)
          if (sb[s].on)
            opk<T, SM, SN>(acc[s], Ss + js[s] * G.u_pad + sb[s].r0, G.LWS, Ein + r0 * LDE + sb[s].c0, LDE, kcur);
        pipe.release();
      }
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        if (!sb[s].on) continue;
        const int i = i0 + js[s];
#pragma unroll
        for (int a = 0; a < SM; ++a)
#pragma unroll
          for (int b = 0; b < SN; ++b) {
            const int uu = sb[s].r0 + a, y = sb[s].c0 + b;
            if (uu < G.u && y < G.n) {
              T v = acc[s][a][b];
              if (fold) {
                const T v0 = v;
                v = scale_pow2_sat<T>(v, log2s);
                if (isfinite(v0) && !isfinite(v)) ebits |= TT_STATUS_OVERFLOW;
              }
              if (!isfinite(v)) ebits |= TT_STATUS_NONFINITE;
              cout[(static_cast<int64_t>(uu) * G.I + i) * G.n + y] = v;
            }
          }
      }
    }
    if (ebits) set_status(o.status, ebits);
    if (tid == 0 && em.z_log2_out != nullptr) *em.z_log2_out = log2s;
  };

  using I1 = std::integral_constant<int, 1>;
  using I2 = std::integral_constant<int, 2>;
  using I4 = std::integral_constant<int, 4>;
  cbar();  // start environment written
  for (int gi = 0; gi < ng; ++gi) {
    const Geo G = geo[gi];
    if (G.kind == 0) {
      const int nl = gi + 1 < ng ? layout_of(geo[gi + 1]) : 1;
      if (sizeof(T) == 8 || G.tile == kTile4x1) mode(G, nl, I4{}, I1{});
      else if constexpr (sizeof(T) == 4) mode(G, nl, I4{}, I2{});
    } else if (G.kind == 1) {
      final_mode(G);
    } else {
      if (sizeof(T) == 8 || G.tile == kTile4x1) emission(G, I4{}, I1{});
      else if constexpr (sizeof(T) == 4) emission(G, I4{}, I2{});
    }
  }
  cp_async_wait<0>();
  if (tid == 0 && bad && !p.final_scalar) set_status(o.status, TT_STATUS_NONFINITE);
  __syncthreads();  // the next pair reuses shared memory
}

}  // namespace eng
}  // namespace ttc
