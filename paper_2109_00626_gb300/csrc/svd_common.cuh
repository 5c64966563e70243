// One-sided Jacobi SVD of a small matrix by one CTA of 1024 threads
// (Hestenes 1958), shared by the TT decomposition of a dense tensor and the
// rounding of a TT.  The p = min(rows, columns) vectors of the shorter side
// are made mutually orthogonal by plane rotations, swept in the round-robin
// order of the circle method (p / 2 disjoint pairs per round, a warp per
// pair), each rotation also applied to an accumulated orthogonal p x p
// matrix; their norms are the singular values.  svd_factor() then keeps the
// rank that the TT-SVD's truncation rule gives and writes the two factors.
//
// The kernels run as a cluster of CTAs.  CTA 0 (the leader) does everything
// but the sweeps; the sweeps run in one of these places: in the leader's
// shared memory when the vectors and the rotations fit there; else, for many
// vectors of moderate length, with the vectors themselves spread over the
// cluster (jacobi_rowdist below); else spread over the cluster by columns
// when every CTA's slice fits (each CTA holds
// columns [c0, c1) of every vector and of the rotations, computes its part of
// each pair's three inner products, the pair's owner sums them and sends the
// rotation to every CTA, which applies it to its slice: two cluster barriers
// per round, exchanges through distributed shared memory); else the same
// in place in the workspace (L2), or by a leader without a cluster alone.
#pragma once

#include <cooperative_groups.h>
#include <math.h>
#include <stdint.h>

#include "tc_common.cuh"
#include "ttc_internal.h"

namespace ttc {

constexpr int kSvdThreads = 1024;
constexpr int kSvdWarps = kSvdThreads / 32;
constexpr int kSvdMaxP = 512;       // the shorter side of an unfolding
constexpr int kSvdMaxSweeps = 40;   // a bound on the Jacobi sweeps of one SVD
constexpr size_t kSvdSmemCap = 200 * 1024;  // shared memory for the sweeps of an SVD that fits

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block (every thread gets it).
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum_t(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < kSvdWarps; ++w) s += red[w];
  return s;
}

// dst (n x m) = src (m x n)^T through 32 x 33 shared-memory tiles.
template <typename T>
__device__ void transpose_rows(T* __restrict__ dst, const T* __restrict__ src, int m, int n, T* tile) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int b0 = 0; b0 < m; b0 += 32)
    for (int b1 = 0; b1 < n; b1 += 32) {
      const int r = b0 + ty, c = b1 + tx;
      if (r < m && c < n) tile[ty * 33 + tx] = src[static_cast<int64_t>(r) * n + c];
      __syncthreads();
      const int r2 = b1 + ty, c2 = b0 + tx;
      if (r2 < n && c2 < m) dst[static_cast<int64_t>(r2) * m + c2] = tile[tx * 33 + ty];
      __syncthreads();
    }
}

// ---- the cluster a decomposition runs on ----
//
// Every CTA runs the same sequence of barriers: the control flow of the
// sweeps depends only on values that all CTAs compute identically (the same
// sums in the same order), so the hardware cluster barrier (arrive with
// release, wait with acquire semantics at cluster scope) serves, as in the
// contraction sweeps.
struct SvdCluster {
  int C, rank;
  int32_t* status;
  int* bc;                 // the leader's broadcast block [16] (shared): problem shape and path
  unsigned long long* bcp; // the leader's broadcast pointers [4]
};

__device__ __forceinline__ void svd_barrier(const SvdCluster& cl) {
  if (cl.C > 1)
    cooperative_groups::this_cluster().sync();
  else
    __syncthreads();
}

__device__ __forceinline__ SvdCluster svd_cluster_begin(int32_t* status, int* bc, unsigned long long* bcp) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  SvdCluster cl;
  cl.C = static_cast<int>(cluster.num_blocks());
  cl.rank = static_cast<int>(cluster.block_rank());
  cl.status = status;
  cl.bc = bc;
  cl.bcp = bcp;
  cluster.sync();  // every CTA's shared memory exists before a peer maps it
  return cl;
}

// A flag of the leader's, read by every CTA (after a barrier that follows
// the leader's write).
__device__ __forceinline__ int svd_leader_flag(const SvdCluster& cl, int slot) {
  namespace cg = cooperative_groups;
  return cl.C > 1 ? *cg::this_cluster().map_shared_rank(cl.bc + slot, 0) : cl.bc[slot];
}

// Pair i of round t of the circle method over P (even) indices.
__device__ __forceinline__ void rr_pair(int P, int t, int i, int& a, int& b) {
  if (i == 0) {
    a = P - 1;
    b = t;
  } else {
    // t < P - 1 and 0 < i < P / 2: both sums lie in [0, 2 (P - 1))
    a = t + i;
    if (a >= P - 1) a -= P - 1;
    b = t - i + P - 1;
    if (b >= P - 1) b -= P - 1;
  }
}

// One-sided Jacobi on the p rows (length L) of W, rotations also applied to
// the rows of Qt (p x p).  Returns the number of sweeps taken.
template <typename T>
__device__ int jacobi_rows(T* __restrict__ W, T* __restrict__ Qt, int p, int L, int* s_rot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // a pair counts as orthogonal once |<a, b>| <= 4 u sqrt(L) |a| |b|: the
  // rounding of an L-term dot product, below which rotations only chase noise
  const T tol = T(4) * (sizeof(T) == 8 ? T(1.1102230246251565e-16) : T(5.9604645e-08)) * sqrt(T(L > 1 ? L : 1));
  const int P = (p + 1) & ~1;
  int sweep = 0;
  for (; sweep < kSvdMaxSweeps; ++sweep) {
    if (threadIdx.x == 0) *s_rot = 0;
    __syncthreads();
    for (int t = 0; t < P - 1; ++t) {
      for (int i = warp; i < P / 2; i += kSvdWarps) {
        int a, b;
        rr_pair(P, t, i, a, b);
        if (a >= p || b >= p) continue;  // the dummy index of an odd p
        T* wa = W + static_cast<int64_t>(a) * L;
        T* wb = W + static_cast<int64_t>(b) * L;
        T al = T(0), be = T(0), ga = T(0);
        for (int e = lane; e < L; e += 32) {
          const T u = wa[e], v = wb[e];
          al = fma(u, u, al);
          be = fma(v, v, be);
          ga = fma(u, v, ga);
        }
        al = warp_sum_t(al);
        be = warp_sum_t(be);
        ga = warp_sum_t(ga);
        if (ga == T(0) || al == T(0) || be == T(0) || fabs(ga) <= tol * sqrt(al) * sqrt(be)) continue;
        // rotation that zeroes the inner product of the two new rows:
        // t^2 + 2 zeta t - 1 = 0, the root of modulus <= 1
        const T zeta = (be - al) / (T(2) * ga);
        const T tn = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
        const T c = T(1) / sqrt(T(1) + tn * tn), s = c * tn;
        for (int e = lane; e < L; e += 32) {
          const T u = wa[e], v = wb[e];
          wa[e] = c * u - s * v;
          wb[e] = s * u + c * v;
        }
        T* qa = Qt + static_cast<int64_t>(a) * p;
        T* qb = Qt + static_cast<int64_t>(b) * p;
        for (int e = lane; e < p; e += 32) {
          const T u = qa[e], v = qb[e];
          qa[e] = c * u - s * v;
          qb[e] = s * u + c * v;
        }
        if (lane == 0) *s_rot = 1;
      }
      __syncthreads();
    }
    if (*s_rot == 0) break;
    __syncthreads();
  }
  return sweep;
}

// Shared memory of the column-distributed sweeps: each CTA's slice of the p
// vectors (ceil(L / C) columns) and of the rotations (ceil(p / C) columns)
// when they are held there, then (from a multiple of four entries, for vector
// stores) the partial inner products this CTA collects for the pairs it owns
// (four entries per pair and source CTA) and a round's rotations (c, s per
// pair).
__host__ __device__ inline size_t dist_part_offset(int p, int L, int C) {
  const int cw = (L + C - 1) / C, cq = (p + C - 1) / C;
  return (static_cast<size_t>(p) * cw + static_cast<size_t>(p) * cq + 3) & ~static_cast<size_t>(3);
}
__host__ __device__ inline size_t dist_comm_elems(int p, int C) {
  const int np = (p + 1) / 2, owned = (np + C - 1) / C;
  return static_cast<size_t>(owned) * C * 4 + 2 * static_cast<size_t>(np);
}
__host__ __device__ inline size_t dist_smem_elems(int p, int L, int C) {
  return dist_part_offset(p, L, C) + dist_comm_elems(p, C);
}

__device__ __forceinline__ void store4(float* q, float a, float b, float c) { *reinterpret_cast<float4*>(q) = make_float4(a, b, c, 0.f); }
__device__ __forceinline__ void store4(double* q, double a, double b, double c) {
  reinterpret_cast<double2*>(q)[0] = make_double2(a, b);
  q[2] = c;
}
__device__ __forceinline__ void store2(float* q, float a, float b) { *reinterpret_cast<float2*>(q) = make_float2(a, b); }
__device__ __forceinline__ void store2(double* q, double a, double b) { *reinterpret_cast<double2*>(q) = make_double2(a, b); }

// Sum over the g lanes (a power of two) of an aligned lane group; every lane
// gets it.
template <typename T>
__device__ __forceinline__ T group_sum(T v, int g) {
  for (int o = g >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One-sided Jacobi on the p rows (length L) of W with the rotations
// accumulated into Qt, spread over the cluster by columns (see above); every
// CTA of the cluster calls it.  kInSmem: each CTA copies its slices of W and
// Qt into its shared memory (dist_smem_elems) and back at the end; else it
// works on them in place in the workspace (only the exchange buffers,
// dist_comm_elems, are in shared memory).  The rotations start from the
// identity.
//
// A round takes two cluster barriers.  Each CTA forms its part of every
// pair's three inner products and stores it into the shared memory of the
// pair's owner (CTA i mod C for pair i); after the first barrier each owner
// sums the C parts of its pairs, takes the rotation (or none: c = 1, s = 0)
// and stores (c, s) into every CTA; after the second barrier every CTA
// applies the round's rotations to its slices.  All transfers are stores, one
// per pair and CTA plus one per owned pair and CTA, so no CTA waits on a
// remote load.  Single buffers suffice: a CTA can store a round's parts only
// after the previous round's second barrier, which every owner reaches after
// reading the previous parts, and its rotations only after the first barrier
// of the round, which every CTA reaches after applying the previous ones.
// A pair's parts and its rotation are handled by a group of g lanes, g the
// largest power of two <= 32 with g (p / 2) <= the block's threads.
template <typename T, bool kInSmem>
__device__ void jacobi_dist(T* W, T* Qt, int p, int L, T* dsm, const SvdCluster& cl) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int C = cl.C, rank = cl.rank;
  const int cw = (L + C - 1) / C, c0 = min(L, rank * cw), nw = min(L, c0 + cw) - c0;
  const int cq = (p + C - 1) / C, q0 = min(p, rank * cq), nq = min(p, q0 + cq) - q0;
  const int P = (p + 1) & ~1, NP = P / 2, owned = (NP + C - 1) / C;
  int g = 32;
  while (g > 1 && g * NP > static_cast<int>(blockDim.x)) g >>= 1;
  const int gl = threadIdx.x & (g - 1), grp = threadIdx.x / g, ngrp = blockDim.x / g;
  T* Ws = kInSmem ? dsm : W + c0;
  const int ldw = kInSmem ? cw : L;
  T* Qs = kInSmem ? Ws + static_cast<int64_t>(p) * cw : Qt + q0;
  const int ldq = kInSmem ? cq : p;
  T* part = kInSmem ? dsm + dist_part_offset(p, L, C) : dsm;  // [owned][C][4]
  T* rot = part + static_cast<int64_t>(owned) * C * 4;         // [NP][2]
  __shared__ int rotated;
  if (kInSmem)
    for (int64_t e = threadIdx.x; e < static_cast<int64_t>(p) * cw; e += blockDim.x) {
      const int i = static_cast<int>(e / cw), j = static_cast<int>(e - static_cast<int64_t>(i) * cw);
      Ws[e] = j < nw ? __ldcg(W + static_cast<int64_t>(i) * L + c0 + j) : T(0);
    }
  for (int64_t e = threadIdx.x; e < static_cast<int64_t>(p) * nq; e += blockDim.x) {
    const int i = static_cast<int>(e / nq), j = static_cast<int>(e - static_cast<int64_t>(i) * nq);
    Qs[static_cast<int64_t>(i) * ldq + j] = i == q0 + j ? T(1) : T(0);
  }
  const T tol = T(4) * (sizeof(T) == 8 ? T(1.1102230246251565e-16) : T(5.9604645e-08)) * sqrt(T(L > 1 ? L : 1));
  // the owners' lanes: C per owned pair (C <= 32, a power of two)
  const int oh = threadIdx.x & (C - 1), og = threadIdx.x / C, nog = blockDim.x / C;
  svd_barrier(cl);  // every CTA's buffers exist before a peer stores into them
  for (int sweep = 0; sweep < kSvdMaxSweeps; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    for (int t = 0; t < P - 1; ++t) {
      // this CTA's parts of every pair's inner products, stored at the owner
      // (the group loops run the same trip count in every lane, for the shuffles)
      for (int base = 0; base < NP; base += ngrp) {
        const int i = base + grp;
        int a = p, b = p;
        if (i < NP) rr_pair(P, t, i, a, b);
        const bool valid = a < p && b < p;
        T al = T(0), be = T(0), ga = T(0);
        if (valid) {
          const T* wa = Ws + static_cast<int64_t>(a) * ldw;
          const T* wb = Ws + static_cast<int64_t>(b) * ldw;
          for (int j = gl; j < nw; j += g) {
            const T u = kInSmem ? wa[j] : __ldcg(wa + j), v = kInSmem ? wb[j] : __ldcg(wb + j);
            al = fma(u, u, al);
            be = fma(v, v, be);
            ga = fma(u, v, ga);
          }
        }
        al = group_sum(al, g);
        be = group_sum(be, g);
        ga = group_sum(ga, g);
        if (valid && gl == 0)
          store4(cluster.map_shared_rank(part + (static_cast<int64_t>(i / C) * C + rank) * 4, i % C), al, be, ga);
      }
      svd_barrier(cl);
      // the owned pairs: sum the parts, take the rotation, store it everywhere
      for (int base = 0; base < owned; base += nog) {
        const int j = base + og, i = j * C + rank;
        int a = p, b = p;
        if (j < owned && i < NP) rr_pair(P, t, i, a, b);
        const bool valid = a < p && b < p;
        T al = T(0), be = T(0), ga = T(0);
        if (valid) {
          const T* q = part + (static_cast<int64_t>(j) * C + oh) * 4;
          al = q[0];
          be = q[1];
          ga = q[2];
        }
        al = group_sum(al, C);
        be = group_sum(be, C);
        ga = group_sum(ga, C);
        if (!valid) continue;
        T c = T(1), sn = T(0);
        if (!(ga == T(0) || al == T(0) || be == T(0) || fabs(ga) <= tol * sqrt(al) * sqrt(be))) {
          const T zeta = (be - al) / (T(2) * ga);
          const T tn = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
          c = T(1) / sqrt(T(1) + tn * tn);
          sn = c * tn;
        }
        store2(cluster.map_shared_rank(rot + static_cast<int64_t>(i) * 2, oh), c, sn);
      }
      svd_barrier(cl);
      // the round's rotations applied to this CTA's slices
      for (int i = grp; i < NP; i += ngrp) {
        int a, b;
        rr_pair(P, t, i, a, b);
        if (a >= p || b >= p) continue;
        const T c = rot[2 * i], sn = rot[2 * i + 1];
        if (sn == T(0)) continue;
        T* wa = Ws + static_cast<int64_t>(a) * ldw;
        T* wb = Ws + static_cast<int64_t>(b) * ldw;
        for (int j = gl; j < nw; j += g) {
          const T u = kInSmem ? wa[j] : __ldcg(wa + j), v = kInSmem ? wb[j] : __ldcg(wb + j);
          wa[j] = c * u - sn * v;
          wb[j] = sn * u + c * v;
        }
        T* qa = Qs + static_cast<int64_t>(a) * ldq;
        T* qb = Qs + static_cast<int64_t>(b) * ldq;
        for (int j = gl; j < nq; j += g) {
          const T u = kInSmem ? qa[j] : __ldcg(qa + j), v = kInSmem ? qb[j] : __ldcg(qb + j);
          qa[j] = c * u - sn * v;
          qb[j] = sn * u + c * v;
        }
        rotated = 1;
      }
      __syncthreads();  // the rows rotated before the next round reads them
    }
    if (rotated == 0) break;
    __syncthreads();
  }
  if (kInSmem) {
    for (int64_t e = threadIdx.x; e < static_cast<int64_t>(p) * cw; e += blockDim.x) {
      const int i = static_cast<int>(e / cw), j = static_cast<int>(e - static_cast<int64_t>(i) * cw);
      if (j < nw) W[static_cast<int64_t>(i) * L + c0 + j] = Ws[e];
    }
    for (int64_t e = threadIdx.x; e < static_cast<int64_t>(p) * cq; e += blockDim.x) {
      const int i = static_cast<int>(e / cq), j = static_cast<int>(e - static_cast<int64_t>(i) * cq);
      if (j < nq) Qt[static_cast<int64_t>(i) * p + q0 + j] = Qs[e];
    }
  }
  svd_barrier(cl);
}

// ---- row-distributed sweeps ----
//
// For many vectors of moderate length (p large, L moderate) the vectors
// themselves are spread over the cluster: CTA c holds the pair slots
// [k0, k1) of the round-robin tournament, each slot a "top" and a "bottom"
// vector (its W row followed by its Qt row, L + p entries, in shared
// memory).  A round rotates every slot's pair locally (whole dot products,
// no reduction across CTAs); then every vector but the one in top slot 0
// moves one place along the cycle top 1 -> top 2 -> ... -> top NP-1 ->
// bottom NP-1 -> ... -> bottom 0 -> top 1, so each CTA sends its last top
// vector to the next CTA and its first bottom vector to the previous one
// (distributed shared memory, receive buffers alternating by round parity)
// and renames the rest in place: one cluster barrier per round.  After the
// P - 1 rounds of a sweep every vector is back in its first place and every
// pair has met once.  Needs at least two slots per CTA (NP >= 2 C); taken
// for vectors no longer than 4 p.
__host__ __device__ inline int rowdist_slots(int NP, int C, int rank) {
  return (rank + 1) * NP / C - rank * NP / C;
}
__host__ __device__ inline size_t rowdist_smem_elems(int p, int L, int C) {
  const int NP = (p + 1) / 2;
  // long vectors with few per CTA leave most warps idle: the column split
  // serves those better (a 4096 x 64 unfolding: 12.3 vs 10.2 ms a rounding)
  if (C < 2 || NP / C < 2 || L > 4 * p) return 0;
  const int nsmax = (NP + C - 1) / C;
  return static_cast<size_t>(2 * nsmax + 4) * (static_cast<size_t>(L) + p);
}
constexpr int kRowDistMaxSlots = kSvdMaxP / 2;

template <typename T>
__device__ void jacobi_rowdist(T* W, T* Qt, int p, int L, T* dsm, const SvdCluster& cl) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int C = cl.C, rank = cl.rank;
  const int P = (p + 1) & ~1, NP = P / 2;
  const int k0 = rank * NP / C, ns = rowdist_slots(NP, C, rank);
  const int Lp = L + p;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  __shared__ int topb[kRowDistMaxSlots], botb[kRowDistMaxSlots];
  __shared__ int rflag[2];
  __shared__ T pairsum[15 * 2 * 3];  // dual mode: each pair's two halves of its three sums
  const bool dual = 2 * ns <= nwarps && ns <= 15;  // named barriers 1..15
  auto buf = [&](int b) { return dsm + static_cast<int64_t>(b) * Lp; };
  // slot s starts with vectors 2 (k0 + s) (top) and 2 (k0 + s) + 1 (bottom) in buffers 2 s, 2 s + 1
  for (int s = threadIdx.x; s < ns; s += blockDim.x) {
    topb[s] = 2 * s;
    botb[s] = 2 * s + 1;
  }
  for (int64_t e = threadIdx.x; e < static_cast<int64_t>(2 * ns) * Lp; e += blockDim.x) {
    const int b = static_cast<int>(e / Lp), j = static_cast<int>(e - static_cast<int64_t>(b) * Lp);
    const int v = 2 * k0 + b;
    T val = T(0);
    if (v < p) val = j < L ? __ldcg(W + static_cast<int64_t>(v) * L + j) : (j - L == v ? T(1) : T(0));
    dsm[e] = val;
  }
  const T tol = T(4) * (sizeof(T) == 8 ? T(1.1102230246251565e-16) : T(5.9604645e-08)) * sqrt(T(L > 1 ? L : 1));
  const int ns_next = rank + 1 < C ? rowdist_slots(NP, C, rank + 1) : 0;
  const int ns_prev = rank > 0 ? rowdist_slots(NP, C, rank - 1) : 0;
  int parity = 0;
  svd_barrier(cl);
  for (int sweep = 0; sweep < kSvdMaxSweeps; ++sweep) {
    int rotated = 0;  // thread-local: a rotation this thread's warp took
    for (int t = 0; t < P - 1; ++t) {
      // this CTA's pairs: two warps a pair when there are warps enough (their
      // halves of the dot products met through shared memory at a named
      // barrier of the pair's 64 threads), else one
      if (dual) {
        const int s = warp >> 1, half = warp & 1, gl = half * 32 + lane;
        if (s < ns) {
          T* wa = buf(topb[s]);
          T* wb = buf(botb[s]);
          T al = T(0), be = T(0), ga = T(0);
          for (int j = gl; j < L; j += 64) {
            const T u = wa[j], v = wb[j];
            al = fma(u, u, al);
            be = fma(v, v, be);
            ga = fma(u, v, ga);
          }
          al = warp_sum_t(al);
          be = warp_sum_t(be);
          ga = warp_sum_t(ga);
          T* pr = pairsum + (s * 2 + half) * 3;
          if (lane == 0) {
            pr[0] = al;
            pr[1] = be;
            pr[2] = ga;
          }
          asm volatile("bar.sync %0, 64;" ::"r"(1 + s) : "memory");
          const T* qo = pairsum + (s * 2 + (half ^ 1)) * 3;
          // the same sum in both warps: lower half first
          al = half == 0 ? al + qo[0] : qo[0] + al;
          be = half == 0 ? be + qo[1] : qo[1] + be;
          ga = half == 0 ? ga + qo[2] : qo[2] + ga;
          if (!(ga == T(0) || al == T(0) || be == T(0) || fabs(ga) <= tol * sqrt(al) * sqrt(be))) {
            const T zeta = (be - al) / (T(2) * ga);
            const T tn = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
            const T c = T(1) / sqrt(T(1) + tn * tn), sn = c * tn;
            for (int j = gl; j < Lp; j += 64) {  // the W row and the Qt row
              const T u = wa[j], v = wb[j];
              wa[j] = c * u - sn * v;
              wb[j] = sn * u + c * v;
            }
            rotated = 1;
          }
        }
      } else {
        for (int s = warp; s < ns; s += nwarps) {
          T* wa = buf(topb[s]);
          T* wb = buf(botb[s]);
          T al = T(0), be = T(0), ga = T(0);
          for (int j = lane; j < L; j += 32) {
            const T u = wa[j], v = wb[j];
            al = fma(u, u, al);
            be = fma(v, v, be);
            ga = fma(u, v, ga);
          }
          al = warp_sum_t(al);
          be = warp_sum_t(be);
          ga = warp_sum_t(ga);
          if (ga == T(0) || al == T(0) || be == T(0) || fabs(ga) <= tol * sqrt(al) * sqrt(be)) continue;
          const T zeta = (be - al) / (T(2) * ga);
          const T tn = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
          const T c = T(1) / sqrt(T(1) + tn * tn), sn = c * tn;
          for (int j = lane; j < Lp; j += 32) {  // the W row and the Qt row
            const T u = wa[j], v = wb[j];
            wa[j] = c * u - sn * v;
            wb[j] = sn * u + c * v;
          }
          rotated = 1;
        }
      }
      __syncthreads();
      // the two vectors leaving this CTA, into the neighbours' receive buffers
      const int out_top = topb[ns - 1], out_bot = botb[0];
      if (rank + 1 < C) {
        const T* src = buf(out_top);
        T* dst = cluster.map_shared_rank(dsm + static_cast<int64_t>(2 * ns_next + parity) * Lp, rank + 1);
        for (int j = threadIdx.x; j < Lp; j += blockDim.x) dst[j] = src[j];
      }
      if (rank > 0) {
        const T* src = buf(out_bot);
        T* dst = cluster.map_shared_rank(dsm + static_cast<int64_t>(2 * ns_prev + 2 + parity) * Lp, rank - 1);
        for (int j = threadIdx.x; j < Lp; j += blockDim.x) dst[j] = src[j];
      }
      svd_barrier(cl);  // every send has landed (and every thread has read topb / botb)
      if (threadIdx.x == 0) {
        // the vectors that stay move one slot by renaming their buffers; the
        // two sent away free theirs for the two that arrived
        for (int k = ns - 2; k >= (rank == 0 ? 1 : 0); --k) topb[k + 1] = topb[k];
        if (rank == 0) topb[1] = out_bot;  // topb[0] stays
        else topb[0] = out_bot;             // filled from the previous CTA below
        for (int k = 1; k < ns; ++k) botb[k - 1] = botb[k];
        botb[ns - 1] = out_top;  // stays here on the last CTA, filled from the next CTA elsewhere
      }
      if (rank > 0) {
        const T* src = buf(2 * ns + parity);
        T* dst = buf(out_bot);
        for (int j = threadIdx.x; j < Lp; j += blockDim.x) dst[j] = src[j];
      }
      if (rank + 1 < C) {
        const T* src = buf(2 * ns + 2 + parity);
        T* dst = buf(out_top);
        for (int j = threadIdx.x; j < Lp; j += blockDim.x) dst[j] = src[j];
      }
      parity ^= 1;
      __syncthreads();
    }
    // any rotation anywhere in the cluster this sweep?  (flags alternate by
    // sweep parity, so a peer's next write waits behind two barriers)
    rotated = __syncthreads_or(rotated);
    if (threadIdx.x == 0) rflag[sweep & 1] = rotated;
    svd_barrier(cl);
    int any = 0;
    for (int r = 0; r < C; ++r) any |= *cluster.map_shared_rank(&rflag[sweep & 1], r);
    if (!any) break;
  }
  // every vector is back in its first slot: write W and Qt rows
  for (int s = 0; s < ns; ++s)
    for (int h = 0; h < 2; ++h) {
      const int v = 2 * (k0 + s) + h;
      if (v >= p) continue;
      const T* src = buf(h == 0 ? topb[s] : botb[s]);
      for (int j = threadIdx.x; j < Lp; j += blockDim.x) {
        if (j < L) W[static_cast<int64_t>(v) * L + j] = src[j];
        else Qt[static_cast<int64_t>(v) * p + (j - L)] = src[j];
      }
    }
  svd_barrier(cl);
}

// Per-CTA shared scalars of svd_factor and its dynamic shared memory.
template <typename T>
struct SvdShared {
  double* red;   // kSvdWarps
  int* s_rot;
  int* s_r;
  T* tile;       // 32 x 33
  unsigned char* dsm;
  size_t smem_bytes;
};

// SVD of the row-major m x n matrix M = U S V^T, truncated: the smallest
// r >= 1 whose dropped singular values have squared 2-norm <= delta2, then at
// most max_rank (0: no cap).  Writes U's first r columns to u_out (m x r,
// row-major) and the first r rows of S V^T to svt_out (r x n); returns r.
// M is overwritten; scratch holds m n entries (the transpose of a tall M),
// qt p^2, sig and ord p.  svt_out may alias M (not scratch), u_out neither.
// Every CTA of the cluster calls it; only the leader's arguments are read
// (the others may pass anything) and only the leader's result is meaningful.
template <typename T>
__device__ int svd_factor(T* M, T* scratch, T* qt, double* sig, int32_t* ord, int m, int n, double delta2,
                          int max_rank, T* u_out, T* svt_out, const SvdShared<T>& sh, SvdCluster& cl) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool leader = cl.rank == 0;
  if (leader) {
    const bool wide = m < n;
    const int pp = wide ? m : n, L = wide ? n : m;
    T* W = M;
    if (!wide) {
      transpose_rows<T>(scratch, M, m, n, sh.tile);
      W = scratch;
    }
    // where the sweeps run: 0 the leader's shared memory; 4 the cluster's,
    // vectors spread over the CTAs; 1 the cluster's, columns spread; 3 the
    // same in place in the workspace; 2 the leader alone in the workspace
    const int64_t wl = static_cast<int64_t>(pp) * L;
    const size_t rd = rowdist_smem_elems(pp, L, cl.C);
    int path = 2;
    if (static_cast<size_t>(wl + static_cast<int64_t>(pp) * pp) * sizeof(T) <= sh.smem_bytes) path = 0;
    else if (cl.C > 1 && rd > 0 && rd * sizeof(T) <= sh.smem_bytes) path = 4;
    else if (cl.C > 1 && dist_smem_elems(pp, L, cl.C) * sizeof(T) <= sh.smem_bytes) path = 1;
    else if (cl.C > 1) path = 3;
    if (tid == 0) {
      cl.bc[0] = pp;
      cl.bc[1] = L;
      cl.bc[2] = path;
      cl.bcp[0] = reinterpret_cast<unsigned long long>(W);
      cl.bcp[1] = reinterpret_cast<unsigned long long>(qt);
    }
  }
  svd_barrier(cl);
  int pp, L, path;
  T* W;
  {
    namespace cg = cooperative_groups;
    const int* bc = cl.C > 1 ? cg::this_cluster().map_shared_rank(cl.bc, 0) : cl.bc;
    const unsigned long long* bcp = cl.C > 1 ? cg::this_cluster().map_shared_rank(cl.bcp, 0) : cl.bcp;
    pp = bc[0];
    L = bc[1];
    path = bc[2];
    W = reinterpret_cast<T*>(bcp[0]);
    qt = reinterpret_cast<T*>(bcp[1]);
  }
  if (path == 1 || path == 3 || path == 4) {
    if (path == 4)
      jacobi_rowdist<T>(W, qt, pp, L, reinterpret_cast<T*>(sh.dsm), cl);
    else if (path == 1)
      jacobi_dist<T, true>(W, qt, pp, L, reinterpret_cast<T*>(sh.dsm), cl);
    else
      jacobi_dist<T, false>(W, qt, pp, L, reinterpret_cast<T*>(sh.dsm), cl);
  } else if (leader) {
    const int64_t wl = static_cast<int64_t>(pp) * L;
    T* Wj = path == 0 ? reinterpret_cast<T*>(sh.dsm) : W;
    T* Qj = path == 0 ? Wj + wl : qt;
    if (path == 0)
      for (int64_t e = tid; e < wl; e += kSvdThreads) Wj[e] = W[e];
    for (int e = tid; e < pp * pp; e += kSvdThreads) Qj[e] = (e / pp == e % pp) ? T(1) : T(0);
    __syncthreads();
    jacobi_rows<T>(Wj, Qj, pp, L, sh.s_rot);
    if (path == 0) {
      for (int64_t e = tid; e < wl; e += kSvdThreads) W[e] = Wj[e];
      for (int e = tid; e < pp * pp; e += kSvdThreads) qt[e] = Qj[e];
    }
  }
  svd_barrier(cl);
  if (!leader) return 0;
  const bool wide = m < n;
  // singular values: the row norms (float64 sums), warp per row
  for (int i = warp; i < pp; i += kSvdWarps) {
    double s2 = 0.0;
    const T* w = W + static_cast<int64_t>(i) * L;
    for (int e = lane; e < L; e += 32) {
      const double v = static_cast<double>(__ldcg(w + e));  // peers may have written W: read it from L2
      s2 += v * v;
    }
    s2 = warp_sum_t(s2);
    if (lane == 0) sig[i] = sqrt(s2);
  }
  __syncthreads();
  // order, largest first (ties by index): position of value i
  for (int i = tid; i < pp; i += kSvdThreads) {
    const double si = sig[i];
    int pos = 0;
    for (int j = 0; j < pp; ++j) {
      const double sj = sig[j];
      pos += (sj > si || (sj == si && j < i)) ? 1 : 0;
    }
    ord[pos] = i;
  }
  __syncthreads();
  if (tid == 0) {
    int r = pp;
    double dropped = 0.0;
    while (r > 1) {
      const double s = sig[ord[r - 1]];
      if (dropped + s * s > delta2) break;
      dropped += s * s;
      --r;
    }
    if (max_rank > 0 && r > max_rank) r = max_rank;
    *sh.s_r = r;
  }
  __syncthreads();
  const int r = *sh.s_r;
  if (wide) {
    // U = Q (u_out[i][t] = qt[ord t][i]); S V^T = the rows of W in order
    for (int64_t e = tid; e < static_cast<int64_t>(r) * n; e += kSvdThreads) {
      const int t = static_cast<int>(e / n);
      const int64_t j = e - static_cast<int64_t>(t) * n;
      svt_out[e] = __ldcg(W + static_cast<int64_t>(ord[t]) * n + j);
    }
    for (int e = tid; e < m * r; e += kSvdThreads) {
      const int i = e / r, t = e - i * r;
      u_out[e] = __ldcg(qt + static_cast<int64_t>(ord[t]) * pp + i);
    }
  } else {
    // W = S U^T row by row: u_out[i][t] = W[ord t][i] / sigma; S V^T = sigma qt rows
    for (int64_t e = tid; e < static_cast<int64_t>(m) * r; e += kSvdThreads) {
      const int64_t i = e / r;
      const int t = static_cast<int>(e - i * r);
      const int o = ord[t];
      const double s = sig[o];
      u_out[e] = s > 0.0 ? static_cast<T>(static_cast<double>(__ldcg(W + static_cast<int64_t>(o) * m + i)) / s) : T(0);
    }
    for (int e = tid; e < r * n; e += kSvdThreads) {
      const int t = e / n, j = e - t * n;
      const int o = ord[t];
      svt_out[e] = static_cast<T>(sig[o] * static_cast<double>(__ldcg(qt + static_cast<int64_t>(o) * pp + j)));
    }
  }
  __syncthreads();
  return r;
}

// Launch one of the decomposition kernels on a cluster of CTAs: the largest
// of 16, 8, 4, 2, 1 the device can place with the dynamic shared memory
// `smem_of(C)` asks for (the sweeps' needs depend on C).  Returns the launch
// status; *c_out gets the cluster size.
template <typename Params, typename SmemOf>
static cudaError_t svd_launch(void (*kernel)(Params), Params params, SmemOf smem_of, cudaStream_t s) {
  cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (err != cudaSuccess) return err;
  for (int c = 16; c >= 1; c >>= 1) {
    // at least the exchange buffers of the largest SVD (p <= 512)
    const size_t smem = c > 1 ? std::max<size_t>(smem_of(c), dist_comm_elems(kSvdMaxP, c) * sizeof(double)) : smem_of(c);
    err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(kSvdThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kernel, &cfg) != cudaSuccess || nclusters < 1) {
      cudaGetLastError();  // a size the device cannot place: try the next
      continue;
    }
    params.smem_bytes = smem;
    return cudaLaunchKernelEx(&cfg, kernel, params);
  }
  return cudaErrorInvalidConfiguration;
}

}  // namespace ttc
