// Free-core copies of chain-layout outputs (and of their cotangents), cut
// into jobs of at most kCopyJobBytes (copy_cut / copy_job_at in
// ttc_internal.h) and run by whole CTAs of kCopyThreads threads.
//
// Every job goes through shared memory: its loads are all issued at once with
// cp.async, and the next job's loads are issued before this one is written
// out (two staging buffers), so a CTA keeps up to two jobs of loads in flight
// while holding no data in registers.  (Loading a job into registers instead
// was slower: fewer CTAs fit on an SM.)
//   plain job:      rows [a0, a1) x slices [i0, i1), one contiguous run per
//                   row (one run in all when the rows span every slice),
//                   staged densely, 16 bytes a copy when every run is aligned;
//   transposed job: element (row ar, slice il, column c1) is staged at
//                   c1 * P + il * na + ar, i.e. in destination order with an
//                   odd pitch P >= ni * na per column: the reads run along
//                   the source rows, the writes along the destination rows
//                   (a slice of the output core, or all of the job's slices of
//                   it, is contiguous), and neither side has bank conflicts
//                   to speak of.
// The loops are rows of a warp each, lanes stepping by 32 along the row, so
// that an element costs a few instructions (the copies are issue-bound).
#pragma once

#include "ttc_device.cuh"
#include "ttc_internal.h"

namespace ttc {

constexpr int kCopyThreads = 256;
constexpr int kCopyWarps = kCopyThreads / 32;

struct CopyGeo {
  int na, ni, rows, lw, w, P;
  bool vec;
  int rstride;  // elements between two rows of the core (I * r1 < 2^31)
  int64_t base;
};

template <typename T>
__device__ __forceinline__ CopyGeo copy_geo(const CopyJob& j) {
  constexpr int VW = 16 / static_cast<int>(sizeof(T));
  CopyGeo g;
  g.ni = j.i1 - j.i0;
  g.na = j.a1 - j.a0;
  const int run = g.ni * j.r1;  // contiguous source elements of one row
  g.rstride = j.I * j.r1;
  g.base = (static_cast<int64_t>(j.a0) * j.I + j.i0) * j.r1;
  g.P = (g.ni * g.na) | 1;
  if (j.swap) {
    g.vec = false;
    g.rows = g.na;
    g.lw = run;
  } else {
    const int len = g.ni == j.I ? g.na * run : run;
    g.rows = g.ni == j.I ? 1 : g.na;
    const T* s0 = static_cast<const T*>(j.src) + g.base;
    const T* d0 = static_cast<const T*>(j.dst) + g.base;
    g.vec = ((reinterpret_cast<uintptr_t>(s0) | reinterpret_cast<uintptr_t>(d0)) & 15) == 0 && len % VW == 0 &&
            g.rstride % VW == 0;
    g.lw = g.vec ? len / VW : len;
  }
  g.w = g.vec ? VW : 1;  // elements per copy
  return g;
}

// A plain job: copy unit (row, c), c < lw, between the core (row stride
// rstride, units of w elements) and the dense staging.  f(core_offset,
// staging_offset) in elements.
template <typename F>
__device__ __forceinline__ void plain_units(const CopyGeo& g, F f) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (g.rows == 1) {
    for (int e = threadIdx.x; e < g.lw; e += kCopyThreads) f(e * g.w, e * g.w);
  } else if (g.lw >= 32) {
    for (int row = warp; row < g.rows; row += kCopyWarps) {
      const int so = row * g.rstride, to = row * g.lw * g.w;
      for (int c = lane; c < g.lw; c += 32) f(so + c * g.w, to + c * g.w);
    }
  } else {
    const int tot = g.rows * g.lw;  // short rows: dealt flat (udiv16 is exact below 2^16)
    for (int e = threadIdx.x; e < tot; e += kCopyThreads) {
      const int row = udiv16(e, g.lw), c = e - row * g.lw;
      f(row * g.rstride + c * g.w, e * g.w);
    }
  }
}

template <typename T>
__device__ __forceinline__ void copy_issue(const CopyJob& j, T* st) {
  const CopyGeo g = copy_geo<T>(j);
  const T* __restrict__ src = static_cast<const T*>(j.src) + g.base;
  if (!j.swap) {
    if (g.vec)
      plain_units(g, [&](int so, int to) { cp_async16(st + to, src + so); });
    else
      plain_units(g, [&](int so, int to) { cp_async_elem(st + to, src + so); });
  } else {
    const int r1 = j.r1, na = g.na, P = g.P, run = g.lw;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (run >= 32) {
      // lane's column c = il * r1 + c1 advances by 32 = d0 * r1 + d1
      const int d0 = udiv16(32, r1), d1 = 32 - d0 * r1;
      const int ds = d1 * P + d0 * na, dw = na - r1 * P;
      const int il0 = udiv16(lane, r1), c10 = lane - il0 * r1, s0 = c10 * P + il0 * na;
      for (int ar = warp; ar < na; ar += kCopyWarps) {
        const T* __restrict__ row = src + ar * g.rstride;
        int c1 = c10, sidx = s0 + ar;
        for (int c = lane; c < run; c += 32) {
          cp_async_elem(st + sidx, row + c);
          c1 += d1;
          sidx += ds;
          if (c1 >= r1) {
            c1 -= r1;
            sidx += dw;
          }
        }
      }
    } else {
      const int tot = na * run;
      for (int e = threadIdx.x; e < tot; e += kCopyThreads) {
        const int ar = udiv16(e, run), c = e - ar * run;
        const int il = udiv16(c, r1), c1 = c - il * r1;
        cp_async_elem(st + c1 * P + il * na + ar, src + ar * g.rstride + c);
      }
    }
  }
  cp_async_commit();
}

template <typename T>
__device__ __forceinline__ void copy_drain(const CopyJob& j, const T* st) {
  const CopyGeo g = copy_geo<T>(j);
  if (!j.swap) {
    T* __restrict__ dst = static_cast<T*>(j.dst) + g.base;
    if (g.vec)
      plain_units(g, [&](int so, int to) {
        *reinterpret_cast<uint4*>(dst + so) = *reinterpret_cast<const uint4*>(st + to);
      });
    else
      plain_units(g, [&](int so, int to) { dst[so] = st[to]; });
    return;
  }
  // destination column c1 of the job: nq contiguous elements at
  // (c1 * I + i0) * r0 + a0 (all of a slice's rows, or one slice's rows a0..a1)
  const int r1 = j.r1, nq = g.ni * g.na, P = g.P;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* __restrict__ dst = static_cast<T*>(j.dst) + static_cast<int64_t>(j.i0) * j.r0 + j.a0;
  const int64_t ir0 = static_cast<int64_t>(j.I) * j.r0;
  if (nq >= 32) {
    for (int c1 = warp; c1 < r1; c1 += kCopyWarps) {
      T* __restrict__ drow = dst + c1 * ir0;
      const T* srow = st + c1 * P;
      for (int q = lane; q < nq; q += 32) drow[q] = srow[q];
    }
  } else {
    const int tot = r1 * nq;
    for (int f = threadIdx.x; f < tot; f += kCopyThreads) {
      const int c1 = udiv16(f, nq), q = f - c1 * nq;
      dst[c1 * ir0 + q] = st[c1 * P + q];
    }
  }
}

template <typename T>
__host__ __device__ constexpr int copy_job_elems() {
  return kCopyJobBytes / static_cast<int>(sizeof(T));
}
// Staging elements of one buffer: a transposed job pads its rows (na of them)
// to an odd length only when na is even, which adds run = tot / na <= cap / 2.
template <typename T>
__host__ __device__ constexpr int copy_buf_elems() {
  return copy_job_elems<T>() + copy_job_elems<T>() / 2;
}
template <typename T>
constexpr size_t copy_smem_bytes() {
  return 2 * static_cast<size_t>(copy_buf_elems<T>()) * sizeof(T);  // two buffers
}

// A CTA's share of a list of copy jobs: jobs first, first + step, ... < n,
// where job_of(jb) returns job jb.  Two staging buffers (buf0, buf1 of
// copy_buf_elems<T>() elements): the next job's loads are in flight while
// this one is written out; descriptors are read one job ahead.
template <typename T, typename JobOf>
__device__ __forceinline__ void copy_jobs_block(JobOf job_of, int first, int n, int step, T* buf0, T* buf1) {
  int jb = first;
  if (jb >= n) return;
  CopyJob cur = job_of(jb);
  CopyJob nxt = jb + step < n ? job_of(jb + step) : cur;
  copy_issue<T>(cur, buf0);
  for (int k = 0;; ++k) {
    const bool more = jb + step < n;
    CopyJob after = nxt;
    if (more) {
      if (jb + 2 * step < n) after = job_of(jb + 2 * step);
      copy_issue<T>(nxt, (k & 1) ? buf0 : buf1);  // that buffer was drained in the previous iteration
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    copy_drain<T>(cur, (k & 1) ? buf1 : buf0);
    __syncthreads();
    if (!more) break;
    cur = nxt;
    nxt = after;
    jb += step;
  }
}

}  // namespace ttc
