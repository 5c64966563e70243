// Persistent batched contraction: one launch works through thousands of
// independent pairs of uneven order, mode size and rank.
//
// The grid holds as many CTAs as fit on the GPU at once.  Each CTA takes the
// next pair from a global counter (pairs are pre-sorted longest-first, so the
// queue is an LPT schedule) and runs the whole environment sweep of that pair
// -- and, for a partial contraction, its chain emission -- with the per-CTA
// engine of pair_engine.cuh, following the evaluation order and panels the plan chose
// for each mode.  Nothing in
// the launch depends on the host: the counter is reset by a memset node, so
// the pair (memset, kernel) can be captured in a CUDA graph and replayed.
#include "pair_engine.cuh"

namespace ttc {

struct BatchKernelParams {
  const SweepParams* table;  // [n] per-pair sweep parameters
  const int32_t* order;      // [n] pair indices, longest first
  const int32_t* tile;       // [n] rank tile per pair: 0 -> 32, 1 -> 64, 2 -> 128
  int n;
  const CopyJob* jobs;       // free-core copies of the partial pairs
  int n_jobs;
  int* counter;              // [0] pair queue head, [1] copy queue head (zeroed before the launch)
  double* out;               // [n]
  int64_t* out_log2;         // [n] or NULL
  int32_t* status;
};

constexpr int kBatchThreads = eng::NTOT;

template <typename T>
__global__ void __launch_bounds__(eng::NTOT, 1) batched_kernel(const __grid_constant__ BatchKernelParams bp) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_idx;
  // The copy kernel that follows depends on none of this launch's work: let it
  // take each SM this launch leaves (it waits for this grid before it ends).
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  for (;;) {
    __syncthreads();  // every thread has read the previous s_idx
    if (threadIdx.x == 0) s_idx = atomicAdd(bp.counter, 1);
    __syncthreads();
    const int idx = s_idx;
    if (idx >= bp.n) break;
    const int pair = bp.order[idx];
    SweepOut o{bp.out + pair, bp.out_log2 != nullptr ? bp.out_log2 + pair : nullptr, bp.status};
    o.skip_copies = 1;
    eng::run_pair<T>(bp.table[pair], o, smem);
  }
}

// Free-core copies of the partial pairs (they depend on no sweep).  Jobs are
// dealt statically (job j to CTA j mod grid).  Every job (at most
// kCopyJobBytes) goes through shared memory: its loads are all issued at once
// with cp.async, and the next job's loads are issued before this one is
// written out (two staging buffers), so a CTA keeps up to two jobs of loads in
// flight while holding no data in registers.  (Loading a job into registers
// instead was slower: fewer CTAs fit on an SM.)
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
// that an element costs a few instructions (the kernel is issue-bound).
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
      const int row = eng::udiv16(e, g.lw), c = e - row * g.lw;
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
      const int d0 = eng::udiv16(32, r1), d1 = 32 - d0 * r1;
      const int ds = d1 * P + d0 * na, dw = na - r1 * P;
      const int il0 = eng::udiv16(lane, r1), c10 = lane - il0 * r1, s0 = c10 * P + il0 * na;
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
        const int ar = eng::udiv16(e, run), c = e - ar * run;
        const int il = eng::udiv16(c, r1), c1 = c - il * r1;
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
      const int c1 = eng::udiv16(f, nq), q = f - c1 * nq;
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

template <typename T>
__global__ void __launch_bounds__(kCopyThreads) copy_jobs_kernel(const CopyJob* __restrict__ jobs, int n_jobs) {
  extern __shared__ __align__(16) unsigned char copy_smem[];
  T* const buf0 = reinterpret_cast<T*>(copy_smem);
  T* const buf1 = buf0 + copy_buf_elems<T>();
  const int G = gridDim.x;
  int jb = blockIdx.x;
  if (jb < n_jobs) {
    CopyJob cur = jobs[jb];
    CopyJob nxt = jb + G < n_jobs ? jobs[jb + G] : cur;  // descriptors are read one job ahead
    copy_issue<T>(cur, buf0);
    for (int k = 0;; ++k) {
      const bool more = jb + G < n_jobs;
      CopyJob after = nxt;
      if (more) {
        if (jb + 2 * G < n_jobs) after = jobs[jb + 2 * G];
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
      jb += G;
    }
  }
  // Launched as a programmatic dependent of the batched kernel: end only once
  // that grid has completed, so that stream order holds for later work.
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename T>
static cudaError_t launch_batched_impl(const BatchKernelParams& bp, int grid, cudaStream_t s) {
  const size_t smem = eng::smem_bytes<T>();
  cudaError_t err =
      cudaFuncSetAttribute(batched_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  if (grid <= 0) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batched_kernel<T>, kBatchThreads, smem);
    if (err != cudaSuccess) return err;
    grid = sms * std::max(per, 1);
  }
  grid = std::min(grid, std::max(bp.n, 1));
  count_launch();
  batched_kernel<T><<<grid, kBatchThreads, smem, s>>>(bp);
  err = cudaGetLastError();
  if (err != cudaSuccess || bp.n_jobs == 0) return err;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t csmem = copy_smem_bytes<T>();
  err = cudaFuncSetAttribute(copy_jobs_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(csmem));
  if (err != cudaSuccess) return err;
  int cper = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cper, copy_jobs_kernel<T>, kCopyThreads, csmem);
  if (err != cudaSuccess) return err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(std::min(bp.n_jobs, sms * std::max(cper, 1)));
  cfg.blockDim = dim3(kCopyThreads);
  cfg.dynamicSmemBytes = csmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;  // start on the SMs the sweeps leave
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, copy_jobs_kernel<T>, bp.jobs, bp.n_jobs);
}

cudaError_t launch_batched(const void* table, const int32_t* order, const int32_t* tile, int n,
                           const CopyJob* jobs, int n_jobs, int* counters, double* out, int64_t* out_log2,
                           int32_t* status, int dtype, int grid, cudaStream_t s) {
  BatchKernelParams bp;
  bp.table = static_cast<const SweepParams*>(table);
  bp.order = order;
  bp.tile = tile;
  bp.n = n;
  bp.jobs = jobs;
  bp.n_jobs = n_jobs;
  bp.counter = counters;
  bp.out = out;
  bp.out_log2 = out_log2;
  bp.status = status;
  if (dtype == TT_F64) return launch_batched_impl<double>(bp, grid, s);
  return launch_batched_impl<float>(bp, grid, s);
}

}  // namespace ttc
