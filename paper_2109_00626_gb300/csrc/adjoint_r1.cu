// Adjoint of a full contraction whose second operand has every rank 1.  The
// sum of a TT's entries is its contraction with the all-ones rank-1 TT -- the
// usual way a partial contraction is reduced to a loss -- and with one operand
// of rank 1 the environments are vectors (y_k[i] = Gy_k[0][i][0]).  With the
// folded cores M_k = sum_i y_k[i] Gx_k[:, i, :] (rx x rx2 matrices),
//   L_0 = 1,  L_{k+1} = L_k M_k          (row vectors)
//   F_N = 1,  F_k     = M_k F_{k+1}      (column vectors)
// z = L_N = F_0, and, z being linear in each core (Eq. 9), the gradients are
//   dGx_k[a][i][a'] = g L_k[a] y_k[i] F_{k+1}[a']
//   dGy_k[0][i][0]  = g sum_{a,a'} L_k[a] Gx_k[a][i][a'] F_{k+1}[a'].
// Three launches: the fold of every core at once (the cores are read once,
// by every SM), the two chains of vector-matrix products (one block each,
// on the folded cores, which sit in L2; a 128-thread kernel when every rank
// is at most 64), and the gradients, one block per (k, i).  Every vector is
// kept with a power-of-two scale (no checkpoints: the vectors are small).
// The forward value alone takes the fold and the left chain.
#include "ttc_device.cuh"
#include "ttc_internal.h"

namespace ttc {

namespace {

constexpr int kR1Threads = 512;
constexpr int kR1Warps = kR1Threads / 32;
constexpr int kNoExpR1 = -(1 << 30);
constexpr int kFoldThreads = 256;

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

// M_k[a][c] = sum_i y_k[i] Gx_k[a][i][c] (i in order); with mtbuf set also
// M_k^T[c][a].  A block takes fold_rows(k) = max(1, 256 / rx2) rows of one
// core, a thread per (row, column), so narrow cores keep every lane busy.
__host__ __device__ inline int fold_rows(int rx2) { return rx2 >= kFoldThreads ? 1 : kFoldThreads / rx2; }

template <typename T>
__global__ void __launch_bounds__(kFoldThreads) r1_fold_kernel(const __grid_constant__ AdjR1Params p) {
  int k = 0, b = static_cast<int>(blockIdx.x);
  while (k + 1 < p.n) {
    const int nb = (p.step[k].rx + fold_rows(p.step[k].rx2) - 1) / fold_rows(p.step[k].rx2);
    if (b < nb) break;
    b -= nb;
    ++k;
  }
  const AdjStep& st = p.step[k];
  const int I = st.I, R = st.rx, R2 = st.rx2, fr = fold_rows(R2);
  const T* y = static_cast<const T*>(st.gy);
  T* m = static_cast<T*>(p.mbuf) + p.moff[k];
  T* mt = p.mtbuf != nullptr ? static_cast<T*>(p.mtbuf) + p.moff[k] : nullptr;
  const int q = static_cast<int>(threadIdx.x) / (fr > 1 ? R2 : kFoldThreads);  // row of this block
  const int a = b * fr + q;
  if (q >= fr || a >= R) return;
  const T* gx = static_cast<const T*>(st.gx) + static_cast<int64_t>(a) * I * R2;
  for (int c = fr > 1 ? static_cast<int>(threadIdx.x) % R2 : static_cast<int>(threadIdx.x); c < R2;
       c += fr > 1 ? R2 : kFoldThreads) {
    T acc = T(0);
#pragma unroll 4
    for (int i = 0; i < I; ++i) acc = fma(ldg(y + i), ldg(gx + static_cast<int64_t>(i) * R2 + c), acc);
    m[static_cast<int64_t>(a) * R2 + c] = acc;
    if (mt != nullptr) mt[static_cast<int64_t>(c) * R + a] = acc;
  }
}

// The chains: block 0 forms L_1..L_N (out = in M_k: A = M_k, [R][R2]),
// block 1 F_{N-1}..F_0 (out = M_k in: A = M_k^T, [R2][R]).  Each output
// entry is summed by G threads over strided rows of A (rows g, g + G, ...;
// neighbouring threads take neighbouring entries, so the loads of A are
// coalesced), then its G parts are added in order.
template <typename T>
__global__ void __launch_bounds__(kR1Threads) r1_chain_kernel(const __grid_constant__ AdjR1Params p) {
  extern __shared__ __align__(16) unsigned char r1_smem[];
  T* cur = reinterpret_cast<T*>(r1_smem);  // [kR1MaxRank] the current vector
  T* nxt = cur + kR1MaxRank;                // [kR1MaxRank] the next vector
  T* part = nxt + kR1MaxRank;               // [kR1Threads] partial sums
  __shared__ int red[2][2 * kR1Warps];
  __shared__ double zr[kR1Warps];
  const bool left = blockIdx.x == 0;
  const int tid = threadIdx.x;
  const int n = p.n;
  int bad = 0;
  T* vecs = static_cast<T*>(left ? p.lvec : p.fvec);
  int64_t* scl = left ? p.llog : p.flog;
  int64_t lg = 0;
  if (tid == 0) cur[0] = T(1);
  if (!p.fwd && tid == 0) {
    vecs[static_cast<int64_t>(left ? 0 : n) * p.vstride] = T(1);
    scl[left ? 0 : n] = 0;
  }
  __syncthreads();
  const int steps = p.fwd ? n - 1 : n;  // the forward value's last step is summed in float64
  // A step whose matrix has <= kR1Threads columns and <= kPre rows per thread
  // has its loads issued during the step before (registers `pre`), so the
  // chain waits on no memory latency but the first
  constexpr int kPre = 16;
  auto geo = [&](int step, const T*& A, int& rows, int& cols) {
    const int k = left ? step : n - 1 - step;
    const AdjStep& st = p.step[k];
    rows = left ? st.rx : st.rx2;
    cols = left ? st.rx2 : st.rx;
    A = static_cast<const T*>(left ? p.mbuf : p.mtbuf) + p.moff[k];
    return cols <= kR1Threads && (rows + kR1Threads / cols - 1) / (kR1Threads / cols) <= kPre;
  };
  auto prefetch = [&](const T* A, int rows, int cols, T (&pre)[kPre]) {
    const int G = kR1Threads / cols, c = tid % cols, g = tid / cols;
#pragma unroll
    for (int j = 0; j < kPre; ++j) {
      const int r = g + j * G;
      pre[j] = (g < G && r < rows) ? ldg(A + static_cast<int64_t>(r) * cols + c) : T(0);
    }
  };
  T pre[kPre];
  {
    const T* A0;
    int r0, c0;
    if (steps > 0 && geo(0, A0, r0, c0)) prefetch(A0, r0, c0, pre);
  }
  for (int step = 0; step < steps; ++step) {
    const int k = left ? step : n - 1 - step;
    const T* A;
    int rows, cols;
    const bool fast = geo(step, A, rows, cols);
    int e = kNoExpR1, lbad = 0;
    for (int c0 = 0; c0 < cols; c0 += kR1Threads) {
      const int nc = min(kR1Threads, cols - c0);
      const int G = max(1, kR1Threads / nc);
      const int c = tid % nc, g = tid / nc;
      T acc = T(0);
      if (fast) {
#pragma unroll
        for (int j = 0; j < kPre; ++j) {
          const int r = g + j * G;
          if (g < G && r < rows) acc = fma(cur[r], pre[j], acc);
        }
        const T* An;
        int rn, cn;
        if (step + 1 < steps && geo(step + 1, An, rn, cn)) prefetch(An, rn, cn, pre);
      } else if (g < G) {
#pragma unroll 8
        for (int r = g; r < rows; r += G) acc = fma(cur[r], ldg(A + static_cast<int64_t>(r) * cols + c0 + c), acc);
      }
      __syncthreads();  // the previous pass has read `part`
      part[tid] = acc;
      __syncthreads();
      if (tid < nc) {
        T sum = T(0);
        for (int q = 0; q < G; ++q) sum += part[q * nc + tid];
        if (!isfinite(sum)) lbad = 1;
        else if (sum != T(0)) e = max(e, exp2_bits(sum));
        nxt[c0 + tid] = sum;
      }
    }
    block_max_or_r1(e, lbad, red[step & 1]);  // also: every thread is past its reads of cur
    if (lbad) bad = 1;
    const int sh = (e != kNoExpR1 && (e > p.renorm_bits || e < -p.renorm_bits)) ? e : 0;
    lg += sh;
    const int64_t vk = left ? k + 1 : k;
    for (int c = tid; c < cols; c += kR1Threads) {
      const T v = sh ? mul_pow2<T>(nxt[c], -sh) : nxt[c];
      cur[c] = v;
      if (!p.fwd) vecs[vk * p.vstride + c] = v;
    }
    if (!p.fwd && tid == 0) scl[vk] = lg;
    if (!fast && step + 1 < steps) {  // a fast step after a slow one: its loads now
      const T* An;
      int rn, cn;
      if (geo(step + 1, An, rn, cn)) prefetch(An, rn, cn, pre);
    }
    __syncthreads();  // cur is complete before the next step reads it
  }
  if (p.fwd && left) {
    // z = L_{N-1} M_{N-1} (a 1 x 1 result), summed in float64
    const AdjStep& st = p.step[n - 1];
    const T* A = static_cast<const T*>(p.mbuf) + p.moff[n - 1];
    double s = 0.0;
    for (int r = tid; r < st.rx; r += kR1Threads) s = fma(static_cast<double>(cur[r]), static_cast<double>(A[r]), s);
    s = warp_sum(s);
    if ((tid & 31) == 0) zr[tid >> 5] = s;
    __syncthreads();
    if (tid == 0) {
      double z = 0.0;
      for (int w = 0; w < kR1Warps; ++w) z += zr[w];
      int st_bits = (isfinite(z) && !bad) ? 0 : TT_STATUS_NONFINITE;
      if (p.z_out_log2 != nullptr) {
        *p.z_out = z;
        *p.z_out_log2 = lg;
      } else {
        // the scale folded in: infinity (and TT_STATUS_OVERFLOW) beyond the
        // float64 range, zero below it
        double v = z;
        if (z != 0.0 && isfinite(z)) {
          const int64_t tot = static_cast<int64_t>(exp2_of(z)) + lg;
          if (tot > 1024) {
            v = z > 0 ? INFINITY : -INFINITY;
            st_bits |= TT_STATUS_OVERFLOW;
          } else if (tot < -1074) {
            v = 0.0;
          } else {
            v = ldexp(z, static_cast<int>(lg));
          }
        }
        *p.z_out = v;
      }
      if (st_bits) set_status(p.status, st_bits);
    }
    return;
  }
  if (bad && tid == 0) set_status(p.status, TT_STATUS_NONFINITE);
}

// The chains when every rank is at most 64: 128 threads, output column c of
// a step taken by the 16-lane half-warps of warp c / 16, lane half h summing
// rows h, h + 2, ... of A (32 registers, loaded during the step before), the
// halves joined by one shuffle; two block barriers a step.  Same sums and
// scaling rules as r1_chain_kernel.
constexpr int kC64Threads = 128;
template <typename T>
__global__ void __launch_bounds__(kC64Threads) r1_chain64_kernel(const __grid_constant__ AdjR1Params p) {
  __shared__ T cur[64];
  __shared__ T nxt[64];
  __shared__ int wred[2][8];
  __shared__ double zr[4];
  const bool left = blockIdx.x == 0;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c = warp * 16 + (lane & 15), h = lane >> 4;
  const int n = p.n;
  int bad = 0;
  T* vecs = static_cast<T*>(left ? p.lvec : p.fvec);
  int64_t* scl = left ? p.llog : p.flog;
  int64_t lg = 0;
  if (tid < 64) cur[tid] = tid == 0 ? T(1) : T(0);
  if (!p.fwd && tid == 0) {
    vecs[static_cast<int64_t>(left ? 0 : n) * p.vstride] = T(1);
    scl[left ? 0 : n] = 0;
  }
  const int steps = p.fwd ? n - 1 : n;  // the forward value's last step is summed in float64
  T pre[32];
  auto fetch = [&](int step) {
    const int k = left ? step : n - 1 - step;
    const AdjStep& st = p.step[k];
    const int rows = left ? st.rx : st.rx2, cols = left ? st.rx2 : st.rx;
    const T* A = static_cast<const T*>(left ? p.mbuf : p.mtbuf) + p.moff[k];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int r = h + 2 * j;
      pre[j] = (r < rows && c < cols) ? ldg(A + static_cast<int64_t>(r) * cols + c) : T(0);
    }
  };
  if (steps > 0) fetch(0);
  __syncthreads();
  for (int step = 0; step < steps; ++step) {
    const int k = left ? step : n - 1 - step;
    const AdjStep& st = p.step[k];
    const int cols = left ? st.rx2 : st.rx;
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < 32; ++j) acc = fma(cur[h + 2 * j], pre[j], acc);
    acc += __shfl_xor_sync(0xffffffffu, acc, 16);
    if (step + 1 < steps) fetch(step + 1);  // the next matrix's loads during this step's reductions
    int e = kNoExpR1, lbad = 0;
    if (h == 0 && c < cols) {
      nxt[c] = acc;
      if (!isfinite(acc)) lbad = 1;
      else if (acc != T(0)) e = exp2_bits(acc);
    }
    e = __reduce_max_sync(0xffffffffu, e);
    lbad = __reduce_or_sync(0xffffffffu, lbad);
    if (lane == 0) {
      wred[step & 1][warp] = e;
      wred[step & 1][4 + warp] = lbad;
    }
    __syncthreads();  // nxt complete, every thread past its reads of cur
    e = kNoExpR1;
    lbad = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      e = max(e, wred[step & 1][w]);
      lbad |= wred[step & 1][4 + w];
    }
    if (lbad) bad = 1;
    const int sh = (e != kNoExpR1 && (e > p.renorm_bits || e < -p.renorm_bits)) ? e : 0;
    lg += sh;
    if (tid < 64) {
      const T v = tid < cols ? (sh ? mul_pow2<T>(nxt[tid], -sh) : nxt[tid]) : T(0);
      cur[tid] = v;
      if (!p.fwd && tid < cols) vecs[static_cast<int64_t>(left ? k + 1 : k) * p.vstride + tid] = v;
    }
    if (!p.fwd && tid == 0) scl[left ? k + 1 : k] = lg;
    __syncthreads();  // cur is complete before the next step reads it
  }
  if (p.fwd && left) {
    // z = L_{N-1} M_{N-1} (a 1 x 1 result), summed in float64
    const AdjStep& st = p.step[n - 1];
    const T* A = static_cast<const T*>(p.mbuf) + p.moff[n - 1];
    double s = 0.0;
    for (int r = tid; r < st.rx; r += kC64Threads) s = fma(static_cast<double>(cur[r]), static_cast<double>(A[r]), s);
    s = warp_sum(s);
    if (lane == 0) zr[warp] = s;
    __syncthreads();
    if (tid == 0) {
      const double z = zr[0] + zr[1] + zr[2] + zr[3];
      int st_bits = (isfinite(z) && !bad) ? 0 : TT_STATUS_NONFINITE;
      if (p.z_out_log2 != nullptr) {
        *p.z_out = z;
        *p.z_out_log2 = lg;
      } else {
        // the scale folded in: infinity (and TT_STATUS_OVERFLOW) beyond the
        // float64 range, zero below it
        double v = z;
        if (z != 0.0 && isfinite(z)) {
          const int64_t tot = static_cast<int64_t>(exp2_of(z)) + lg;
          if (tot > 1024) {
            v = z > 0 ? INFINITY : -INFINITY;
            st_bits |= TT_STATUS_OVERFLOW;
          } else if (tot < -1074) {
            v = 0.0;
          } else {
            v = ldexp(z, static_cast<int>(lg));
          }
        }
        *p.z_out = v;
      }
      if (st_bits) set_status(p.status, st_bits);
    }
    return;
  }
  if (bad && tid == 0) set_status(p.status, TT_STATUS_NONFINITE);
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

static cudaError_t r1_fold(const AdjR1Params& p, int dtype, cudaStream_t s) {
  int blocks = 0;
  for (int k = 0; k < p.n; ++k) blocks += (p.step[k].rx + fold_rows(p.step[k].rx2) - 1) / fold_rows(p.step[k].rx2);
  count_launch();
  if (dtype == TT_F64) r1_fold_kernel<double><<<blocks, kFoldThreads, 0, s>>>(p);
  else r1_fold_kernel<float><<<blocks, kFoldThreads, 0, s>>>(p);
  return cudaGetLastError();
}

static cudaError_t r1_chains(const AdjR1Params& p, int dtype, int nblocks, cudaStream_t s) {
  bool small = true;
  for (int k = 0; k < p.n; ++k) small = small && p.step[k].rx <= 64 && p.step[k].rx2 <= 64;
  if (small) {
    count_launch();
    if (dtype == TT_F64) r1_chain64_kernel<double><<<nblocks, kC64Threads, 0, s>>>(p);
    else r1_chain64_kernel<float><<<nblocks, kC64Threads, 0, s>>>(p);
    return cudaGetLastError();
  }
  const size_t esz = dtype == TT_F64 ? 8 : 4;
  const size_t smem = (2 * static_cast<size_t>(kR1MaxRank) + kR1Threads) * esz;
  const void* k = dtype == TT_F64 ? reinterpret_cast<const void*>(r1_chain_kernel<double>)
                                  : reinterpret_cast<const void*>(r1_chain_kernel<float>);
  const cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  count_launch();
  if (dtype == TT_F64) r1_chain_kernel<double><<<nblocks, kR1Threads, smem, s>>>(p);
  else r1_chain_kernel<float><<<nblocks, kR1Threads, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_r1(const AdjR1Params& p, int dtype, cudaStream_t s) {
  if (p.mbuf == nullptr || p.mtbuf == nullptr) return cudaErrorInvalidValue;
  cudaError_t err = r1_fold(p, dtype, s);
  if (err == cudaSuccess) err = r1_chains(p, dtype, 2, s);
  if (err != cudaSuccess) return err;
  int imax = 1;
  for (int k = 0; k < p.n; ++k) imax = std::max(imax, p.step[k].I);
  count_launch();
  if (dtype == TT_F64) r1_grad_kernel<double><<<dim3(imax, p.n), 256, 0, s>>>(p);
  else r1_grad_kernel<float><<<dim3(imax, p.n), 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_full_r1(const AdjR1Params& p, int dtype, cudaStream_t s) {
  if (p.mbuf == nullptr || p.z_out == nullptr || !p.fwd) return cudaErrorInvalidValue;
  AdjR1Params q = p;
  q.mtbuf = nullptr;  // the left chain alone: no transposes
  cudaError_t err = r1_fold(q, dtype, s);
  if (err == cudaSuccess) err = r1_chains(q, dtype, 1, s);
  return err;
}

}  // namespace ttc
