// Partial contraction over any contracted set (Eq. 8 over every mode pair in
// S), merged (TT-matrix) layout.
//
// With free positions f_0 < ... < f_{m-1}, output core t is built from the
// Kronecker pair
//   W_t[(a,b)][i][j][(a',b')] = Gx_{f_t}[a][i][a'] Gy_{f_t}[b][j][b']
// (pair rank index a*R^y + b), with two corrections:
//  * the left environment E_L of the contracted modes before f_0 is folded
//    into W_0:  W_0[0][i][j][(a',b')] = sum_a Gx[a][i][a'] V[a][j][b'],
//    V = E_L Gy (per j, renormalised before the second product);
//  * the contracted run after f_t (modes f_t+1 .. f_{t+1}-1, or up to the
//    end) acts on the right leg of W_t as a linear map M_t:
//      Z_t[(a,b)][i][j][col] = sum_{a',b'} Gx[a][i][a'] Gy[b][j][b'] M_t[(a',b')][col].
//    For an interior run M_t is the run swept from every basis environment
//    e_a' e_b'^T (R^x R^y small sweeps, each row with its own power-of-two
//    scale: transfer_kernel); for a run that reaches the end it is the right
//    environment E_R of one right-to-left sweep.  The product is taken in two
//    steps,
//      P[a][i][b'][col]       = sum_a' Gx[a][i][a'] M_t[(a',b')][col]   (scaled_gemm_kernel)
//      Z_t[(a,b)][i][j][col]  = sum_b' Gy[b][j][b'] P[a][i][b'][col]    (zrows_kernel)
//    so an entry of Z_t costs R^y_{f+1} multiply-adds and the run is swept
//    R^x R^y times instead of once per row of W_t (I J times fewer).  M and P
//    are both kept renormalised (their scales are powers of two applied once,
//    with saturation, to the finished entries), so a run far outside the
//    float range between free cores far inside it still gives finite cores.
// zrows_kernel, which writes the merged cores, is bound by HBM writes; at small
// ranks the short dependent launches before it set the time, and the host
// builds the output cores, which are independent, on forked streams.
#include <limits.h>

#include <algorithm>

#include "ttc_device.cuh"
#include "ttc_internal.h"

namespace ttc {

constexpr int kMT = 256;  // threads of every merged-layout kernel

// s * 2^e with the saturation of scale_pow2_sat, for one e applied to many
// values: the two factors of mul_pow2 are formed once (the same products in
// the same order, so the same roundings).
template <typename T>
struct Pow2Sat {
  T f1, f2;
  int mode;  // 0: s f1 f2;  1: e above the range (+-Inf);  2: e below it (signed zero)
  __device__ explicit Pow2Sat(int64_t e) {
    constexpr int64_t lim = sizeof(T) == 4 ? 250 : 2000;
    mode = e > lim ? 1 : (e < -lim ? 2 : 0);
    const int ei = mode == 0 ? static_cast<int>(e) : 0;
    const int e1 = ei / 2;
    f1 = pow2<T>(e1);
    f2 = pow2<T>(ei - e1);
  }
  __device__ __forceinline__ T operator()(T s) const {
    if (mode == 0) return s * f1 * f2;
    if (s == T(0) || !isfinite(s)) return s;
    return mode == 1 ? (s > T(0) ? T(INFINITY) : T(-INFINITY)) : s * T(0);
  }
};

// ---- left core with E_L folded in ----

// V[a][j][b2] = sum_b E_L[a][b] gy[b][j][b2]   (then W_0 from V)
template <typename T>
__global__ void __launch_bounds__(kMT) kron0_v_kernel(const __grid_constant__ KronParams p) {
  const T* el = static_cast<const T*>(p.el);
  const T* gy = static_cast<const T*>(p.gy);
  T* v = static_cast<T*>(p.tmp);
  const int64_t n = static_cast<int64_t>(p.rx) * p.J * p.ry2;
  int vmax = INT_MIN;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int b2 = static_cast<int>(e % p.ry2);
    const int64_t r = e / p.ry2;
    const int j = static_cast<int>(r % p.J), a = static_cast<int>(r / p.J);
    T s = T(0);
    if (el == nullptr) {  // no contracted mode before the first free one: E_L = [1]
      s = gy[static_cast<int64_t>(j) * p.ry2 + b2];
    } else {
#pragma unroll 4
      for (int b = 0; b < p.ry; ++b) s = fma(el[a * p.ry + b], gy[(static_cast<int64_t>(b) * p.J + j) * p.ry2 + b2], s);
    }
    v[e] = s;
    if (isfinite(s) && s != T(0)) vmax = max(vmax, exp2_bits(s));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) vmax = max(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  if ((threadIdx.x & 31) == 0 && vmax != INT_MIN) atomicMax(reinterpret_cast<long long*>(p.vexp), static_cast<long long>(vmax));
}

// W_0[i][j][(a2*ry2 + b2)] = 2^(lg + ev) * sum_a gx[a][i][a2] 2^-ev V[a][j][b2]
template <typename T>
__global__ void __launch_bounds__(kMT) kron0_w_kernel(const __grid_constant__ KronParams p) {
  const T* gx = static_cast<const T*>(p.gx);
  const T* v = static_cast<const T*>(p.tmp);
  T* w = static_cast<T*>(p.out);
  const int64_t ev = *p.vexp;
  const int64_t lg = (p.el_log2 != nullptr ? *p.el_log2 : 0) + ev;
  if (!p.scale_out && blockIdx.x == 0 && threadIdx.x == 0) *p.wexp = lg;
  const int64_t ncol = static_cast<int64_t>(p.rx2) * p.ry2;
  const int64_t n = static_cast<int64_t>(p.I) * p.J * ncol;
  const Pow2Sat<T> vsc(-ev), osc(lg);
  int bits = 0;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t c = e % ncol;
    const int64_t r = e / ncol;
    const int j = static_cast<int>(r % p.J), i = static_cast<int>(r / p.J);
    const int a2 = static_cast<int>(c / p.ry2), b2 = static_cast<int>(c % p.ry2);
    T s = T(0);
#pragma unroll 4
    for (int a = 0; a < p.rx; ++a)
      s = fma(gx[(static_cast<int64_t>(a) * p.I + i) * p.rx2 + a2], vsc(v[(static_cast<int64_t>(a) * p.J + j) * p.ry2 + b2]), s);
    if (p.scale_out) {
      const T s0 = s;
      s = osc(s);
      if (isfinite(s0) && !isfinite(s)) bits |= TT_STATUS_OVERFLOW;
    }
    if (!isfinite(s)) bits |= TT_STATUS_NONFINITE;
    w[e] = s;
  }
  if (bits) set_status(p.status, bits);
}

// ---- transfer matrix of an interior run ----

// Largest binary exponent over the non-zero entries of v[0, n), block-wide
// (INT_MIN when all are zero); a non-finite entry sets TT_STATUS_NONFINITE.
template <typename T>
__device__ int block_max_exp(const T* v, int n, int* red, int& bits) {
  int m = INT_MIN;
  for (int e = threadIdx.x; e < n; e += kMT) {
    const T x = v[e];
    if (!isfinite(x))
      bits |= TT_STATUS_NONFINITE;
    else if (x != T(0))
      m = max(m, exp2_bits(x));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  int r = red[0];
#pragma unroll
  for (int w = 1; w < kMT / 32; ++w) r = max(r, red[w]);
  __syncthreads();
  return r;
}

// Scale v[0, n) by an exact power of two so that its largest magnitude lies in
// [1/2, 1); returns the exponent taken out (INT_MIN, nothing done, when v = 0).
template <typename T>
__device__ int renorm_block(T* v, int n, int* red, int& bits) {
  const int e = block_max_exp(v, n, red, bits);
  if (e != INT_MIN)
    for (int k = threadIdx.x; k < n; k += kMT) v[k] = mul_pow2<T>(v[k], -e);
  __syncthreads();
  return e;
}

// One CTA per row (a, b) of M (grid-stride).  The first mode starts from the
// basis environment, E[c][d] = sum_i Gx[a][i][c] Gy[b][i][d]; every further
// mode is E' = sum_i A_i^T E B_i, taken as T = E [B_i0 .. B_i1) (a chunk of
// slices, T[c][i][v]) and E' += sum_{c,i} Gx[c][i][u] T[c][i][v].  Shared
// memory: E and E' (e_cap elements each) and the chunk T (t_cap elements,
// t_cap < 2^16 so that udiv16 is exact).
template <typename T>
__global__ void __launch_bounds__(kMT) transfer_kernel(const __grid_constant__ TransferParams p, int e_cap, int t_cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int red[kMT / 32];
  T* const ea = reinterpret_cast<T*>(smem);
  T* const eb = ea + e_cap;
  T* const tb = eb + e_cap;
  const int tid = threadIdx.x;
  const SweepStep& s0 = p.step[0];
  const SweepStep& sl = p.step[p.n_steps - 1];
  const int nq = s0.rin_x * s0.rin_y;
  const int C = sl.rout_x * sl.rout_y;
  int bits = 0;
  for (int q = blockIdx.x; q < nq; q += gridDim.x) {
    const int a = q / s0.rin_y, b = q - a * s0.rin_y;
    T* e = ea;
    T* e2 = eb;
    {
      const T* gx = static_cast<const T*>(s0.gx) + static_cast<int64_t>(a) * s0.I * s0.rout_x;
      const T* gy = static_cast<const T*>(s0.gy) + static_cast<int64_t>(b) * s0.I * s0.rout_y;
      const int n = s0.rout_x * s0.rout_y;
      for (int k = tid; k < n; k += kMT) {
        const int c = udiv16(k, s0.rout_y), d = k - c * s0.rout_y;
        T acc = T(0);
#pragma unroll 8
        for (int i = 0; i < s0.I; ++i) acc = fma(gx[i * s0.rout_x + c], gy[i * s0.rout_y + d], acc);
        e[k] = acc;
      }
    }
    __syncthreads();
    int r = renorm_block(e, s0.rout_x * s0.rout_y, red, bits);
    bool zero = r == INT_MIN;
    int64_t lg = zero ? 0 : r;
    for (int j = 1; j < p.n_steps && !zero; ++j) {
      const SweepStep& st = p.step[j];
      const int rx = st.rin_x, ry = st.rin_y, rx2 = st.rout_x, ry2 = st.rout_y, I = st.I;
      const T* gx = static_cast<const T*>(st.gx);
      const T* gy = static_cast<const T*>(st.gy);
      const int n2 = rx2 * ry2;
      for (int k = tid; k < n2; k += kMT) e2[k] = T(0);
      const int ic = max(1, min(I, t_cap / (rx * ry2)));
      for (int i0 = 0; i0 < I; i0 += ic) {
        const int ni = min(ic, I - i0), w = ni * ry2, nt = rx * w;
        // T[c][ii][v] = sum_d E[c][d] Gy[d][i0 + ii][v]
        for (int k = tid; k < nt; k += kMT) {
          const int c = udiv16(k, w), rem = k - c * w;
          const T* er = e + c * ry;
          const T* gcol = gy + static_cast<int64_t>(i0) * ry2 + rem;
          const int64_t gs = static_cast<int64_t>(I) * ry2;
          T acc = T(0);
#pragma unroll 8
          for (int d = 0; d < ry; ++d) acc = fma(er[d], gcol[d * gs], acc);
          tb[k] = acc;
        }
        __syncthreads();
        // E'[u][v] += sum_c sum_ii Gx[c][i0 + ii][u] T[c][ii][v]
        for (int k = tid; k < n2; k += kMT) {
          const int u = udiv16(k, ry2), v = k - u * ry2;
          T acc = e2[k];
          for (int c = 0; c < rx; ++c) {
            const T* gr = gx + (static_cast<int64_t>(c) * I + i0) * rx2 + u;
            const T* tr = tb + c * w + v;
            for (int ii = 0; ii < ni; ++ii) acc = fma(gr[ii * rx2], tr[ii * ry2], acc);
          }
          e2[k] = acc;
        }
        __syncthreads();
      }
      r = renorm_block(e2, n2, red, bits);
      if (r == INT_MIN)
        zero = true;
      else
        lg += r;
      T* t = e;
      e = e2;
      e2 = t;
    }
    T* mrow = static_cast<T*>(p.m) + static_cast<int64_t>(q) * C;
    for (int k = tid; k < C; k += kMT) mrow[k] = zero ? T(0) : e[k];
    if (tid == 0) {
      const int64_t x = zero ? kMergedZeroExp : lg;
      p.mexp[q] = x;
      atomicMax(reinterpret_cast<long long*>(p.emax), static_cast<long long>(x));
    }
    __syncthreads();  // e is rewritten by the next row
  }
  bits = __syncthreads_or(bits);
  if (tid == 0 && bits) set_status(p.status, bits);
}

// ---- P = Gx M (or W_0 M): a small tiled product with per-row scales of M ----
//
// 16 x 16 outputs per CTA, one per thread (the products here are small, so the
// grid is what needs to be wide), K in chunks of 64; the next chunk's loads are
// in flight while the current one is multiplied.

constexpr int kGT = 16, kGKC = 64;

template <typename T>
__global__ void __launch_bounds__(kMT) scaled_gemm_kernel(const __grid_constant__ ScaledGemmParams p) {
  __shared__ T as[kGKC][kGT + 1];  // A chunk, transposed: as[k][r]
  __shared__ T bs[kGKC][kGT];
  const int tid = threadIdx.x;
  const int tr = tid >> 4, tc = tid & 15;
  const int r0 = blockIdx.x * kGT, c0 = blockIdx.y * kGT, z = blockIdx.z;
  const int64_t em = *p.emax;
  const T* A = static_cast<const T*>(p.a);
  const T* B = static_cast<const T*>(p.b) + z * p.bz;
  constexpr int U = kGT * kGKC / kMT;  // elements of each tile a thread loads
  T ra[U], rb[U];
  int64_t rs[U];
  auto load = [&](int k0) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = tid + u * kMT;
      const int ar = e / kGKC, ak = e - ar * kGKC;  // A: along k
      const int gr = r0 + ar, gk = k0 + ak;
      ra[u] = (gr < p.rows && gk < p.K) ? A[gr * p.lda + gk] : T(0);
      const int bk = e / kGT, bc = e - bk * kGT;  // B: along c
      const int hk = k0 + bk, hc = c0 + bc;
      const bool in = hk < p.K && hc < p.C;
      rb[u] = in ? B[hk * p.ldb + hc] : T(0);
      rs[u] = in ? p.mexp[hk * p.es + z * p.ez] - em : 0;
    }
  };
  T acc = T(0);
  load(0);
  for (int k0 = 0; k0 < p.K; k0 += kGKC) {
    __syncthreads();  // the previous chunk is multiplied
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = tid + u * kMT;
      const int ar = e / kGKC, ak = e - ar * kGKC;
      as[ak][ar] = ra[u];
      const int bk = e / kGT, bc = e - bk * kGT;
      bs[bk][bc] = scale_pow2_sat<T>(rb[u], rs[u]);
    }
    __syncthreads();
    if (k0 + kGKC < p.K) load(k0 + kGKC);
#pragma unroll 16
    for (int k = 0; k < kGKC; ++k) acc = fma(as[k][tr], bs[k][tc], acc);
  }
  const int r = r0 + tr, c = c0 + tc;
  int bits = 0, omax = INT_MIN;
  if (r < p.rows && c < p.C) {
    T val = acc;
    if (p.out_log2 != nullptr) {
      const T v0 = val;
      val = Pow2Sat<T>(*p.out_log2 + em)(val);
      if (isfinite(v0) && !isfinite(val)) bits |= TT_STATUS_OVERFLOW;
    }
    if (!isfinite(val))
      bits |= TT_STATUS_NONFINITE;
    else if (val != T(0))
      omax = exp2_bits(val);
    static_cast<T*>(p.out)[z * p.oz + r * p.ldo + c] = val;
  }
  if (bits) set_status(p.status, bits);
  if (p.oexp != nullptr) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) omax = max(omax, __shfl_xor_sync(0xffffffffu, omax, o));
    if ((tid & 31) == 0 && omax != INT_MIN)
      atomicMax(reinterpret_cast<long long*>(p.oexp), static_cast<long long>(omax));
  }
}

// ---- rows of a merged core ----

template <typename T, int VW>
struct alignas(sizeof(T) * VW) Pack {
  T v[VW];
};

constexpr int kZRR = 4;  // rows a thread carries at once

// Block (a, i) = blockIdx.x, rows (b, j) in chunks of rb (blockIdx.y, grid
// stride), columns [c0, c0 + ct) with c0 = blockIdx.z * ct.  A thread owns VW
// adjacent columns (g) of every NL-th row of the chunk; the Gy rows of the
// chunk (rows b J + j, contiguous in the core) and, for prod, the P tile of
// (a, i) sit in shared memory.  VW > 1 only when the columns, the output rows
// and (kron) the Gy rows are 16-byte aligned.
template <typename T, bool PROD, int VW>
__global__ void __launch_bounds__(kMT) zrows_kernel(const __grid_constant__ ZRowsParams p, int ct, int rb) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x;
  const int ry2 = p.ry2, C = p.C;
  T* gys = reinterpret_cast<T*>(smem);  // [rb][ry2]
  T* ps = reinterpret_cast<T*>(smem + ((static_cast<size_t>(rb) * ry2 * sizeof(T) + 15) & ~static_cast<size_t>(15)));
  const int ai = blockIdx.x;
  const int a = ai / p.I, i = ai - a * p.I;
  const int c0 = blockIdx.z * ct;
  const int ncol = min(ct, C - c0);
  const int G = (ct + VW - 1) / VW, NL = kMT / G;
  const int g = tid % G, lane = tid / G;
  const int col = c0 + g * VW;
  const bool active = lane < NL && g * VW < ncol;
  const int nrho = p.ry * p.J;
  const int64_t ep = PROD ? *p.ep : 0;
  if (PROD) {
    // the P tile of (a, i), all copies in flight at once, then 2^-ep in place
    const T* P = static_cast<const T*>(p.p) + static_cast<int64_t>(ai) * ry2 * C + c0;
    const int cv = ct / VW;
    for (int e = tid; e < ry2 * cv; e += kMT) {
      const int bp = e / cv, c = (e - bp * cv) * VW;
      if (c < ncol) {
        if (VW > 1)
          cp_async16(ps + bp * ct + c, P + static_cast<int64_t>(bp) * C + c);
        else
          cp_async_elem(ps + bp * ct + c, P + static_cast<int64_t>(bp) * C + c);
      }
    }
    cp_async_commit();  // completes with the first chunk's Gy rows
  }
  T gxv = T(0);
  int d0 = 0;
  if (!PROD && active) {
    const int c = col / ry2;
    d0 = col - c * ry2;
    gxv = static_cast<const T*>(p.gx)[static_cast<int64_t>(ai) * p.rx2 + c];
  }
  const Pow2Sat<T> zsc(PROD ? *p.e + ep : 0);
  const int64_t IJ = static_cast<int64_t>(p.I) * p.J;
  T* const out = static_cast<T*>(p.out) + (static_cast<int64_t>(a) * p.ry * IJ + static_cast<int64_t>(i) * p.J) * C + col;
  int bits = 0;
  bool first = true;
  for (int yb = blockIdx.y; static_cast<int64_t>(yb) * rb < nrho; yb += gridDim.y) {
    const int rho0 = yb * rb, nr = min(rb, nrho - rho0);
    __syncthreads();  // the previous chunk's rows are consumed
    const T* gy = static_cast<const T*>(p.gy) + static_cast<int64_t>(rho0) * ry2;
    for (int e = tid; e < nr * ry2; e += kMT) cp_async_elem(gys + e, gy + e);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    if (PROD && first) {  // P's tile to scale 2^-ep, in place
      const Pow2Sat<T> psc(-ep);
      for (int e = tid; e < ry2 * ct; e += kMT) {
        const int c = e - (e / ct) * ct;
        ps[e] = c < ncol ? psc(ps[e]) : T(0);
      }
      __syncthreads();
    }
    first = false;
    if (!active) continue;
    for (int rl = lane; rl < nr; rl += NL * kZRR) {
      Pack<T, VW> res[kZRR];
      if (PROD) {
        T acc[kZRR][VW];
#pragma unroll
        for (int q = 0; q < kZRR; ++q)
#pragma unroll
          for (int v = 0; v < VW; ++v) acc[q][v] = T(0);
        const T* grow[kZRR];
#pragma unroll
        for (int q = 0; q < kZRR; ++q) grow[q] = gys + min(rl + q * NL, nr - 1) * ry2;
        for (int bp = 0; bp < ry2; ++bp) {
          const Pack<T, VW> pv = *reinterpret_cast<const Pack<T, VW>*>(ps + bp * ct + g * VW);
#pragma unroll
          for (int q = 0; q < kZRR; ++q) {
            const T gv = grow[q][bp];
#pragma unroll
            for (int v = 0; v < VW; ++v) acc[q][v] = fma(gv, pv.v[v], acc[q][v]);
          }
        }
#pragma unroll
        for (int q = 0; q < kZRR; ++q) {
          const bool live = rl + q * NL < nr;  // rows past the chunk repeat its last row
#pragma unroll
          for (int v = 0; v < VW; ++v) {
            const T s0 = acc[q][v];
            const T s = zsc(s0);
            if (live && isfinite(s0) && !isfinite(s)) bits |= TT_STATUS_OVERFLOW;
            if (live && !isfinite(s)) bits |= TT_STATUS_NONFINITE;
            res[q].v[v] = s;
          }
        }
      } else {
#pragma unroll
        for (int q = 0; q < kZRR; ++q) {
          const Pack<T, VW> gv = *reinterpret_cast<const Pack<T, VW>*>(gys + min(rl + q * NL, nr - 1) * ry2 + d0);
#pragma unroll
          for (int v = 0; v < VW; ++v) res[q].v[v] = gxv * gv.v[v];
        }
      }
#pragma unroll
      for (int q = 0; q < kZRR; ++q) {
        const int row = rl + q * NL;
        if (row < nr) {
          const int rho = rho0 + row;
          const int b = rho / p.J, j = rho - b * p.J;
          *reinterpret_cast<Pack<T, VW>*>(out + (b * IJ + j) * C) = res[q];
        }
      }
    }
  }
  if (bits) set_status(p.status, bits);
}

// ---- launches ----

static int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

template <typename T>
static cudaError_t kron0_impl(const KronParams& p, int which, cudaStream_t s) {
  const int grid = sm_count() * 8;
  count_launch();
  if (which == 1)
    kron0_v_kernel<T><<<grid, kMT, 0, s>>>(p);
  else
    kron0_w_kernel<T><<<grid, kMT, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_kron0(const KronParams& p, int which, int dtype, cudaStream_t s) {
  return dtype == TT_F64 ? kron0_impl<double>(p, which, s) : kron0_impl<float>(p, which, s);
}

template <typename T>
static cudaError_t transfer_impl(const TransferParams& p, cudaStream_t s) {
  int e_cap = 1, t_need = 1, t_min = 1;
  for (int j = 0; j < p.n_steps; ++j) {
    const SweepStep& st = p.step[j];
    e_cap = std::max({e_cap, st.rin_x * st.rin_y, st.rout_x * st.rout_y});
    if (j > 0) {
      t_need = std::max(t_need, st.rin_x * st.I * st.rout_y);
      t_min = std::max(t_min, st.rin_x * st.rout_y);
    }
  }
  const int budget = static_cast<int>(200 * 1024 / sizeof(T)) - 2 * e_cap;
  const int t_cap = std::min({t_need, budget, 32768});
  if (t_cap < t_min) return cudaErrorInvalidValue;
  const size_t smem = (2 * static_cast<size_t>(e_cap) + t_cap) * sizeof(T);
  cudaError_t err =
      cudaFuncSetAttribute(transfer_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  int per = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, transfer_kernel<T>, kMT, smem);
  if (err != cudaSuccess) return err;
  const int nq = p.step[0].rin_x * p.step[0].rin_y;
  const int grid = std::min(nq, sm_count() * std::max(per, 1));
  count_launch();
  transfer_kernel<T><<<grid, kMT, smem, s>>>(p, e_cap, t_cap);
  return cudaGetLastError();
}

cudaError_t launch_transfer(const TransferParams& p, int dtype, cudaStream_t s) {
  if (p.n_steps < 1) return cudaErrorInvalidValue;
  return dtype == TT_F64 ? transfer_impl<double>(p, s) : transfer_impl<float>(p, s);
}

template <typename T>
static cudaError_t gemm_impl(const ScaledGemmParams& p, cudaStream_t s) {
  const dim3 grid((p.rows + kGT - 1) / kGT, (p.C + kGT - 1) / kGT, p.nz);
  count_launch();
  scaled_gemm_kernel<T><<<grid, kMT, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_scaled_gemm(const ScaledGemmParams& p, int dtype, cudaStream_t s) {
  if (p.rows < 1 || p.C < 1 || p.nz < 1 || (p.C + kGT - 1) / kGT > 65535 || p.nz > 65535) return cudaErrorInvalidValue;
  return dtype == TT_F64 ? gemm_impl<double>(p, s) : gemm_impl<float>(p, s);
}

template <typename T, bool PROD, int VW>
static cudaError_t zrows_impl(const ZRowsParams& p, cudaStream_t s) {
  const int ct = std::min(p.C, 64 * VW);
  const int G = (ct + VW - 1) / VW, NL = kMT / G;
  const int rb_cap = std::max(1, static_cast<int>(65536 / (static_cast<size_t>(p.ry2) * sizeof(T))));
  const int rb = std::min(std::max(32, NL * kZRR), rb_cap);
  size_t smem = (static_cast<size_t>(rb) * p.ry2 * sizeof(T) + 15) & ~static_cast<size_t>(15);
  if (PROD) smem += static_cast<size_t>(p.ry2) * ct * sizeof(T);
  cudaError_t err = cudaFuncSetAttribute(zrows_kernel<T, PROD, VW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  const int64_t nrho = static_cast<int64_t>(p.ry) * p.J;
  const dim3 grid(static_cast<unsigned>(static_cast<int64_t>(p.rx) * p.I),
                  static_cast<unsigned>(std::min<int64_t>((nrho + rb - 1) / rb, 65535)),
                  static_cast<unsigned>((p.C + ct - 1) / ct));
  count_launch();
  zrows_kernel<T, PROD, VW><<<grid, kMT, smem, s>>>(p, ct, rb);
  return cudaGetLastError();
}

template <typename T, bool PROD>
static cudaError_t zrows_pick(const ZRowsParams& p, cudaStream_t s) {
  constexpr int VW = 16 / static_cast<int>(sizeof(T));
  const bool vec = p.C % VW == 0 && (PROD || p.ry2 % VW == 0) && (reinterpret_cast<uintptr_t>(p.out) & 15) == 0;
  return vec ? zrows_impl<T, PROD, VW>(p, s) : zrows_impl<T, PROD, 1>(p, s);
}

cudaError_t launch_zrows(const ZRowsParams& p, bool prod, int dtype, cudaStream_t s) {
  if (p.rx < 1 || p.ry < 1 || p.I < 1 || p.J < 1 || p.C < 1 || p.ry2 < 1) return cudaErrorInvalidValue;
  if (static_cast<int64_t>(p.rx) * p.I > INT_MAX || (p.C + 63) / 64 > 65535) return cudaErrorInvalidValue;
  if (dtype == TT_F64) return prod ? zrows_pick<double, true>(p, s) : zrows_pick<double, false>(p, s);
  return prod ? zrows_pick<float, true>(p, s) : zrows_pick<float, false>(p, s);
}

}  // namespace ttc
