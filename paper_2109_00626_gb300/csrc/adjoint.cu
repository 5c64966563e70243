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
// dGy_i = L^T W.
//
// Order of work: the environments are formed by two ordinary environment
// sweeps (the sweep kernel of the forward contraction, started from the
// seeds and storing the environment before every mode): L_1..L_{n-1} left to
// right (the forward sweep of a partial contraction has already stored them)
// and F_{n-1}..F_1 right to left, F_k = sum_i Gx_i F_{k+1} Gy_i^T.  Then
// adjoint_grads_kernel forms the gradients of every (mode, slice) at once,
// two blocks each (dGx, dGy): the gradient products are off the sweeps'
// dependent path and spread over the whole GPU.  Workspace: 2n environments
// and leg-swapped copies of the block's cores.
#include "copy_jobs.cuh"
#include "ttc_device.cuh"
#include "ttc_internal.h"

namespace ttc {

namespace {

template <typename T, int RM>
struct AdjCfg {
  static constexpr int NT = 256;
  static constexpr int TM = RM / 16;
  static constexpr int V = 16 / sizeof(T);
  static constexpr int LD = RM + V;
  static constexpr int TILE = RM * LD;
  // the gradient blocks: L, F, one slice, one intermediate
  static constexpr size_t SMEM = 4 * TILE * sizeof(T);
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

// Load an environment (row-major [nu][nv] in global memory; the sum of
// `parts` consecutive such matrices, added in order) into D as [u][v], or
// as [v][u] when transposed.
template <typename T, int LD, int NT>
__device__ void load_env1(const T* src, int nu, int nv, T* D, bool transposed, int parts = 1) {
  sum_parts<T, NT>(src, nu * nv, parts > 1 ? parts : 1, [&](int idx, T e) {
    const int u = idx / nv, v = idx - u * nv;
    if (transposed) D[v * LD + u] = e;
    else D[u * LD + v] = e;
  });
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

// The gradients of every (mode k, slice i), two blocks each:
//   kind 0: U = L_k Gy_i,   dGx_i = U F_{k+1}^T,
//   kind 1: W = Gx_i F_{k+1}, dGy_i = L_k^T W,
// scaled by cot * 2^(log2 L_k + log2 F_{k+1}).  Four tiles of shared memory a
// block, so several blocks share an SM.
template <typename T, int RM>
__global__ void __launch_bounds__(256, 2) adjoint_grads_kernel(const __grid_constant__ AdjointParams p) {
  using Cfg = AdjCfg<T, RM>;
  constexpr int NT = Cfg::NT, TM = Cfg::TM, LD = Cfg::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Lt = reinterpret_cast<T*>(smem_raw);  // kind 0: L[b][a]      kind 1: L[a][b]
  T* Ft = Lt + Cfg::TILE;                  // kind 0: F[b'][a']    kind 1: F[a'][b']
  T* Sl = Ft + Cfg::TILE;                  // kind 0: Gy_i[b][b']  kind 1: Gx_i[a'][a]
  T* X1 = Sl + Cfg::TILE;                  // kind 0: U^T[b'][a]   kind 1: W[a][b']
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  const int u0 = ty * TM, v0 = tx * TM;
  const int kind = static_cast<int>(blockIdx.x) & 1;
  int k = 0, i = static_cast<int>(blockIdx.x) >> 1;
  while (k + 1 < p.n && i >= p.step[k].I) {
    i -= p.step[k].I;
    ++k;
  }
  const AdjStep& st = p.step[k];
  if (kind == 0)
    slice_async<T, LD, NT>(Sl, static_cast<const T*>(st.gy), i, st.I, st.ry, st.ry2, 0);  // [b][b']
  else if (st.gxs != nullptr)  // [a'][a] from the leg-swapped copy, 16 bytes a copy
    slice_async<T, LD, NT>(Sl, static_cast<const T*>(st.gxs), i, st.I, st.rx2, st.rx, 0);
  else
    slice_async<T, LD, NT>(Sl, static_cast<const T*>(st.gx), i, st.I, st.rx2, st.rx, 1);
  cp_async_commit();
  // L_k and F_{k+1} in the orientation this kind reads: stored by the
  // sweeps, or the seeds at the block's ends
  const bool tr = kind == 0;
  int64_t esum = 0;
  if (k > 0) {
    load_env1<T, LD, NT>(static_cast<const T*>(p.lenv) + k * p.env_elems, st.rx, st.ry, Lt, tr);
    esum += p.lenv_log2[k];
  } else if (p.l_seed != nullptr) {
    load_env1<T, LD, NT>(static_cast<const T*>(p.l_seed), st.rx, st.ry, Lt, tr, p.seed_parts);
    if (p.l_seed_log2 != nullptr) esum += *p.l_seed_log2;
  } else if (tid == 0) {
    Lt[0] = T(1);
  }
  if (k + 1 < p.n) {
    load_env1<T, LD, NT>(static_cast<const T*>(p.fenv) + k * p.env_elems, st.rx2, st.ry2, Ft, tr);
    esum += p.fenv_log2[p.n - 1 - k];
  } else if (p.f_seed != nullptr) {
    load_env1<T, LD, NT>(static_cast<const T*>(p.f_seed), st.rx2, st.ry2, Ft, tr, p.seed_parts);
    if (p.f_seed_log2 != nullptr) esum += *p.f_seed_log2;
  } else if (tid == 0) {
    Ft[0] = T(1);
  }
  cp_async_wait<0>();
  __syncthreads();
  const double gbar = p.cot != nullptr ? *p.cot : 1.0;
  esum = esum < -4000 ? -4000 : (esum > 4000 ? 4000 : esum);
  const double fac = ldexp(gbar, static_cast<int>(esum));
  // float gradients are scaled in float: fac = fm * 2^fe with fm the
  // float-rounded mantissa of gbar
  int ge = 0;
  const float fm = static_cast<float>(frexp(gbar, &ge));
  const int fe = ge + static_cast<int>(esum);
  int sbits = 0;
  T t[TM][TM];
  if (kind == 0) {
    // U[a][b'] = L Gy_i : A = L^T[b][a], B = Gy[b][b'] -> X1 as U^T[b'][a]
    zero<T, TM>(t);
    if (u0 < st.rx && v0 < st.ry2) op_acc<T, TM, LD>(t, Lt, Sl, st.ry, u0, v0);
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TM; ++b) X1[(v0 + b) * LD + u0 + a] = t[a][b];
    __syncthreads();
    // dGx[a][a'] = U F^T : A = U^T[b'][a], B = F^T[b'][a']
    zero<T, TM>(t);
    if (u0 < st.rx && v0 < st.rx2) op_acc<T, TM, LD>(t, X1, Ft, st.ry2, u0, v0);
    T* dgx = static_cast<T*>(st.dgx);
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TM; ++b)
        if (u0 + a < st.rx && v0 + b < st.rx2)
          dgx[(static_cast<int64_t>(u0 + a) * st.I + i) * st.rx2 + v0 + b] = grad_out<T>(t[a][b], fac, fm, fe, sbits);
  } else {
    // W[a][b'] = Gx_i F : A = Gx^T[a'][a], B = F[a'][b']
    zero<T, TM>(t);
    if (u0 < st.rx && v0 < st.ry2) op_acc<T, TM, LD>(t, Sl, Ft, st.rx2, u0, v0);
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TM; ++b) X1[(u0 + a) * LD + v0 + b] = t[a][b];
    __syncthreads();
    // dGy[b][b'] = L^T W : A = L[a][b], B = W[a][b']
    zero<T, TM>(t);
    if (u0 < st.ry && v0 < st.ry2) op_acc<T, TM, LD>(t, Lt, X1, st.rx, u0, v0);
    T* dgy = static_cast<T*>(st.dgy);
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TM; ++b)
        if (u0 + a < st.ry && v0 + b < st.ry2)
          dgy[(static_cast<int64_t>(u0 + a) * st.I + i) * st.ry2 + v0 + b] = grad_out<T>(t[a][b], fac, fm, fe, sbits);
  }
  if (sbits) set_status(p.status, sbits);
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

template <typename T>
__global__ void __launch_bounds__(kCopyThreads) swap_copies_kernel(const __grid_constant__ SwapParams p) {
  extern __shared__ __align__(16) unsigned char swap_smem[];
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
  T* const buf0 = reinterpret_cast<T*>(swap_smem);
  copy_jobs_block<T>(job_of, blockIdx.x, p.n_jobs, gridDim.x, buf0, buf0 + copy_buf_elems<T>());
}

cudaError_t launch_swap_copies(const SwapParams& p, int dtype, cudaStream_t s) {
  const int eb = dtype == TT_F64 ? 8 : 4;
  SwapParams q = p;
  q.n_jobs = 0;
  for (int t = 0; t < p.n_copies; ++t) {
    if (p.copy[t].r1 > kCopyJobBytes / eb) return cudaErrorInvalidValue;  // a slice row must fit a job
    const CopyCut cut = copy_cut(p.copy[t].r0, p.copy[t].I, p.copy[t].r1, eb);
    q.n_jobs += cut.n_i * cut.n_a;
  }
  if (q.n_jobs < 1) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::min(q.n_jobs, 2 * std::max(sms, 1));
  const size_t smem = dtype == TT_F64 ? copy_smem_bytes<double>() : copy_smem_bytes<float>();
  cudaError_t err = dtype == TT_F64 ? cudaFuncSetAttribute(swap_copies_kernel<double>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                           static_cast<int>(smem))
                                    : cudaFuncSetAttribute(swap_copies_kernel<float>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                           static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  count_launch();
  if (dtype == TT_F64) swap_copies_kernel<double><<<grid, kCopyThreads, smem, s>>>(q);
  else swap_copies_kernel<float><<<grid, kCopyThreads, smem, s>>>(q);
  return cudaGetLastError();
}

template <typename T, int RM>
static cudaError_t adjoint_grads_impl(const AdjointParams& p, cudaStream_t s) {
  const size_t smem = AdjCfg<T, RM>::SMEM;
  const cudaError_t err = cudaFuncSetAttribute(adjoint_grads_kernel<T, RM>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  count_launch();
  adjoint_grads_kernel<T, RM><<<2 * p.total_slices, 256, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_grads(const AdjointParams& p, int dtype, int rmax, cudaStream_t s) {
  if (p.n < 1 || p.total_slices < 1) return cudaErrorInvalidValue;
  if (dtype == TT_F64) {
    if (rmax <= 16) return adjoint_grads_impl<double, 16>(p, s);
    return adjoint_grads_impl<double, 32>(p, s);
  }
  if (rmax <= 32) return adjoint_grads_impl<float, 32>(p, s);
  return adjoint_grads_impl<float, 64>(p, s);
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
