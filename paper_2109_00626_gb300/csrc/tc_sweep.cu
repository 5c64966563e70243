// Full contraction on the tensor cores (bfloat16 products, float32 sums), for
// ranks that make each step a real GEMM (interior ranks multiples of 128 on X
// and of 64 on Y, at most 256).
//
// Each interior mode k is one launch (programmatic dependent launch: the next
// mode's CTAs set up while this one finishes).  Its work, E' = sum_i Gx_i^T (E Gy_i),
// is split over 64-column blocks of E' (one thread-block cluster per block)
// and, inside a cluster, over the mode index i (CTA c owns i = c, c + C, ...).
// Per slice a CTA runs two chained tcgen05 GEMMs:
//   GEMM1  T = E Gy_i[:, vblk]      A = E (K-major), B = Gy slice (MN-major)
//   GEMM2  P += Gx_i^T T            A = Gx slice (MN-major), B = T (MN-major)
// with T and P accumulated in tensor memory.  One warp streams E panels (bulk
// copies) and core tiles (TMA, 128-byte swizzle) through an mbarrier ring; one
// thread issues the MMAs; four warps drain T from tensor memory, round it to
// bfloat16 and stage it as GEMM2's operand, and at the end drain P.  The
// native variant keeps two T buffers and issues GEMM1 of the next slice before
// GEMM2 of the current one, so a slice's T drain overlaps the next GEMM1.  The
// cluster then sums the per-CTA P's through distributed shared memory and
// writes E' both in float32 and as the bfloat16 K-major panels the next mode
// streams in.
//
// The split-bfloat16 variant keeps every float32 operand as hi + lo bfloat16
// pieces and issues three products per step (hi*hi + hi*lo + lo*hi).
//
// Scaling: each mode divides its output by 2^M, M being the largest binary
// exponent of its input environment (collected per CTA by the previous mode),
// and carries M in the int64 log2 scale, so magnitudes stay within a mode's
// growth of 1 however long the train is.  The first mode (rank 1 on the left)
// and the last mode (float64 sum to the scalar) run on CUDA cores.
#include <cooperative_groups.h>

#include "tc_common.cuh"
#include "ttc_device.cuh"
#include "ttc_internal.h"

namespace cg = cooperative_groups;

namespace ttc {

constexpr int kTcThreads = 192;   // warp 0 producer, warp 1 MMA, warps 2-5 epilogue
constexpr int kNoExpT = -(1 << 30);

template <bool X3>
struct TcCfg {
  static constexpr int NST = X3 ? 2 : 4;
  static constexpr uint32_t STG = X3 ? 81920u : 40960u;
  static constexpr uint32_t OFF_A_HI = 0;                     // E panel / Gx tile
  static constexpr uint32_t OFF_A_LO = 32768;
  static constexpr uint32_t OFF_B_HI = X3 ? 65536u : 32768u;  // Gy tile
  static constexpr uint32_t OFF_B_LO = OFF_B_HI + 8192u;
  // T buffers (tensor memory and the bf16 staging GEMM2 reads): with two, the
  // next slice's GEMM1 runs while this slice's T is drained (no room for a
  // second pair of hi / lo staging buffers in the split variant)
  static constexpr int NTB = X3 ? 1 : 2;
  static constexpr uint32_t OFF_T = NST * STG;                // T hi (and lo), per buffer
  static constexpr uint32_t T_BYTES = 32768;
  static constexpr uint32_t T_STAGE = (X3 ? 2 : 1) * T_BYTES;
  static constexpr uint32_t OFF_BAR = OFF_T + NTB * T_STAGE;
  static constexpr uint32_t TMEM_COLS = NTB == 2 ? 512 : 256;  // T buffers of 128 columns, then P
  static constexpr size_t SMEM = OFF_BAR + 256 + 1024;        // barriers + alignment slack
};

template <bool X3>
__global__ void __launch_bounds__(kTcThreads, 1) tc_mode_kernel(const __grid_constant__ TcModeParams p) {
  using Cfg = TcCfg<X3>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + Cfg::OFF_BAR);
  uint64_t* empty = full + Cfg::NST;
  uint64_t* t_full = empty + Cfg::NST;   // [NTB]
  uint64_t* t_ready = t_full + Cfg::NTB;  // [NTB]
  uint64_t* t_free = t_ready + Cfg::NTB;  // [NTB]
  uint64_t* p_full = t_free + Cfg::NTB;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(p_full + 1);
  int* sh_int = reinterpret_cast<int*>(tmem_slot + 1);  // [0] status bits, [1] M, [2..9] warp maxima, [10] abort
  volatile int* abort = sh_int + 10;

  cg::cluster_group cluster = cg::this_cluster();
  const int C = static_cast<int>(cluster.num_blocks());
  const int crank = static_cast<int>(cluster.block_rank());
  const int vblk = blockIdx.x / C;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int MT1 = p.rx / 128, MT2 = p.rx2 / 128;
  const int NPY = p.ry / 64, NPX = p.rx / 64;
  const int nslices = crank < p.I ? (p.I - 1 - crank) / C + 1 : 0;

  if (warp == 0) tc::tmem_alloc(tmem_slot, Cfg::TMEM_COLS);
  if (tid == 32) {
    for (int s = 0; s < Cfg::NST; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < Cfg::NTB; ++b) {
      tc::mbar_init(&t_full[b], 1);
      tc::mbar_init(&t_ready[b], 128);
      tc::mbar_init(&t_free[b], 1);
    }
    tc::mbar_init(p_full, 1);
    tc::mbar_init_fence();
  }
  if (tid == 64) {
    sh_int[0] = 0;
    sh_int[10] = 0;
  }
  // Launched with programmatic stream serialisation: the next mode's grid may
  // start its set-up (tensor memory, barriers) on idle SMs now; it waits below
  // for this grid's results before touching global memory.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  asm volatile("griddepcontrol.wait;" ::: "memory");  // the previous mode's E, maxima and scale are complete
  if (tid == 64) {
    int m = kNoExpT;
    for (int q = 0; q < p.n_bmax_in; ++q) m = max(m, p.bmax_in[q]);
    sh_int[1] = m == kNoExpT ? 0 : m;
  }
  __syncthreads();
  const uint32_t tmem = *tmem_slot;
  const uint32_t tmem_T = tmem, tmem_P = tmem + Cfg::NTB * 128;  // T buffer b at tmem_T + 128 b
  // Slice order of the operand ring (producer and MMA issuer alike): step t
  // takes GEMM1 of slice t and GEMM2 of slice t - LAG, so with two T buffers
  // GEMM1 of the next slice overlaps the drain of this slice's T.
  constexpr int LAG = Cfg::NTB - 1;
  int bits = 0;

  if (warp == 0) {
    // ---------------- producer ----------------
    if (lane == 0) {
      uint32_t it = 0;
      for (int t = 0; t < nslices + LAG; ++t) {
        if (t < nslices) {
          const int i = crank + t * C;
          for (int kp = 0; kp < NPY; ++kp, ++it) {
            const int s = it % Cfg::NST;
            const uint32_t round = it / Cfg::NST;
            if (!tc::mbar_wait(&empty[s], (round & 1) ^ 1, abort)) bits |= TT_STATUS_TIMEOUT;
            unsigned char* st = sm + s * Cfg::STG;
            const uint32_t eb = static_cast<uint32_t>(p.rx) * 128;
            tc::mbar_expect_tx(&full[s], (X3 ? 2 : 1) * (eb + 8192));
            tc::bulk_load(st + Cfg::OFF_A_HI, p.e_hi + static_cast<size_t>(kp) * p.rx * 64, eb, &full[s]);
            tc::tma_load_3d(st + Cfg::OFF_B_HI, &p.gy_hi, 64 * vblk, i, 64 * kp, &full[s]);
            if (X3) {
              tc::bulk_load(st + Cfg::OFF_A_LO, p.e_lo + static_cast<size_t>(kp) * p.rx * 64, eb, &full[s]);
              tc::tma_load_3d(st + Cfg::OFF_B_LO, &p.gy_lo, 64 * vblk, i, 64 * kp, &full[s]);
            }
          }
        }
        if (t >= LAG) {
          const int i = crank + (t - LAG) * C;
          for (int kp = 0; kp < NPX; ++kp, ++it) {
            const int s = it % Cfg::NST;
            const uint32_t round = it / Cfg::NST;
            if (!tc::mbar_wait(&empty[s], (round & 1) ^ 1, abort)) bits |= TT_STATUS_TIMEOUT;
            unsigned char* st = sm + s * Cfg::STG;
            const int nmb = p.rx2 / 64;
            tc::mbar_expect_tx(&full[s], (X3 ? 2 : 1) * nmb * 8192);
            for (int mb = 0; mb < nmb; ++mb) {
              tc::tma_load_3d(st + Cfg::OFF_A_HI + mb * 8192, &p.gx_hi, 64 * mb, i, 64 * kp, &full[s]);
              if (X3) tc::tma_load_3d(st + Cfg::OFF_A_LO + mb * 8192, &p.gx_lo, 64 * mb, i, 64 * kp, &full[s]);
            }
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr uint32_t id1 = tc::idesc_bf16(128, 64, false, true);
      constexpr uint32_t id2 = tc::idesc_bf16(128, 64, true, true);
      uint32_t it = 0;
      for (int t = 0; t < nslices + LAG; ++t) {
        if (t < nslices) {
          // GEMM1 of slice t into T buffer t % NTB (its previous contents were
          // drained before GEMM2 of slice t - NTB, issued earlier)
          const uint32_t tT = tmem_T + (t % Cfg::NTB) * 128;
          for (int kp = 0; kp < NPY; ++kp, ++it) {
            const int s = it % Cfg::NST;
            if (!tc::mbar_wait(&full[s], (it / Cfg::NST) & 1, abort)) bits |= TT_STATUS_TIMEOUT;
            tc::fence_after_sync();
            const uint32_t st = tc::su32(sm + s * Cfg::STG);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
              for (int mt = 0; mt < MT1; ++mt) {
                const uint32_t acc = (kp | ks) != 0;
                const uint64_t a = tc::sdesc(st + Cfg::OFF_A_HI + mt * 128 * 128 + ks * 32, 16, 1024);
                const uint64_t b = tc::sdesc(st + Cfg::OFF_B_HI + ks * 2048, 8192, 1024);
                tc::mma_bf16(tT + mt * 64, a, b, id1, acc);
                if (X3) {
                  const uint64_t al = tc::sdesc(st + Cfg::OFF_A_LO + mt * 128 * 128 + ks * 32, 16, 1024);
                  const uint64_t bl = tc::sdesc(st + Cfg::OFF_B_LO + ks * 2048, 8192, 1024);
                  tc::mma_bf16(tT + mt * 64, a, bl, id1, 1);
                  tc::mma_bf16(tT + mt * 64, al, b, id1, 1);
                }
              }
            tc::mma_commit(&empty[s]);
          }
          tc::mma_commit(&t_full[t % Cfg::NTB]);
        }
        const int u = t - LAG;
        if (u >= 0) {
          // GEMM2 of slice u from the bf16 staging of T buffer u % NTB
          const int tbuf = u % Cfg::NTB;
          if (!tc::mbar_wait(&t_ready[tbuf], (u / Cfg::NTB) & 1, abort)) bits |= TT_STATUS_TIMEOUT;
          tc::fence_after_sync();
          const uint32_t tb = tc::su32(sm + Cfg::OFF_T + tbuf * Cfg::T_STAGE);
          for (int kp = 0; kp < NPX; ++kp, ++it) {
            const int s = it % Cfg::NST;
            if (!tc::mbar_wait(&full[s], (it / Cfg::NST) & 1, abort)) bits |= TT_STATUS_TIMEOUT;
            tc::fence_after_sync();
            const uint32_t st = tc::su32(sm + s * Cfg::STG);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
              for (int mt = 0; mt < MT2; ++mt) {
                const uint32_t acc = (u | kp | ks) != 0;
                const uint64_t a = tc::sdesc(st + Cfg::OFF_A_HI + (2 * mt) * 8192 + ks * 2048, 8192, 1024);
                const uint64_t b = tc::sdesc(tb + (64 * kp + 16 * ks) * 128, 8192, 1024);
                tc::mma_bf16(tmem_P + mt * 64, a, b, id2, acc);
                if (X3) {
                  const uint64_t al = tc::sdesc(st + Cfg::OFF_A_LO + (2 * mt) * 8192 + ks * 2048, 8192, 1024);
                  const uint64_t bl = tc::sdesc(tb + Cfg::T_BYTES + (64 * kp + 16 * ks) * 128, 8192, 1024);
                  tc::mma_bf16(tmem_P + mt * 64, a, bl, id2, 1);
                  tc::mma_bf16(tmem_P + mt * 64, al, b, id2, 1);
                }
              }
            tc::mma_commit(&empty[s]);
          }
          tc::mma_commit(&t_free[tbuf]);
        }
      }
      tc::mma_commit(p_full);
    }
  } else {
    // ---------------- epilogue: T -> bf16 operand of GEMM2 ----------------
    const int q = warp & 3;  // tensor-memory lane quadrant of this warp
    for (int sl = 0; sl < nslices; ++sl) {
      const int tbuf = sl % Cfg::NTB;
      const uint32_t ph = (sl / Cfg::NTB) & 1;
      unsigned char* tsm = sm + Cfg::OFF_T + tbuf * Cfg::T_STAGE;
      const uint32_t tT = tmem_T + tbuf * 128;
      if (!tc::mbar_wait(&t_full[tbuf], ph, abort)) bits |= TT_STATUS_TIMEOUT;
      tc::fence_after_sync();
      // this staging buffer was last read by GEMM2 of slice sl - NTB
      if (sl >= Cfg::NTB && !tc::mbar_wait(&t_free[tbuf], ph ^ 1, abort)) bits |= TT_STATUS_TIMEOUT;
      for (int mt = 0; mt < MT1; ++mt) {
        const int row = mt * 128 + q * 32 + lane;
#pragma unroll
        for (int c16 = 0; c16 < 4; ++c16) {
          float v[16];
          tc::tmem_ld16(tT + (static_cast<uint32_t>(q * 32) << 16) + mt * 64 + c16 * 16, v);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            uint4 hi, lo;
            uint32_t* hp = reinterpret_cast<uint32_t*>(&hi);
            uint32_t* lp = reinterpret_cast<uint32_t*>(&lo);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float x0 = v[h * 8 + 2 * e], x1 = v[h * 8 + 2 * e + 1];
              hp[e] = tc::pack_bf16(x0, x1);
              if (X3) {
                const __nv_bfloat162 hb = *reinterpret_cast<const __nv_bfloat162*>(&hp[e]);
                lp[e] = tc::pack_bf16(x0 - __low2float(hb), x1 - __high2float(hb));
              }
            }
            const uint32_t off = tc::sw128_chunk(row, c16 * 2 + h);
            *reinterpret_cast<uint4*>(tsm + off) = hi;
            if (X3) *reinterpret_cast<uint4*>(tsm + Cfg::T_BYTES + off) = lo;
          }
        }
      }
      tc::fence_proxy_async();
      tc::fence_before_sync();
      tc::mbar_arrive(&t_ready[tbuf]);
    }
  }

  // ---------------- P: tensor memory -> shared staging ----------------
  float* pst = reinterpret_cast<float*>(sm);  // [rx2][68] float32 (stage memory is idle now)
  constexpr int PLD = 68;
  if (warp >= 2) {
    const int q = warp & 3;
    if (!tc::mbar_wait(p_full, 0, abort)) bits |= TT_STATUS_TIMEOUT;
    tc::fence_after_sync();
    for (int mt = 0; mt < MT2; ++mt) {
      const int row = mt * 128 + q * 32 + lane;
#pragma unroll
      for (int c16 = 0; c16 < 4; ++c16) {
        float v[16];
        tc::tmem_ld16(tmem_P + (static_cast<uint32_t>(q * 32) << 16) + mt * 64 + c16 * 16, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) pst[row * PLD + c16 * 16 + j] = nslices > 0 ? v[j] : 0.f;
      }
    }
  }
  if (bits) atomicOr(&sh_int[0], bits);
  tc::fence_before_sync();
  __syncthreads();
  cluster.sync();

  // ---------------- cluster reduction and outputs ----------------
  const int rows_per = p.rx2 / C;
  const int r0 = crank * rows_per;
  const int M = sh_int[1];
  int lexp = kNoExpT, lbad = 0;
  const int col0 = 64 * vblk;
  for (int idx = tid; idx < rows_per * 16; idx += kTcThreads) {
    const int row = r0 + idx / 16, c = (idx % 16) * 4;
    float4 part[16];
#pragma unroll
    for (int r = 0; r < 16; ++r)
      if (r < C) part[r] = *reinterpret_cast<const float4*>(cluster.map_shared_rank(pst + row * PLD + c, r));
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int r = 0; r < 16; ++r)
      if (r < C) {
        s.x += part[r].x;
        s.y += part[r].y;
        s.z += part[r].z;
        s.w += part[r].w;
      }
    float o[4] = {mul_pow2<float>(s.x, -M), mul_pow2<float>(s.y, -M), mul_pow2<float>(s.z, -M),
                  mul_pow2<float>(s.w, -M)};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (!isfinite(o[j])) lbad = 1;
      else if (o[j] != 0.f) lexp = max(lexp, exp2_bits(o[j]));
    }
    *reinterpret_cast<float4*>(p.eo_f32 + static_cast<size_t>(row) * p.ry2 + col0 + c) =
        make_float4(o[0], o[1], o[2], o[3]);
    // next mode's K-major panel vblk: row `row`, columns c..c+3 of the panel
    uint2 hi, lo;
    hi.x = tc::pack_bf16(o[0], o[1]);
    hi.y = tc::pack_bf16(o[2], o[3]);
    const __nv_bfloat162 h0 = *reinterpret_cast<const __nv_bfloat162*>(&hi.x);
    const __nv_bfloat162 h1 = *reinterpret_cast<const __nv_bfloat162*>(&hi.y);
    lo.x = tc::pack_bf16(o[0] - __low2float(h0), o[1] - __high2float(h0));
    lo.y = tc::pack_bf16(o[2] - __low2float(h1), o[3] - __high2float(h1));
    const size_t pbase = static_cast<size_t>(vblk) * p.rx2 * 128;
    const uint32_t off = tc::sw128(row, c);
    *reinterpret_cast<uint2*>(reinterpret_cast<unsigned char*>(p.eo_hi) + pbase + off) = hi;
    *reinterpret_cast<uint2*>(reinterpret_cast<unsigned char*>(p.eo_lo) + pbase + off) = lo;
  }
  lexp = __reduce_max_sync(0xffffffffu, lexp);
  lbad = __reduce_or_sync(0xffffffffu, lbad);
  if (lane == 0) {
    sh_int[2 + warp] = lexp;
    if (lbad) atomicOr(&sh_int[0], TT_STATUS_NONFINITE);
  }
  __syncthreads();
  if (tid == 0) {
    int m = kNoExpT;
    for (int w = 0; w < kTcThreads / 32; ++w) m = max(m, sh_int[2 + w]);
    p.bmax_out[blockIdx.x] = m;
    if (blockIdx.x == 0) *p.l_out = *p.l_in + M;
    if (sh_int[0]) set_status(p.status, sh_int[0]);
  }
  tc::fence_before_sync();
  __syncthreads();
  cluster.sync();  // peers are done reading this CTA's staging
  if (warp == 0) tc::tmem_dealloc(tmem, Cfg::TMEM_COLS);
}

// ---------------------------------------------------------------------------
// First mode (left rank 1): E_1[a][b] = sum_i x0[i][a] y0[i][b], CUDA cores.
// ---------------------------------------------------------------------------
template <typename Tin>
__global__ void __launch_bounds__(256) tc_first_kernel(const Tin* __restrict__ x0, const Tin* __restrict__ y0, int I,
                                                      int rx2, int ry2, float* eo_f32, __nv_bfloat16* eo_hi,
                                                      __nv_bfloat16* eo_lo, int* bmax_out, int64_t* l_out,
                                                      int32_t* status) {
  __shared__ int smax[8];
  const int a = blockIdx.x;
  int lexp = kNoExpT, lbad = 0;
  for (int b = threadIdx.x; b < ry2; b += blockDim.x) {
    float s = 0.f;
    for (int i = 0; i < I; ++i) s = fmaf(static_cast<float>(x0[i * rx2 + a]), static_cast<float>(y0[i * ry2 + b]), s);
    if (!isfinite(s)) lbad = 1;
    else if (s != 0.f) lexp = max(lexp, exp2_bits(s));
    eo_f32[static_cast<size_t>(a) * ry2 + b] = s;
    const __nv_bfloat16 h = __float2bfloat16_rn(s);
    const __nv_bfloat16 l = __float2bfloat16_rn(s - __bfloat162float(h));
    const size_t pbase = static_cast<size_t>(b / 64) * rx2 * 128;
    const uint32_t off = tc::sw128(a, b % 64);
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(eo_hi) + pbase + off) = h;
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(eo_lo) + pbase + off) = l;
  }
  lexp = __reduce_max_sync(0xffffffffu, lexp);
  lbad = __reduce_or_sync(0xffffffffu, lbad);
  if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = lexp;
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = kNoExpT;
    for (int w = 0; w < blockDim.x / 32; ++w) m = max(m, smax[w]);
    bmax_out[a] = m;
    if (a == 0) *l_out = 0;
  }
  if (lbad && (threadIdx.x & 31) == 0) set_status(status, TT_STATUS_NONFINITE);
}

// ---------------------------------------------------------------------------
// Last mode (right rank 1), float64 sums:
//   t[a][i] = sum_b E[a][b] y[b][i],  z = 2^L sum_{a,i} x[a][i] t[a][i]
// Blocks of kLastRB rows of E x kLastIB mode indices: the rows and the y slab
// are staged in shared memory, each thread forms one t[a][i] (its warp shares
// the row, so E is read as a broadcast) and the block sums x * t in float64
// into one partial (partials summed in order by tc_last_sum_kernel).
// ---------------------------------------------------------------------------
constexpr int kLastRB = 8, kLastIB = 32;  // kLastRB * kLastIB = 256 threads

template <typename Tin>
__global__ void __launch_bounds__(256) tc_last_parts_kernel(const float* __restrict__ e, const Tin* __restrict__ x,
                                                           const Tin* __restrict__ y, int I, int rx, int ry,
                                                           double* parts) {
  extern __shared__ float lsm[];  // es[kLastRB][ry], ys[ry][kLastIB]
  __shared__ double red[8];
  float* es = lsm;
  float* ys = lsm + kLastRB * ry;
  const int a0 = blockIdx.x * kLastRB, i0 = blockIdx.y * kLastIB;
  const int nr = min(kLastRB, rx - a0), ni = min(kLastIB, I - i0);
  for (int t = threadIdx.x; t < nr * ry; t += blockDim.x) es[t] = e[static_cast<size_t>(a0) * ry + t];
  for (int t = threadIdx.x; t < ry * kLastIB; t += blockDim.x) {
    const int bq = t / kLastIB, j = t - bq * kLastIB;
    ys[t] = j < ni ? static_cast<float>(y[static_cast<size_t>(bq) * I + i0 + j]) : 0.f;
  }
  __syncthreads();
  const int r = threadIdx.x / kLastIB, j = threadIdx.x - r * kLastIB;
  double part = 0.0;
  if (r < nr && j < ni) {
    const float* er = es + r * ry;
    float t = 0.f;
#pragma unroll 8
    for (int bq = 0; bq < ry; ++bq) t = fmaf(er[bq], ys[bq * kLastIB + j], t);
    part = static_cast<double>(x[static_cast<size_t>(a0 + r) * I + i0 + j]) * static_cast<double>(t);
  }
  part = warp_sum(part);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x) / 32; ++w) sum += red[w];
    parts[blockIdx.y * gridDim.x + blockIdx.x] = sum;
  }
}

__global__ void tc_last_sum_kernel(const double* parts, int nparts, const int64_t* l_in, double* out,
                                   int64_t* out_log2, int32_t* status) {
  double z = 0.0;
  for (int q = 0; q < nparts; ++q) z += parts[q];
  const int64_t lg = *l_in;
  int bits = isfinite(z) ? 0 : TT_STATUS_NONFINITE;
  if (out_log2 != nullptr) {
    *out = z;
    *out_log2 = lg;
  } else {
    double v = z;
    if (z != 0.0 && isfinite(z)) {
      const int64_t tot = static_cast<int64_t>(exp2_of(z)) + lg;
      if (tot > 1024) {
        v = z > 0 ? INFINITY : -INFINITY;
        bits |= TT_STATUS_OVERFLOW;
      } else if (tot < -1074) {
        v = 0.0;
      } else {
        v = ldexp(z, static_cast<int>(lg));
      }
    }
    *out = v;
  }
  set_status(status, bits);
}

// float32 -> bfloat16 hi (+ lo = bf16(x - hi)), elementwise over n values.
__global__ void __launch_bounds__(256) tc_split_kernel(const float* __restrict__ src, __nv_bfloat16* hi,
                                                      __nv_bfloat16* lo, int64_t n) {
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float x = src[e];
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[e] = h;
    if (lo != nullptr) lo[e] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
cudaError_t tc_split(const float* src, void* hi, void* lo, int64_t n, cudaStream_t s) {
  count_launch();
  const int grid = static_cast<int>(std::min<int64_t>((n + 255) / 256, 152 * 16));
  tc_split_kernel<<<grid, 256, 0, s>>>(src, static_cast<__nv_bfloat16*>(hi), static_cast<__nv_bfloat16*>(lo), n);
  return cudaGetLastError();
}

cudaError_t tc_first(const void* x0, const void* y0, bool f32_in, int I, int rx2, int ry2, float* eo_f32, void* eo_hi,
                     void* eo_lo, int* bmax_out, int64_t* l_out, int32_t* status, cudaStream_t s) {
  count_launch();
  if (f32_in)
    tc_first_kernel<float><<<rx2, 256, 0, s>>>(static_cast<const float*>(x0), static_cast<const float*>(y0), I, rx2,
                                               ry2, eo_f32, static_cast<__nv_bfloat16*>(eo_hi),
                                               static_cast<__nv_bfloat16*>(eo_lo), bmax_out, l_out, status);
  else
    tc_first_kernel<__nv_bfloat16><<<rx2, 256, 0, s>>>(
        static_cast<const __nv_bfloat16*>(x0), static_cast<const __nv_bfloat16*>(y0), I, rx2, ry2, eo_f32,
        static_cast<__nv_bfloat16*>(eo_hi), static_cast<__nv_bfloat16*>(eo_lo), bmax_out, l_out, status);
  return cudaGetLastError();
}

cudaError_t tc_last(const float* e, const void* x, const void* y, bool f32_in, int I, int rx, int ry, double* parts,
                    const int64_t* l_in, double* out, int64_t* out_log2, int32_t* status, cudaStream_t s) {
  count_launch(2);
  const size_t lsm = static_cast<size_t>(kLastRB + kLastIB) * ry * sizeof(float);  // <= 40 KB (ry <= 256)
  const dim3 grid((rx + kLastRB - 1) / kLastRB, (I + kLastIB - 1) / kLastIB);
  if (f32_in)
    tc_last_parts_kernel<float><<<grid, kLastRB * kLastIB, lsm, s>>>(e, static_cast<const float*>(x),
                                                                      static_cast<const float*>(y), I, rx, ry, parts);
  else
    tc_last_parts_kernel<__nv_bfloat16><<<grid, kLastRB * kLastIB, lsm, s>>>(
        e, static_cast<const __nv_bfloat16*>(x), static_cast<const __nv_bfloat16*>(y), I, rx, ry, parts);
  tc_last_sum_kernel<<<1, 1, 0, s>>>(parts, static_cast<int>(grid.x * grid.y), l_in, out, out_log2, status);
  return cudaGetLastError();
}

cudaError_t tc_mode(const TcModeParams& p, int cluster, cudaStream_t s) {
  const bool x3 = p.x3 != 0;
  const void* kern = x3 ? reinterpret_cast<const void*>(tc_mode_kernel<true>)
                        : reinterpret_cast<const void*>(tc_mode_kernel<false>);
  const size_t smem = x3 ? TcCfg<true>::SMEM : TcCfg<false>::SMEM;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  err = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (err != cudaSuccess) return err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster * (p.ry2 / 64), 1, 1);
  cfg.blockDim = dim3(kTcThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;  // overlap with the previous mode's tail
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  count_launch();
  if (x3) return cudaLaunchKernelEx(&cfg, tc_mode_kernel<true>, p);
  return cudaLaunchKernelEx(&cfg, tc_mode_kernel<false>, p);
}

int tc_cluster_size(bool x3, int want) {
  const void* kern = x3 ? reinterpret_cast<const void*>(tc_mode_kernel<true>)
                        : reinterpret_cast<const void*>(tc_mode_kernel<false>);
  const size_t smem = x3 ? TcCfg<true>::SMEM : TcCfg<false>::SMEM;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  for (int C = want; C >= 1; C /= 2) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(kTcThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    const cudaError_t e = x3 ? cudaOccupancyMaxActiveClusters(&n, tc_mode_kernel<true>, &cfg)
                             : cudaOccupancyMaxActiveClusters(&n, tc_mode_kernel<false>, &cfg);
    if (e == cudaSuccess && n >= 1) return C;
    cudaGetLastError();
  }
  return 0;
}

}  // namespace ttc
