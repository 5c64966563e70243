// Environment sweep on the tensor cores with tf32 products (tcgen05.mma
// kind::tf32), for float32 cores whose ranks are at most 64: the
// contracted-mode absorb of Algorithm 2 step 4, generalised to every mode of a
// full or chain-layout partial contraction (Eq. 8 applied mode after mode).
//
// One thread-block cluster of C CTAs carries the whole sweep in one launch
// (persistent across modes): the environment E stays in shared memory, and
// mode k's slices i = crank, crank + C, ... are this CTA's.  Per slice two
// chained tensor-core GEMMs (E'[u][v] = sum_i sum_{p,q} A_i[p][u] E[p][q] B_i[q][v])
//   GEMM 1  T^T = B_i^T E^T     (M = v, N = p, K = q)
//   GEMM 2  P  += A_i^T T       (M = u, N = v, K = p)
// accumulate in tensor memory; the cluster then adds its CTAs' P's through
// distributed shared memory (each CTA sums a block of rows over all peers and
// pushes the reduced rows to every peer with bulk copies completed on
// mbarriers) into E' of the next mode.  Every operand is K-major (a row per M
// or N index, K contiguous; 128-byte swizzle): kind::tf32 takes no MN-major
// operand, so T is formed transposed (a row of T^T is what an epilogue thread
// holds) and the core slices are written to shared memory with the contracted
// rank along the row.
//
// Precision.  Every float32 operand x (core slices, E, T) is held as two tf32
// values hi = rna(x) and lo = x - hi (exact in float32; the tensor core reads
// lo's top 19 bits).  Both operands of every GEMM are stacked: rows 0-63 of
// an operand hold hi, rows 64-127 lo, so one M = 128, N = 128 product over
// K / 8 steps leaves the four products hi*hi, hi*lo, lo*hi and lo*lo in the
// four 64 x 64 quadrants of the accumulator, added by the epilogue (the
// "3xTF32" scheme, with lo*lo kept since it is free here).  The plain tf32
// form uses N = 64 (the other operand's hi rows) and the upper half only.
//
// Warp roles (256 threads, two warps per SM sub-partition so that a thread may
// hold up to 255 registers): warps 0-3 epilogue (tensor-memory lane quadrants
// 0-3: combine the two halves, split T into the GEMM 2 operand, the cluster
// reduction, E' into the GEMM 1 operand, the end of the sweep); warps 4-6
// load and split core slices (global -> registers -> hi / lo swizzled shared
// tiles, zero padded to 64 x 64; a right-to-left sweep reads its slices with
// their rank legs swapped); warp 7 allocates tensor memory and one of its
// threads issues every MMA.
//
// Scaling: as the CUDA-core sweep, E' is rescaled by an exact power of two
// when its largest binary exponent leaves +-renorm_bits, the exponent kept in
// an int64.  Every wait on an mbarrier is bounded (about half a second) and
// reports TT_STATUS_TIMEOUT.
#include "sweep_body.cuh"

namespace ttc {
namespace tf {

constexpr int RM = 64;            // rank tile (ranks above 64 are not taken by this path)
constexpr int kThreads = 256;     // 8 warps
constexpr int kLoadTid0 = 128;    // loader threads 128..223 (warps 4-6)
constexpr int kLoaders = 96;
constexpr int kLoadIters = (64 * 16 + kLoaders - 1) / kLoaders;  // groups of 4 values per loader thread
constexpr int kMmaWarp = 7;
constexpr int NA = 2;             // A-tile buffers (GEMM 2 operand; next mode's A loads during this one)
constexpr int NB = 1;             // B-tile buffers (GEMM 1 operand; freed as soon as GEMM 1 is done)
constexpr uint32_t TILE = 32768;  // one operand buffer: 64 x 64 float32 values as hi and lo tf32
// Stacked operand (every operand): per 32-column K block (16 KB) rows 0-63
// hold hi, rows 64-127 lo.
constexpr int SLD = 68;           // row stride (floats) of the float32 staging buffers
constexpr int RROWS = RM + 16;    // receive rows: C slots of ceil(64 / C) rows
constexpr int DROWS = 32;         // reduced rows one CTA owns (C >= 2)

constexpr uint32_t OFF_E = 0;                         // GEMM 1 B operand E
constexpr uint32_t OFF_T = OFF_E + TILE;              // GEMM 2 B operand T^T; E' rows during the exchange
constexpr uint32_t OFF_A = OFF_T + TILE;              // NA A tiles
constexpr uint32_t OFF_B = OFF_A + NA * TILE;         // NB B tiles
constexpr uint32_t OFF_S = OFF_B + NB * TILE;         // combine scratch / P rows, 64 x SLD floats
constexpr uint32_t OFF_R = OFF_S + RM * SLD * 4;      // receive slots, RROWS x SLD floats
constexpr uint32_t OFF_D = OFF_R + RROWS * SLD * 4;   // reduced rows of this CTA, DROWS x SLD floats
constexpr uint32_t OFF_REC = OFF_D + DROWS * SLD * 4; // 16 records of 16 bytes + this CTA's
constexpr uint32_t OFF_ZP = OFF_REC + 17 * 16;        // 16 float64 partial sums (final scalar)
constexpr uint32_t OFF_BAR = OFF_ZP + 16 * 8;
constexpr int NBAR = 2 * NA + 2 * NB + 7;
constexpr uint32_t OFF_MISC = OFF_BAR + NBAR * 8;     // tmem slot, status, abort, reduction ints
constexpr size_t SMEM = OFF_MISC + 64 * 4 + 1024;     // + alignment slack
static_assert(SMEM <= 232448, "tf32 sweep does not fit in shared memory");

constexpr int kNoExpF = -(1 << 30);

// ---- small helpers ----
__device__ __forceinline__ float rna_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Byte offset of element (row m, K column k) of a K-major 128-byte-swizzled
// operand whose 32-column K blocks are `blk` bytes apart.
__device__ __forceinline__ uint32_t kmaj(int m, int k, uint32_t blk) {
  return (k >> 5) * blk + m * 128 + ((((k & 31) >> 2) ^ (m & 7)) << 4) + ((k & 3) << 2);
}
// Stacked operand: hi at row m, lo at row m + 64 (8192 bytes on).
__device__ __forceinline__ uint32_t st_off(int m, int k) { return kmaj(m, k, 16384); }

// Instruction descriptor: tf32 x tf32 -> f32, dense, both operands K-major,
// M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
         (static_cast<uint32_t>(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// 32 lanes x 64 consecutive 32-bit columns of tensor memory (warp-collective),
// four loads in flight and one wait.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64]) {
  uint32_t r[64];
#pragma unroll
  for (int c = 0; c < 4; ++c)
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[16 * c]), "=r"(r[16 * c + 1]), "=r"(r[16 * c + 2]), "=r"(r[16 * c + 3]), "=r"(r[16 * c + 4]),
          "=r"(r[16 * c + 5]), "=r"(r[16 * c + 6]), "=r"(r[16 * c + 7]), "=r"(r[16 * c + 8]), "=r"(r[16 * c + 9]),
          "=r"(r[16 * c + 10]), "=r"(r[16 * c + 11]), "=r"(r[16 * c + 12]), "=r"(r[16 * c + 13]), "=r"(r[16 * c + 14]),
          "=r"(r[16 * c + 15])
        : "r"(taddr + 16 * c));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 64; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

// Slices of a mode of I slices that CTA crank of C takes.
__device__ __forceinline__ int n_slices(int I, int crank, int C) { return crank < I ? (I - 1 - crank) / C + 1 : 0; }

// Where a sweep's results go (the two-sided kernel points the final
// environment at its workspace half).
struct TfOut {
  double* z_out;
  int64_t* z_out_log2;
  int32_t* status;
  int skip_copies;
};

// ---------------------------------------------------------------------------
// Loader: slice i of a core as a stacked K-major operand: row m = the output
// rank index (M of the GEMM), column k = the contracted rank index (K).
//   out_major == 0: value(m, k) = core[k][i][m]   (core [n_in][I][n_out])
//   out_major == 1: value(m, k) = core[m][i][k]   (core [n_out][I][n_in])
// Entries outside n_out x n_in are zero.  96 threads (tl = 0..95), each with
// kLoadIters groups of 4 values (q = tl + 96 g < 1024): load_regs issues all
// of a thread's global loads before any is used (so a slice's two tiles are in
// flight together), then store_tile splits them into hi / lo and writes them.
//   out_major: group q is row m = q / 16, columns 4 (q % 16) .. + 3
//              (contiguous in global memory);
//   in_major:  column k = q % 64, rows 4 (q / 64) .. + 3 (lanes along k: each
//              4-byte store of a warp covers one row).
// ---------------------------------------------------------------------------
struct TileRegs {
  float4 v[kLoadIters];
};

__device__ __forceinline__ void load_regs(TileRegs& r, const float* __restrict__ core, int i, int I, int n_in, int n_out,
                                          int out_major, int tl) {
  const int inner = out_major ? n_in : n_out;
  const bool vec = (inner & 3) == 0 && (reinterpret_cast<uintptr_t>(core) & 15) == 0;
#pragma unroll
  for (int g = 0; g < kLoadIters; ++g) {
    const int q = tl + kLoaders * g;
    int row, col0, nrow, ncol;  // the run of 4 is along col (contiguous in memory)
    if (out_major) {
      row = q >> 4;
      col0 = (q & 15) * 4;
      nrow = n_out;
      ncol = n_in;
    } else {
      row = q & 63;
      col0 = (q >> 6) * 4;
      nrow = n_in;
      ncol = n_out;
    }
    float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
    if (q < 1024 && row < nrow && col0 < ncol) {
      const float* src = core + (static_cast<int64_t>(row) * I + i) * ncol + col0;
      if (vec) {
        t = __ldg(reinterpret_cast<const float4*>(src));
      } else {
        t.x = __ldg(src);
        if (col0 + 1 < ncol) t.y = __ldg(src + 1);
        if (col0 + 2 < ncol) t.z = __ldg(src + 2);
        if (col0 + 3 < ncol) t.w = __ldg(src + 3);
      }
    }
    r.v[g] = t;
  }
}

__device__ __forceinline__ void store_tile(unsigned char* tile, const TileRegs& r, int out_major, bool x3, int tl) {
#pragma unroll
  for (int g = 0; g < kLoadIters; ++g) {
    const int q = tl + kLoaders * g;
    if (q >= 1024) break;
    const float v[4] = {r.v[g].x, r.v[g].y, r.v[g].z, r.v[g].w};
    if (out_major) {
      const int m = q >> 4, k0 = (q & 15) * 4;
      const float4 h = make_float4(rna_tf32(v[0]), rna_tf32(v[1]), rna_tf32(v[2]), rna_tf32(v[3]));
      const uint32_t off = st_off(m, k0);
      *reinterpret_cast<float4*>(tile + off) = h;
      if (x3) *reinterpret_cast<float4*>(tile + off + 8192) = make_float4(v[0] - h.x, v[1] - h.y, v[2] - h.z, v[3] - h.w);
    } else {
      const int k = q & 63, m0 = (q >> 6) * 4;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float h = rna_tf32(v[e]);
        const uint32_t off = st_off(m0 + e, k);
        *reinterpret_cast<float*>(tile + off) = h;
        if (x3) *reinterpret_cast<float*>(tile + off + 8192) = v[e] - h;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// The sweep body.  Returns with the final environment in `eraw` (float32
// rows, stride SLD, its pending power-of-two in *escale, total scale in
// log2s) for the caller's end-of-sweep work.
// ---------------------------------------------------------------------------
struct TfState {
  int64_t log2s;
  int escale;   // pending exponent: entries of eraw are to be multiplied by 2^-escale
  int bad;
  int nu, nv;   // shape of the final environment
};

template <bool X3>
__device__ void tf_body(const SweepParams& p, const TfOut& o, unsigned char* sm, int C, int crank, TfState& st) {
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + OFF_BAR);
  uint64_t* a_full = bars;
  uint64_t* a_empty = a_full + NA;
  uint64_t* b_full = a_empty + NA;
  uint64_t* b_empty = b_full + NB;
  uint64_t* e_ready = b_empty + NB;
  uint64_t* t_full = e_ready + 1;
  uint64_t* t_ready = t_full + 1;
  uint64_t* p_full = t_ready + 1;
  uint64_t* xbar = p_full + 1;  // [0] partial rows in, [1] reduced rows in
  uint64_t* done = xbar + 2;    // every MMA of this CTA has completed
  int* misc = reinterpret_cast<int*>(sm + OFF_MISC);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(misc);
  int* sh_status = misc + 1;
  volatile int* abort = misc + 2;
  int* ired = misc + 8;  // 40 ints of reduction scratch

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_pipe = p.final_scalar ? p.n_steps - 1 : p.n_steps;
  const bool emit = p.emit.enabled != 0;
  int bits = 0;

  if (warp == kMmaWarp) tc::tmem_alloc(tmem_slot, 256);
  if (tid == 0) {
    for (int s = 0; s < NA; ++s) {
      tc::mbar_init(&a_full[s], kLoaders);
      tc::mbar_init(&a_empty[s], 1);
    }
    for (int s = 0; s < NB; ++s) {
      tc::mbar_init(&b_full[s], kLoaders);
      tc::mbar_init(&b_empty[s], 1);
    }
    tc::mbar_init(e_ready, 128);
    tc::mbar_init(t_full, 1);
    tc::mbar_init(t_ready, 128);
    tc::mbar_init(p_full, 1);
    tc::mbar_init(&xbar[0], 1);
    tc::mbar_init(&xbar[1], 1);
    tc::mbar_init(done, 1);
    tc::mbar_init_fence();
    *sh_status = 0;
    *abort = 0;
  }
  // start environment E_0 = [1]: hi[0][0] = 1, everything else zero
  for (int q = tid; q < static_cast<int>(TILE / 16); q += kThreads)
    reinterpret_cast<float4*>(sm + OFF_E)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  tc::fence_before_sync();
  __syncthreads();
  if (tid == 0) *reinterpret_cast<float*>(sm + OFF_E) = 1.f;
  cg::this_cluster().sync();  // barriers of every CTA exist before any peer pushes; E_0 written
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t tD1 = tmem, tD2 = tmem + 128;  // 128 columns each

  if (warp >= 4 && warp < kMmaWarp) {
    // ---------------- loaders ----------------
    const int tl = tid - kLoadTid0;
    uint32_t ia = 0, ib = 0;
    TileRegs rb, ra;
    for (int j = 0; j < n_pipe; ++j) {
      const SweepStep& s = p.step[j];
      const int ns = n_slices(s.I, crank, C);
      for (int t = 0; t < ns; ++t) {
        const int i = crank + t * C;
        const int sb = ib % NB, sa = ia % NA;
        // both tiles of the slice in flight before either buffer is waited for
        load_regs(rb, static_cast<const float*>(s.gy), i, s.I, s.rin_y, s.rout_y, p.transposed_y, tl);  // B_i^T: rows v, columns q
        load_regs(ra, static_cast<const float*>(s.gx), i, s.I, s.rin_x, s.rout_x, p.transposed, tl);  // A_i^T: rows u, columns p
        if (!tc::mbar_wait(&b_empty[sb], ((ib / NB) & 1) ^ 1, abort)) bits |= TT_STATUS_TIMEOUT;
        store_tile(sm + OFF_B + sb * TILE, rb, p.transposed_y, X3, tl);
        tc::fence_proxy_async();
        tc::mbar_arrive(&b_full[sb]);
        ++ib;
        if (!tc::mbar_wait(&a_empty[sa], ((ia / NA) & 1) ^ 1, abort)) bits |= TT_STATUS_TIMEOUT;
        store_tile(sm + OFF_A + sa * TILE, ra, p.transposed, X3, tl);
        tc::fence_proxy_async();
        tc::mbar_arrive(&a_full[sa]);
        ++ia;
      }
    }
    if (emit) {
      const EmitParams& em = p.emit;
      // lead: C[u][i][y] = sum_a gx[a][i][u] K[a][y]: row u, column a = gx[a][i][u]
      // trail: C[u][i][y] = sum_b gx[u][i][b] K[b][y]: row u, column b = gx[u][i][b]
      const int n_in = em.lead ? em.ra : em.rb, n_out = em.lead ? em.rb : em.ra;
      const int ns = n_slices(em.I, crank, C);
      for (int t = 0; t < ns; ++t) {
        const int sa = ia % NA;
        load_regs(ra, static_cast<const float*>(em.gx), crank + t * C, em.I, n_in, n_out, em.lead ? 0 : 1, tl);
        if (!tc::mbar_wait(&a_empty[sa], ((ia / NA) & 1) ^ 1, abort)) bits |= TT_STATUS_TIMEOUT;
        store_tile(sm + OFF_A + sa * TILE, ra, em.lead ? 0 : 1, X3, tl);
        tc::fence_proxy_async();
        tc::mbar_arrive(&a_full[sa]);
        ++ia;
      }
    }
  } else if (warp == kMmaWarp) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr uint32_t id = idesc_tf32(X3 ? 128 : 64);
      const uint32_t sE = tc::su32(sm + OFF_E), sT = tc::su32(sm + OFF_T);
      uint32_t ia = 0, ib = 0, nt = 0;
      for (int j = 0; j <= n_pipe; ++j) {
        if (j == n_pipe && !emit) break;
        // E_0 is in place from the start; E_j (j >= 1) is the j-th arrival of
        // e_ready, K for the emission the max(n_pipe, 1)-th
        const int nth = j == n_pipe ? max(n_pipe, 1) : j;
        if (nth >= 1 && !tc::mbar_wait(e_ready, (nth - 1) & 1, abort)) bits |= TT_STATUS_TIMEOUT;
        tc::fence_after_sync();
        if (j == n_pipe) {
          // chain emission: D2 = [A_hi^T; A_lo^T] K per slice of the boundary core
          const int kst = ((p.emit.lead ? p.emit.ra : p.emit.rb) + 7) / 8;
          const int ns = n_slices(p.emit.I, crank, C);
          for (int t = 0; t < ns; ++t) {
            if (t > 0 && !tc::mbar_wait(t_ready, (nt - 1) & 1, abort)) bits |= TT_STATUS_TIMEOUT;
            const int sa = ia % NA;
            if (!tc::mbar_wait(&a_full[sa], (ia / NA) & 1, abort)) bits |= TT_STATUS_TIMEOUT;
            tc::fence_after_sync();
            const uint32_t sA = tc::su32(sm + OFF_A + sa * TILE);
            for (int kk = 0; kk < kst; ++kk)
              mma_tf32(tD2, tc::sdesc(sA + (kk >> 2) * 16384 + (kk & 3) * 32, 16, 1024),
                       tc::sdesc(sT + (kk >> 2) * 16384 + (kk & 3) * 32, 16, 1024), id, kk != 0);
            tc::mma_commit(&a_empty[sa]);
            tc::mma_commit(t_full);
            ++ia;
            ++nt;
          }
          break;
        }
        const SweepStep& s = p.step[j];
        const int ns = n_slices(s.I, crank, C);
        const int k1 = (s.rin_y + 7) / 8, k2 = (s.rin_x + 7) / 8;
        for (int t = 0; t < ns; ++t) {
          const int sb = ib % NB, sa = ia % NA;
          if (!tc::mbar_wait(&b_full[sb], (ib / NB) & 1, abort)) bits |= TT_STATUS_TIMEOUT;
          tc::fence_after_sync();
          const uint32_t sB = tc::su32(sm + OFF_B + sb * TILE);
          // GEMM 1: D1 = [B_hi^T; B_lo^T] [E_hi; E_lo]^T
          for (int kk = 0; kk < k1; ++kk)
            mma_tf32(tD1, tc::sdesc(sB + (kk >> 2) * 16384 + (kk & 3) * 32, 16, 1024),
                     tc::sdesc(sE + (kk >> 2) * 16384 + (kk & 3) * 32, 16, 1024), id, kk != 0);
          tc::mma_commit(&b_empty[sb]);
          tc::mma_commit(t_full);
          ++ib;
          // GEMM 2: D2 += [A_hi^T; A_lo^T] [T_hi^T; T_lo^T]^T, once T^T is staged
          if (!tc::mbar_wait(t_ready, nt & 1, abort)) bits |= TT_STATUS_TIMEOUT;
          if (!tc::mbar_wait(&a_full[sa], (ia / NA) & 1, abort)) bits |= TT_STATUS_TIMEOUT;
          tc::fence_after_sync();
          const uint32_t sA = tc::su32(sm + OFF_A + sa * TILE);
          for (int kk = 0; kk < k2; ++kk)
            mma_tf32(tD2, tc::sdesc(sA + (kk >> 2) * 16384 + (kk & 3) * 32, 16, 1024),
                     tc::sdesc(sT + (kk >> 2) * 16384 + (kk & 3) * 32, 16, 1024), id, (t | kk) != 0);
          tc::mma_commit(&a_empty[sa]);
          ++ia;
          ++nt;
        }
        if (ns > 0) tc::mma_commit(p_full);
        else tc::mbar_arrive(p_full);
      }
      // tensor memory is released only after the last MMA has completed
      tc::mma_commit(done);
      if (!tc::mbar_wait(done, 0, abort)) bits |= TT_STATUS_TIMEOUT;
    }
  } else {
    // ---------------- epilogue (warps 0-3) ----------------
    // Each warp owns 32 accumulator rows (r = 32 (q & 1) + lane) and half of
    // the 64 output columns (warps 0, 1 columns 0-31, warps 2, 3 columns
    // 32-63).  The accumulator is 128 x 128 (x3) or 128 x 64: rows 0-63 come
    // from the hi rows of the stacked A operand, rows 64-127 from its lo rows;
    // columns 0-63 from the B operand's hi rows, 64-127 from its lo rows.
    // Warps 0, 1 read lanes 0-63, warps 2, 3 lanes 64-127; each adds its
    // column halves and hands the half it does not own to its partner (warp
    // q ^ 2) through S, so every output is the sum of its four quadrants.
    const int q = warp;  // tensor-memory lane quadrant
    const int r = 32 * (q & 1) + lane;
    const int half = q >> 1;
    float* S = reinterpret_cast<float*>(sm + OFF_S);
    float* R = reinterpret_cast<float*>(sm + OFF_R);
    float* D = reinterpret_cast<float*>(sm + OFF_D);
    float* eraw = C > 1 ? reinterpret_cast<float*>(sm + OFF_T) : S;
    int* rec = reinterpret_cast<int*>(sm + OFF_REC);  // [16][4]: exponent, bad
    int* srec = rec + 64;
    uint32_t nt = 0;
    int xph = 0;
    int64_t log2s = 0;
    int escale = 0, bad = 0;
    int nu = 1, nv = 1;
    const uint32_t lane_base = static_cast<uint32_t>(q * 32) << 16;

    // v = row r, columns 32 half .. + 31 of the sum of tD's quadrants
    auto combine = [&](uint32_t tD, float (&v)[32]) {
      float w[64];
      tmem_ld64(tD + lane_base, w);
      if (X3) {
        float w2[64];
        tmem_ld64(tD + lane_base + 64, w2);
#pragma unroll
        for (int c = 0; c < 64; ++c) w[c] += w2[c];
      }
      // warps 0, 1 pass columns 32-63 of the upper half; warps 2, 3 columns 0-31 of the lower
      if (half == 0 || X3) {
        float* dst = S + r * SLD + (half ? 0 : 32);
        const float* src = w + (half ? 0 : 32);
#pragma unroll
        for (int c = 0; c < 32; c += 4) *reinterpret_cast<float4*>(dst + c) = make_float4(src[c], src[c + 1], src[c + 2], src[c + 3]);
      }
      named_sync(1, 128);
      const float* oth = S + r * SLD + 32 * half;
#pragma unroll
      for (int c = 0; c < 32; c += 4) {
        const float4 a = *reinterpret_cast<const float4*>(oth + c);
        const float o4[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (half == 0) v[c + e] = X3 ? w[c + e] + o4[e] : w[c + e];
          else v[c + e] = X3 ? o4[e] + w[32 + c + e] : o4[e];
        }
      }
    };

    // E' (rows nu, columns nv of src, row stride SLD, times 2^-escale) into
    // the stacked GEMM 1 B operand; every other entry zero
    auto build_e = [&](const float* src) {
      unsigned char* eb = sm + OFF_E;
      const int j4 = tid & 15, c0 = j4 * 4, m0 = tid >> 4;
      float4 x[8];
#pragma unroll
      for (int it = 0; it < 8; ++it) {
        const int m = m0 + 8 * it;
        x[it] = m < nu ? *reinterpret_cast<const float4*>(src + m * SLD + c0) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int it = 0; it < 8; ++it) {
        const int m = m0 + 8 * it;
        float e4[4] = {x[it].x, x[it].y, x[it].z, x[it].w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (c0 + e >= nv) e4[e] = 0.f;
          else if (escale) e4[e] = mul_pow2<float>(e4[e], -escale);
        }
        const float4 h = make_float4(rna_tf32(e4[0]), rna_tf32(e4[1]), rna_tf32(e4[2]), rna_tf32(e4[3]));
        const uint32_t off = st_off(m, c0);
        *reinterpret_cast<float4*>(eb + off) = h;
        *reinterpret_cast<float4*>(eb + off + 8192) =
            X3 ? make_float4(e4[0] - h.x, e4[1] - h.y, e4[2] - h.z, e4[3] - h.w) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };

    for (int j = 0; j < n_pipe; ++j) {
      const SweepStep& s = p.step[j];
      const int ns = n_slices(s.I, crank, C);
      const bool last = j + 1 == n_pipe;
      for (int t = 0; t < ns; ++t) {
        // T^T = D1 rows (v), split into the stacked GEMM 2 B operand (row v, K column p)
        if (!tc::mbar_wait(t_full, nt & 1, abort)) bits |= TT_STATUS_TIMEOUT;
        tc::fence_after_sync();
        float v[32];
        combine(tD1, v);
        unsigned char* tb = sm + OFF_T;
#pragma unroll
        for (int j4 = 0; j4 < 8; ++j4) {
          const float4 h = make_float4(rna_tf32(v[4 * j4]), rna_tf32(v[4 * j4 + 1]), rna_tf32(v[4 * j4 + 2]),
                                       rna_tf32(v[4 * j4 + 3]));
          const uint32_t off = st_off(r, 32 * half + 4 * j4);
          *reinterpret_cast<float4*>(tb + off) = h;
          if (X3)
            *reinterpret_cast<float4*>(tb + off + 8192) =
                make_float4(v[4 * j4] - h.x, v[4 * j4 + 1] - h.y, v[4 * j4 + 2] - h.z, v[4 * j4 + 3] - h.w);
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        tc::mbar_arrive(t_ready);
        ++nt;
      }
      // ---- P of this CTA, rows in S ----
      if (!tc::mbar_wait(p_full, j & 1, abort)) bits |= TT_STATUS_TIMEOUT;
      tc::fence_after_sync();
      nu = s.rout_x;
      nv = s.rout_y;
      {
        float v[32];
        if (ns > 0) {
          combine(tD2, v);
        } else {
          named_sync(1, 128);
#pragma unroll
          for (int c = 0; c < 32; ++c) v[c] = 0.f;
        }
        // this thread read S[r][32 half ..] above and is the only one to write it now
        float* row = S + r * SLD + 32 * half;
#pragma unroll
        for (int c = 0; c < 32; c += 4) *reinterpret_cast<float4*>(row + c) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
      }
      tc::fence_before_sync();
      named_sync(1, 128);
      // ---- cluster reduction: E'[u][v] = sum over CTAs of P_c[u][v] ----
      int gexp = kNoExpF, gbad = 0;
      if (C == 1) {
        float lmax = 0.f;
        int lbad = 0;
        for (int idx = tid; idx < nu * nv; idx += 128) {
          const int u = idx / nv, c = idx - u * nv;
          const float e = S[u * SLD + c];
          if (isfinite(e)) lmax = fmaxf(lmax, fabsf(e));
          else lbad = 1;
        }
        lmax = warp_max(lmax);
        lbad = warp_or(lbad);
        if (lane == 0) {
          ired[warp] = lmax > 0.f ? exp2_bits(lmax) : kNoExpF;
          ired[8 + warp] = lbad;
        }
        named_sync(1, 128);
        for (int w = 0; w < 4; ++w) {
          gexp = max(gexp, ired[w]);
          gbad |= ired[8 + w];
        }
        named_sync(1, 128);  // ired is read before its next use
      } else {
        const int chunk = (nu + C - 1) / C;
        const uint32_t rowb = SLD * 4;
        const int my0 = min(nu, crank * chunk), my_rows = min(nu, my0 + chunk) - my0;
        tc::fence_proxy_async();
        named_sync(1, 128);
        if (tid == 0) tc::mbar_expect_tx(&xbar[0], static_cast<uint32_t>(C * my_rows) * rowb);
        if (tid < C) {
          const int r0o = min(nu, tid * chunk), ro = min(nu, r0o + chunk) - r0o;
          if (ro > 0)
            tc::bulk_s2c(tc::mapa(tc::su32(R + crank * chunk * SLD), tid), S + r0o * SLD, ro * rowb,
                         tc::mapa(tc::su32(&xbar[0]), tid));
        }
        if (!tc::mbar_wait(&xbar[0], xph & 1, abort)) bits |= TT_STATUS_TIMEOUT;
        // owner sum over the C peers, fixed order (deterministic); tpj threads
        // per 4-column job, each over every tpj-th peer, then a shuffle sum
        const int jobs = my_rows * 16;
        const int tpj = jobs <= 32 ? 4 : (jobs <= 64 ? 2 : 1);
        const int per = 128 / tpj;
        const int niter = (jobs + per - 1) / per;  // the same for every thread
        const int sub = tid & (tpj - 1);
        float lmax = 0.f;
        int lbad = 0;
        for (int it = 0; it < niter; ++it) {
          const int job = tid / tpj + it * per;
          const bool act = job < jobs;
          const int vr = act ? job >> 4 : 0, c = (job & 15) * 4;
          float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
          for (int rr = sub; act && rr < C; rr += tpj) {
            const float4 x = *reinterpret_cast<const float4*>(R + (rr * chunk + vr) * SLD + c);
            sum.x += x.x;
            sum.y += x.y;
            sum.z += x.z;
            sum.w += x.w;
          }
          for (int off = 1; off < tpj; off <<= 1) {
            sum.x += __shfl_xor_sync(0xffffffffu, sum.x, off);
            sum.y += __shfl_xor_sync(0xffffffffu, sum.y, off);
            sum.z += __shfl_xor_sync(0xffffffffu, sum.z, off);
            sum.w += __shfl_xor_sync(0xffffffffu, sum.w, off);
          }
          if (act && sub == 0) {
            *reinterpret_cast<float4*>(D + vr * SLD + c) = sum;
            const float e4[4] = {sum.x, sum.y, sum.z, sum.w};
#pragma unroll
            for (int e = 0; e < 4; ++e)
              if (c + e < nv) {
                if (isfinite(e4[e])) lmax = fmaxf(lmax, fabsf(e4[e]));
                else lbad = 1;
              }
          }
        }
        lmax = warp_max(lmax);
        lbad = warp_or(lbad);
        if (lane == 0) {
          ired[warp] = lmax > 0.f ? exp2_bits(lmax) : kNoExpF;
          ired[8 + warp] = lbad;
        }
        named_sync(1, 128);
        if (tid == 0) {
          int m = kNoExpF, b = 0;
          for (int w = 0; w < 4; ++w) {
            m = max(m, ired[w]);
            b |= ired[8 + w];
          }
          srec[0] = m;
          srec[1] = b;
          tc::mbar_expect_tx(&xbar[1], static_cast<uint32_t>(nu) * rowb + 16u * C);
        }
        tc::fence_proxy_async();
        named_sync(1, 128);
        if (tid < C) {
          if (my_rows > 0)
            tc::bulk_s2c(tc::mapa(tc::su32(eraw + my0 * SLD), tid), D, my_rows * rowb, tc::mapa(tc::su32(&xbar[1]), tid));
          tc::bulk_s2c(tc::mapa(tc::su32(rec + 4 * crank), tid), srec, 16, tc::mapa(tc::su32(&xbar[1]), tid));
        }
        if (!tc::mbar_wait(&xbar[1], xph & 1, abort)) bits |= TT_STATUS_TIMEOUT;
        ++xph;
        for (int rr = 0; rr < C; ++rr) {
          gexp = max(gexp, rec[4 * rr]);
          gbad |= rec[4 * rr + 1];
        }
      }
      if (gbad) bad = 1;
      escale = (gexp != kNoExpF && (gexp > p.renorm_bits || gexp < -p.renorm_bits)) ? gexp : 0;
      log2s += escale;
      // ---- E' into the GEMM 1 operand of the next mode ----
      if (!last) {
        build_e(eraw);
        tc::fence_proxy_async();
        tc::fence_before_sync();
        tc::mbar_arrive(e_ready);
      }
    }
    if (n_pipe == 0) {
      nu = p.rx0;
      nv = p.ry0;
      if (tid == 0) eraw[0] = 1.f;
      for (int idx = tid; idx < RM * SLD; idx += 128)
        if (idx != 0) eraw[idx] = 0.f;
      named_sync(1, 128);
    }
    // ---- chain emission: C_i = A_i^T K on the tensor cores ----
    if (emit) {
      const EmitParams& em = p.emit;
      // K^T (row y, K column a; K is nu x nv) into the GEMM 2 B operand; eraw may be the T region
      float kx[32];
#pragma unroll
      for (int e = 0; e < 32; ++e) {
        const int idx = tid + e * 128;
        const int m = idx >> 6, c = idx & 63;
        kx[e] = (m < nu && c < nv) ? eraw[m * SLD + c] : 0.f;
      }
      named_sync(1, 128);
      const bool fold = em.z_log2_out == nullptr;
      unsigned char* tb = sm + OFF_T;
#pragma unroll
      for (int e = 0; e < 32; ++e) {
        const int idx = tid + e * 128;
        const int m = idx >> 6, c = idx & 63;
        const float x = escale ? mul_pow2<float>(kx[e], -escale) : kx[e];
        const float h = rna_tf32(x);
        *reinterpret_cast<float*>(tb + st_off(c, m)) = h;
        *reinterpret_cast<float*>(tb + st_off(c, m) + 8192) = X3 ? x - h : 0.f;
      }
      tc::fence_proxy_async();
      tc::fence_before_sync();
      tc::mbar_arrive(e_ready);
      const int ncol = em.lead ? em.rb : em.ra;  // u range
      const int ns = n_slices(em.I, crank, C);
      int ebits = 0;
      for (int t = 0; t < ns; ++t) {
        const int i = crank + t * C;
        if (!tc::mbar_wait(t_full, nt & 1, abort)) bits |= TT_STATUS_TIMEOUT;
        tc::fence_after_sync();
        float v[32];
        combine(tD2, v);
        {
          const int u = r;
          if (u < ncol) {
            float* dst = static_cast<float*>(em.c_out) + (static_cast<int64_t>(u) * em.I + i) * em.ry;
#pragma unroll
            for (int c = 0; c < 32; ++c) {
              const int y = 32 * half + c;
              if (y < em.ry) {
                float val = v[c];
                if (fold && log2s != 0) {
                  const float v0 = val;
                  val = scale_pow2_sat<float>(val, log2s);
                  if (isfinite(v0) && !isfinite(val)) ebits |= TT_STATUS_OVERFLOW;
                }
                if (!isfinite(val)) ebits |= TT_STATUS_NONFINITE;
                dst[y] = val;
              }
            }
          }
        }
        tc::fence_before_sync();
        tc::mbar_arrive(t_ready);
        ++nt;
      }
      bits |= ebits;
      if (crank == 0 && tid == 0 && em.z_log2_out != nullptr) *em.z_log2_out = log2s;
    }
    st.log2s = log2s;
    st.escale = escale;
    st.bad = bad;
    st.nu = nu;
    st.nv = nv;
  }
  if (bits) atomicOr(sh_status, bits);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid == 0 && *sh_status) set_status(o.status, *sh_status);
  // the end state lives in the epilogue threads; share it through shared memory
  int* stash = misc + 48;
  if (tid == 0) {
    stash[0] = st.escale;
    stash[1] = st.bad;
    stash[2] = st.nu;
    stash[3] = st.nv;
    reinterpret_cast<int64_t*>(misc + 56)[0] = st.log2s;
  }
  __syncthreads();
  st.escale = stash[0];
  st.bad = stash[1];
  st.nu = stash[2];
  st.nv = stash[3];
  st.log2s = reinterpret_cast<int64_t*>(misc + 56)[0];
  if (warp == kMmaWarp) tc::tmem_dealloc(tmem, 256);
}

// Final-environment work shared by the kernels: the last mode of a full
// contraction summed in float64 (t_i[a] = sum_b E[a][b] B_i[b] in float32,
// z = sum_{i,a} A_i[a] t_i[a] in float64, cluster-reduced in CTA 0), or the
// environment written out.
__device__ void tf_finish(const SweepParams& p, const TfOut& o, unsigned char* sm, int C, int crank, const TfState& st) {
  const int tid = threadIdx.x;
  const float* eraw = C > 1 ? reinterpret_cast<const float*>(sm + OFF_T) : reinterpret_cast<const float*>(sm + OFF_S);
  double* zpart = reinterpret_cast<double*>(sm + OFF_ZP);
  cg::cluster_group cluster = cg::this_cluster();
  if (p.final_scalar) {
    const SweepStep& s = p.step[p.n_steps - 1];
    const float* gx = static_cast<const float*>(s.gx);
    const float* gy = static_cast<const float*>(s.gy);
    float* bvec = reinterpret_cast<float*>(sm + OFF_B);  // B_i[q][0], q < rin_y
    double part = 0.0;
    for (int i = crank; i < s.I; i += C) {
      for (int qq = tid; qq < s.rin_y; qq += kThreads)
        bvec[qq] = p.transposed_y ? __ldg(gy + static_cast<int64_t>(i) * s.rin_y + qq) : __ldg(gy + static_cast<int64_t>(qq) * s.I + i);
      __syncthreads();
      for (int a = tid; a < s.rin_x; a += kThreads) {
        float t = 0.f;
        for (int qq = 0; qq < s.rin_y; ++qq) {
          const float e = st.escale ? mul_pow2<float>(eraw[a * SLD + qq], -st.escale) : eraw[a * SLD + qq];
          t = fmaf(e, bvec[qq], t);
        }
        const float av = p.transposed ? __ldg(gx + static_cast<int64_t>(i) * s.rin_x + a) : __ldg(gx + static_cast<int64_t>(a) * s.I + i);
        part = fma(static_cast<double>(av), static_cast<double>(t), part);
      }
      __syncthreads();
    }
    part = warp_sum(part);
    double* dred = reinterpret_cast<double*>(sm + OFF_S);
    if ((tid & 31) == 0) dred[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
      double sum = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) sum += dred[w];
      *cluster.map_shared_rank(zpart + crank, 0) = sum;
    }
    cluster.sync();
    if (crank == 0 && tid == 0) {
      double z = 0.0;
      for (int r = 0; r < C; ++r) z += zpart[r];
      int st_bits = (isfinite(z) && !st.bad) ? 0 : TT_STATUS_NONFINITE;
      if (o.z_out_log2 != nullptr) {
        *o.z_out = z;
        *o.z_out_log2 = st.log2s;
      } else {
        double v = z;
        if (z != 0.0 && isfinite(z)) {
          const int64_t tot = static_cast<int64_t>(exp2_of(z)) + st.log2s;
          if (tot > 1024) {
            v = z > 0 ? INFINITY : -INFINITY;
            st_bits |= TT_STATUS_OVERFLOW;
          } else if (tot < -1074) {
            v = 0.0;
          } else {
            v = ldexp(z, static_cast<int>(st.log2s));
          }
        }
        *o.z_out = v;
      }
      set_status(o.status, st_bits);
    }
    return;
  }
  if (p.e_out != nullptr) {
    // every CTA holds the whole environment: each writes rows u = crank, crank + C, ...
    float* e = static_cast<float*>(p.e_out);
    const int nrow = st.nu > crank ? (st.nu - 1 - crank) / C + 1 : 0;
    for (int idx = tid; idx < nrow * st.nv; idx += kThreads) {
      const int u = crank + (idx / st.nv) * C, c = idx % st.nv;
      e[u * st.nv + c] = st.escale ? mul_pow2<float>(eraw[u * SLD + c], -st.escale) : eraw[u * SLD + c];
    }
    if (crank == 0 && tid == 0 && p.e_out_log2 != nullptr) *p.e_out_log2 = st.log2s;
    __threadfence();  // visible to the other cluster before this cluster counts itself done
  }
  if (tid == 0 && crank == 0 && st.bad) set_status(o.status, TT_STATUS_NONFINITE);
}

// One sweep (full or chain partial).  A chain emission with free-core copies
// is launched with a second cluster that copies the free cores.
template <bool X3>
__global__ void __launch_bounds__(kThreads, 1) tf_sweep_kernel(const __grid_constant__ SweepParams p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  cg::cluster_group cluster = cg::this_cluster();
  const int C = static_cast<int>(cluster.num_blocks());
  const int crank = static_cast<int>(cluster.block_rank());
  if (blockIdx.x >= static_cast<unsigned>(C)) {
    const int64_t g = static_cast<int64_t>(crank) * kThreads + threadIdx.x, gs = static_cast<int64_t>(C) * kThreads;
    for (int t = 0; t < p.emit.n_copies; ++t) {
      const CopyTask& tk = p.emit.copy[t];
      const float* __restrict__ src = static_cast<const float*>(tk.src);
      float* __restrict__ dst = static_cast<float*>(tk.dst);
      if (!tk.swap) copy_plain<float>(dst, src, static_cast<int64_t>(tk.r0) * tk.I * tk.r1, g, gs);
      else copy_swap_tiled<float, kThreads>(dst, src, tk.r0, tk.I, tk.r1, reinterpret_cast<float*>(sm), C, crank);
    }
    return;
  }
  const TfOut o{p.z_out, p.z_out_log2, p.status, gridDim.x > static_cast<unsigned>(C) ? 1 : 0};
  TfState st;
  tf_body<X3>(p, o, sm, C, crank, st);
  if (p.emit.enabled && !o.skip_copies) {
    const int64_t g = static_cast<int64_t>(crank) * kThreads + threadIdx.x, gs = static_cast<int64_t>(C) * kThreads;
    __syncthreads();
    for (int t = 0; t < p.emit.n_copies; ++t) {
      const CopyTask& tk = p.emit.copy[t];
      const float* __restrict__ src = static_cast<const float*>(tk.src);
      float* __restrict__ dst = static_cast<float*>(tk.dst);
      if (!tk.swap) copy_plain<float>(dst, src, static_cast<int64_t>(tk.r0) * tk.I * tk.r1, g, gs);
      else copy_swap_tiled<float, kThreads>(dst, src, tk.r0, tk.I, tk.r1, reinterpret_cast<float*>(sm + OFF_A), C, crank);
    }
  }
  tf_finish(p, o, sm, C, crank, st);
  cluster.sync();  // peers may still be reading this CTA's shared memory
}

// Full contraction from both ends (as the CUDA-core two-sided kernel): cluster
// 0 sweeps the leading modes, cluster 1 the trailing ones (slices read with
// swapped legs), each writes its environment and scale to the workspace, and
// z = sum E_L * F_R is formed in float64 by pairs of CTAs as their rows are
// ready (no CTA waits for another).
template <bool X3>
__global__ void __launch_bounds__(kThreads, 1) tf_two_sided_kernel(const __grid_constant__ TwoSidedParams tp) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ int s_last;
  __shared__ double s_red[kThreads / 32];
  cg::cluster_group cluster = cg::this_cluster();
  const int C = static_cast<int>(cluster.num_blocks());
  const int crank = static_cast<int>(cluster.block_rank());
  const int side = static_cast<int>(blockIdx.x) / C;
  const SweepParams& p = tp.half[side];
  const TfOut o{nullptr, nullptr, tp.status, 0};
  TfState st;
  tf_body<X3>(p, o, sm, C, crank, st);
  tf_finish(p, o, sm, C, crank, st);  // this CTA's rows u = crank, crank + C, ... written and fenced
  cluster.sync();                     // peers' bulk copies out of this CTA's shared memory are done
  // The join z = sum E_L * F_R is split over pairs: CTA c of each cluster
  // wrote rows u = c, c + C, ... of its side; the second of the pair to
  // arrive forms their partial sum (float64), and the last pair to finish
  // adds the C partial sums in order.  Workspace: counter[0] pairs done,
  // counter[1 + c] arrivals of pair c, 16 doubles of partial sums 128 bytes on.
  int* ctr = tp.counter;
  double* psum = reinterpret_cast<double*>(reinterpret_cast<char*>(tp.counter) + 128);
  if (threadIdx.x == 0) s_last = atomicAdd(ctr + 1 + crank, 1);
  __syncthreads();
  if (s_last != 1) return;
  __threadfence();
  const float* el = static_cast<const float*>(tp.half[0].e_out);
  const float* er = static_cast<const float*>(tp.half[1].e_out);
  const int nrow = tp.rx > crank ? (tp.rx - 1 - crank) / C + 1 : 0;
  double part = 0.0;
  for (int idx = threadIdx.x; idx < nrow * tp.ry; idx += kThreads) {
    const int i = (crank + (idx / tp.ry) * C) * tp.ry + idx % tp.ry;
    part = fma(static_cast<double>(__ldcg(el + i)), static_cast<double>(__ldcg(er + i)), part);
  }
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) sum += s_red[w];
    psum[crank] = sum;
    __threadfence();
    s_last = atomicAdd(ctr, 1);
  }
  __syncthreads();
  if (s_last != C - 1 || threadIdx.x != 0) return;
  __threadfence();
  double z = 0.0;
  for (int c = 0; c < C; ++c) z += __ldcg(psum + c);
  const int64_t log2s = __ldcg(tp.half[0].e_out_log2) + __ldcg(tp.half[1].e_out_log2);
  int st_bits = isfinite(z) ? 0 : TT_STATUS_NONFINITE;
  if (tp.z_out_log2 != nullptr) {
    *tp.z_out = z;
    *tp.z_out_log2 = log2s;
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
    *tp.z_out = v;
  }
  set_status(tp.status, st_bits);
}

template <typename K>
static cudaError_t set_attrs(K kern) {
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(SMEM));
  if (err != cudaSuccess) return err;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

template <typename K, typename P>
static cudaError_t launch(K kern, const P& params, int grid, int C, cudaStream_t s) {
  cudaError_t err = set_attrs(kern);
  if (err != cudaSuccess) return err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, kern, params);
}

}  // namespace tf

cudaError_t launch_tf32_sweep(const SweepParams& p, bool x3, int C, cudaStream_t s) {
  const int grid = p.emit.enabled && p.emit.n_copies > 0 ? 2 * C : C;
  return x3 ? tf::launch(tf::tf_sweep_kernel<true>, p, grid, C, s) : tf::launch(tf::tf_sweep_kernel<false>, p, grid, C, s);
}

cudaError_t launch_tf32_two_sided(const TwoSidedParams& tp, bool x3, int C, cudaStream_t s) {
  return x3 ? tf::launch(tf::tf_two_sided_kernel<true>, tp, 2 * C, C, s)
            : tf::launch(tf::tf_two_sided_kernel<false>, tp, 2 * C, C, s);
}

// Largest power-of-two cluster (<= want) of the tf32 sweep kernel that fits.
int tf32_cluster_size(int want) {
  static int cache[17][8];
  int dev = 0;
  cudaGetDevice(&dev);
  int* slot = (dev >= 0 && dev < 8 && want >= 1 && want <= 16) ? &cache[want][dev] : nullptr;
  if (slot != nullptr && *slot > 0) return *slot;
  if (tf::set_attrs(tf::tf_sweep_kernel<true>) != cudaSuccess || tf::set_attrs(tf::tf_sweep_kernel<false>) != cudaSuccess ||
      tf::set_attrs(tf::tf_two_sided_kernel<true>) != cudaSuccess ||
      tf::set_attrs(tf::tf_two_sided_kernel<false>) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int c = 0;
  for (int C = want; C >= 1; C /= 2) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(tf::kThreads, 1, 1);
    cfg.dynamicSmemBytes = tf::SMEM;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, tf::tf_sweep_kernel<true>, &cfg) == cudaSuccess && n >= 1) {
      c = C;
      break;
    }
    cudaGetLastError();
  }
  if (slot != nullptr && c > 0) *slot = c;
  return c;
}

}  // namespace ttc
