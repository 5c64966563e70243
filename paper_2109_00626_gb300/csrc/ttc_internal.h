// Internal declarations shared by the host API and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include <cuda.h>
#include <cuda_bf16.h>

#include "../../include/ttc.h"

namespace ttc {

constexpr int kMaxOrder = TT_MAX_ORDER;

// Power-of-two renormalisation thresholds: an environment whose largest
// magnitude leaves [2^-s, 2^s] is rescaled by an exact power of two.
constexpr int kRenormBitsF32 = 32;
constexpr int kRenormBitsF64 = 256;

// One step of an environment sweep.  The generic step is
//   E'[u][v] = sum_i sum_{p,q} A_i[p][u] E[p][q] B_i[q][v]
// where, for a left-to-right sweep over core k (ranks R_k -> R_{k+1}),
//   A_i[p][u] = Gx_k[p][i][u],  B_i[q][v] = Gy_k[q][i][v],
// and for a right-to-left sweep (ranks R_{k+1} -> R_k)
//   A_i[p][u] = Gx_k[u][i][p],  B_i[q][v] = Gy_k[v][i][q].
struct SweepStep {
  const void* gx;
  const void* gy;
  int I;
  int rin_x, rout_x;  // p range, u range
  int rin_y, rout_y;  // q range, v range
  // Batched engine only (filled by plan_engine_steps): evaluation order
  // (0: T_i = E B_i first, 1: U_i = A_i^T E first), slices per panel, and a
  // cap on the replica thread groups of the second product (0 = none).
  int ord;
  int g;
  int rcap;
};

// Geometry limits of the per-CTA engine of the batched launch (pair_engine.cuh);
// the host planner chooses each step's order and panel within them.
constexpr int kEngThreads = 512;  // threads of a batched-engine CTA
template <typename T>
struct EngLimits;
template <>
struct EngLimits<float> {
  static constexpr int RM = 128;          // largest rank
  static constexpr int V = 4;             // elements per 16 bytes
  static constexpr int LDE = RM + V;      // environment row stride
  static constexpr int TBUF = RM * LDE;   // T panel / reduction scratch (elements)
  static constexpr int STAGE = 32 * LDE;  // one pipeline stage (elements)
  static constexpr int WMAX = 512;        // widest panel (columns)
  static constexpr int TILES = 16384;     // r8(m) * r8(panel width) cap (two 4x4 tiles per thread)
};
template <>
struct EngLimits<double> {
  static constexpr int RM = 64;
  static constexpr int V = 2;
  static constexpr int LDE = RM + V;
  static constexpr int TBUF = RM * LDE;
  static constexpr int STAGE = 32 * LDE;
  static constexpr int WMAX = 256;
  static constexpr int TILES = 4096;      // one 4x4 tile per thread for both products
};

// Copy / leg-swap of one free core into the chain-layout output.
struct CopyTask {
  const void* src;
  void* dst;
  int r0, I, r1;  // source core shape [r0][I][r1]
  int swap;       // 1: dst[r1][I][r0] = src[r0][I][r1]
};
constexpr int kMaxCopies = 2 * kMaxOrder;

// Boundary core of a chain-layout partial contraction, C = (core of X) joined
// with the environment K of the contracted block.
//   lead : C[u][i][y] = sum_a gx[a][i][u] K[a][y]   (gx is [ra][I][rb], u < rb)
//   trail: C[u][i][y] = sum_b gx[u][i][b] K[b][y]   (gx is [ra][I][rb], u < ra)
struct EmitParams {
  int enabled;
  const void* gx;
  int ra, I, rb;
  int lead;
  int ry;               // columns of K
  void* c_out;
  int64_t* z_log2_out;  // optional: scale of K stored here instead of folded into C
  int n_copies;
  CopyTask copy[kMaxCopies];
};

struct SweepParams {
  int n_steps;            // contracted modes in the sweep (may be 0 for an emission only)
  int transposed;         // 1 = X's slices read with swapped legs (right-to-left sweep)
  int transposed_y;       // the same for Y (equal to `transposed` except for mode pairs
                          // that walk one operand forwards and the other backwards)
  int final_scalar;       // 1 = the last step ends at a 1x1 environment summed in float64
  int renorm_bits;
  SweepStep step[kMaxOrder];
  int rx0, ry0;           // shape of the start environment [1] (both 1)
  void* e_out;            // optional final environment [rx][ry], row-major
  int64_t* e_out_log2;    // scale of e_out (written when e_out is set)
  double* z_out;          // final scalar (final_scalar == 1)
  int64_t* z_out_log2;    // optional; if NULL the scale is folded into *z_out
  int32_t* status;
  EmitParams emit;        // fused chain emission after the sweep (partial contractions)
  // optional checkpoints of a left-to-right sweep for a later adjoint: the
  // environment before modes 0, c, 2c, ... (ckpt_n of them, c = ckpt_stride),
  // each row-major at ckpt + g * ckpt_elems, its scale in ckpt_log2[g]
  void* ckpt;
  int64_t* ckpt_log2;
  int ckpt_stride, ckpt_n;
  int64_t ckpt_elems;     // may be negative (environments stored in reverse order)
  // optional start environment instead of [1]: [rx0][ry0] row-major, the sum
  // of e_seed_parts consecutive such matrices, its scale in *e_seed_log2
  const void* e_seed;
  const int64_t* e_seed_log2;
  int e_seed_parts;
};

// Full contraction as two half sweeps meeting in the middle (sweep.cu):
// half[0] covers the leading modes left to right, half[1] the trailing ones
// right to left; both end with an environment of shape rx x ry in e_out (with
// its scale in e_out_log2).
struct TwoSidedParams {
  SweepParams half[2];
  int rx, ry;
  double* z_out;
  int64_t* z_out_log2;  // optional; if NULL the scale is folded into *z_out
  int32_t* status;
  int* counter;         // zeroed before the launch
};

// One mode of an adjoint block (left-to-right orientation): core k of X is
// [rx][I][rx2], of Y [ry][I][ry2]; dgx / dgy receive the gradients.
struct AdjStep {
  const void* gx;
  const void* gy;
  void* dgx;
  void* dgy;
  int I, rx, rx2, ry, ry2;
  const void* gxs;  // optional leg-swapped copy of gx, [rx2][I][rx]
};

// Gradients of an adjoint block from its stored environments (adjoint.cu):
// L_k for k >= 1 at lenv + k env_elems (scale lenv_log2[k]), F_{k+1} for
// k <= n - 2 at fenv + k env_elems (scale fenv_log2[n - 1 - k], the order a
// right-to-left sweep writes them in); L_0 and F_n are the seeds.
struct AdjointParams {
  int n;                 // modes in the block
  AdjStep step[kMaxOrder];
  const void* l_seed;    // L_0 [rx(0)][ry(0)] (NULL = [1])
  const int64_t* l_seed_log2;
  const void* f_seed;    // F_n [rx2(n-1)][ry2(n-1)] (NULL = [1])
  const int64_t* f_seed_log2;
  int seed_parts;        // a seed is the sum of this many consecutive matrices (0 or 1 = one)
  const double* cot;     // optional scalar multiplier (device)
  const void* lenv;
  const int64_t* lenv_log2;
  const void* fenv;
  const int64_t* fenv_log2;
  int64_t env_elems;     // elements per stored environment
  int total_slices;      // sum of step[k].I (blocks of the launch)
  int32_t* status;
};

// Adjoint of a full contraction whose Y has every rank 1 (adjoint_r1.cu): the
// environments are vectors, kept for every mode.
constexpr int kR1MaxRank = 1024;  // ranks of X on this path
struct AdjR1Params {
  int n;
  AdjStep step[kMaxOrder];   // gx, gy, dgx, dgy, I, rx, rx2 (ry = ry2 = 1)
  void* lvec;                // [n + 1][vstride] L_0 .. L_n
  void* fvec;                // [n + 1][vstride] F_0 .. F_n
  int64_t* llog;             // [n + 1] power-of-two scales of L_k
  int64_t* flog;             // [n + 1] power-of-two scales of F_k
  int64_t vstride;
  int renorm_bits;
  const double* cot;         // scalar multiplier (device; NULL = 1)
  int32_t* status;
  // the folded cores M_k = sum_i y_k[i] Gx_k[:, i, :] ([rx][rx2] at
  // mbuf + moff[k]) and their transposes (at mtbuf + moff[k]; the adjoint only)
  void* mbuf;
  void* mtbuf;
  int64_t moff[kMaxOrder];
  // forward only: z = L_n, written as a float64 value (and exponent)
  int fwd;
  double* z_out;
  int64_t* z_out_log2;       // optional; if NULL the scale is folded into *z_out
};
cudaError_t launch_adjoint_r1(const AdjR1Params& p, int dtype, cudaStream_t s);
// <X, Y> for a Y of rank 1: fold, then one chain of vector-matrix products.
cudaError_t launch_full_r1(const AdjR1Params& p, int dtype, cudaStream_t s);

// Most slice groups dK is split into (each group's partial sum is written
// separately and the adjoint adds them as it loads its seed).
constexpr int kDkGroups = 8;

// Cotangents of a chain-layout output -> boundary-core gradient, dK and the
// free-core gradients (see adjoint.cu).
struct ChainAdjParams {
  const void* gx;
  int ra, I, rb;
  int lead;
  int ry;
  const void* k;
  const int64_t* k_log2;
  const void* dc;
  void* dgx;
  void* dk;  // NULL when the contracted block is empty; else dk_parts partial sums
  int dk_parts;  // dK is summed over slice groups: partial g covers slices [g I / parts, (g + 1) I / parts)
  int n_copies;
  CopyTask copy[kMaxCopies];
  int n_copy_jobs;  // jobs the copies are cut into (set by the launch)
  int32_t* status;
};

// Left core of the merged layout with the left environment folded in (see
// merged.cu): V = E_L Gy, whose largest binary exponent ev is folded into
// *vexp (atomic max; the slot is filled with the byte 0xC0 first), then
// W_0 = sum_a Gx[a] 2^-ev V[a], of scale 2^(*el_log2 + ev): applied with
// saturation when scale_out is set, else written to *wexp.  el == NULL (with
// el_log2 == NULL) stands for E_L = [1] (the first mode is free).
struct KronParams {
  const void* gx;
  const void* gy;
  int rx, ry, I, J, rx2, ry2;
  void* out;
  const void* el;           // left environment folded into the first core
  const int64_t* el_log2;
  void* tmp;                // V = E_L Gy
  int64_t* vexp;
  int64_t* wexp;
  int scale_out;
  int32_t* status;
};

// Transfer matrix of an interior contracted run (merged layout):
//   M[(a, b)][(c, d)] = the run swept from the basis environment e_a e_b^T,
// row (a, b) = a * R^y_in + b, column (c, d) = c * R^y_out + d; each row is
// kept with its own power-of-two scale mexp[row] (kMergedZeroExp for a zero
// row), and the largest of them is folded into *emax (atomic max; the slot is
// filled with the byte 0xC0 first, i.e. kMergedNoExp).
struct TransferParams {
  int n_steps;
  SweepStep step[kMaxOrder];
  void* m;
  int64_t* mexp;
  int64_t* emax;
  int32_t* status;
};
constexpr int64_t kMergedZeroExp = INT64_MIN / 4;
constexpr int64_t kMergedNoExp = static_cast<int64_t>(0xC0C0C0C0C0C0C0C0ull);  // < kMergedZeroExp

// out[r][z][c] = sum_k A[r][k] 2^(mexp[k es + z ez] - *emax) B[k][z][c]
// (row strides lda, ldb, ldo; slice offsets bz, oz), scaled by
// 2^(*out_log2 + *emax) with saturation when out_log2 is set; when oexp is
// set, the largest binary exponent of the output is folded into *oexp
// (atomic max; the slot is filled with the byte 0xC0 first).
struct ScaledGemmParams {
  const void* a;
  const void* b;
  void* out;
  int64_t lda, ldb, bz, ldo, oz;
  int rows, K, C, nz;
  const int64_t* mexp;
  int64_t es, ez;
  const int64_t* emax;
  const int64_t* out_log2;
  int64_t* oexp;
  int32_t* status;
};

// Rows of a merged core W_t[(a, b)][i][j][col] (row ((a ry + b) I + i) J + j):
//   kron: col = c ry2 + d, W = Gx[a][i][c] Gy[b][j][d];
//   prod: W = 2^(*e + *ep) sum_b' Gy[b][j][b'] 2^(-*ep) P[a I + i][b'][col]
//         (b' < ry2; *ep is the largest binary exponent of P).
struct ZRowsParams {
  const void* gx;
  const void* gy;
  const void* p;
  const int64_t* e;
  const int64_t* ep;
  void* out;
  int rx, ry, I, J, rx2, ry2, C;
  int32_t* status;
};

// One interior mode of the tensor-core full contraction (see tc_sweep.cu).
struct TcModeParams {
  CUtensorMap gx_hi, gx_lo, gy_hi, gy_lo;  // 3D maps over [R][I][R'] bfloat16 cores, box (64, 1, 64)
  int x3;
  int rx, rx2, ry, ry2, I;
  const __nv_bfloat16* e_hi;  // input environment: ry/64 K-major panels of rx rows x 128 bytes
  const __nv_bfloat16* e_lo;
  const int* bmax_in;         // binary-exponent maxima of the input environment, per producing block
  int n_bmax_in;
  const int64_t* l_in;        // log2 scale of the input environment
  __nv_bfloat16* eo_hi;       // output environment panels (ry2/64 panels of rx2 rows)
  __nv_bfloat16* eo_lo;
  float* eo_f32;              // output environment, float32 row-major [rx2][ry2]
  int* bmax_out;              // [gridDim.x]
  int64_t* l_out;
  int32_t* status;
};

cudaError_t tc_split(const float* src, void* hi, void* lo, int64_t n, cudaStream_t s);
cudaError_t tc_first(const void* x0, const void* y0, bool f32_in, int I, int rx2, int ry2, float* eo_f32, void* eo_hi,
                     void* eo_lo, int* bmax_out, int64_t* l_out, int32_t* status, cudaStream_t s);
cudaError_t tc_last(const float* e, const void* x, const void* y, bool f32_in, int I, int rx, int ry, double* parts,
                    const int64_t* l_in, double* out, int64_t* out_log2, int32_t* status, cudaStream_t s);
cudaError_t tc_mode(const TcModeParams& p, int cluster, cudaStream_t s);
int tc_cluster_size(bool x3, int want);

// Launchers (return cudaError_t of the launch).
cudaError_t launch_kron0(const KronParams& p, int which, int dtype, cudaStream_t s);
cudaError_t launch_transfer(const TransferParams& p, int dtype, cudaStream_t s);
cudaError_t launch_scaled_gemm(const ScaledGemmParams& p, int dtype, cudaStream_t s);
cudaError_t launch_zrows(const ZRowsParams& p, bool prod, int dtype, cudaStream_t s);
cudaError_t launch_adjoint_grads(const AdjointParams& p, int dtype, int rmax, cudaStream_t s);

// Leg-swapped copies of whole cores (dst[r1][I][r0] = src[r0][I][r1]) as copy
// jobs (copy_jobs.cuh): lets a right-to-left environment sweep read its
// slices as a left-to-right one does, 16 bytes a copy.
struct SwapParams {
  int n_copies, n_jobs;
  CopyTask copy[kMaxCopies];
};
cudaError_t launch_swap_copies(const SwapParams& p, int dtype, cudaStream_t s);
cudaError_t launch_chain_adjoint(const ChainAdjParams& p, int dtype, cudaStream_t s);
cudaError_t launch_sweep_f32(const SweepParams& p, int rmax, int cluster, cudaStream_t s);
cudaError_t launch_sweep_f64(const SweepParams& p, int rmax, int cluster, cudaStream_t s);
cudaError_t launch_two_sided(const TwoSidedParams& tp, int dtype, int rmax, int cluster, cudaStream_t s);
// Tensor-core (tf32) sweeps for float32 cores with ranks <= 64 (tf32_sweep.cu).
constexpr int kTf32MaxRank = 64;
cudaError_t launch_tf32_sweep(const SweepParams& p, bool x3, int cluster, cudaStream_t s);
cudaError_t launch_tf32_two_sided(const TwoSidedParams& tp, bool x3, int cluster, cudaStream_t s);
int tf32_cluster_size(int want);

// One piece of a free-core copy: slices [i0, i1) and left-rank rows [a0, a1)
// of a core [r0][I][r1]; swap = 1 writes it as [r1][I][r0].
struct CopyJob {
  const void* src;
  void* dst;
  int r0, I, r1;
  int swap;
  int i0, i1;
  int a0, a1;
};

// Bytes one copy job moves at most (a job is staged whole in shared memory).
constexpr int kCopyJobBytes = 16384;

// How a copy task is cut into jobs: per slices and rows left-rank rows a job,
// n_i x n_a jobs.  Slices of at most kCopyJobBytes go whole, several to a job;
// a larger slice is cut by rows (r1 <= kCopyJobBytes / elem_bytes).
struct CopyCut {
  int per, rows, n_i, n_a;
};
__host__ __device__ inline CopyCut copy_cut(int r0, int I, int r1, int elem_bytes) {
  const int cap = kCopyJobBytes / elem_bytes;
  const int slice = r0 * r1 > 1 ? r0 * r1 : 1;
  CopyCut c;
  c.per = cap / slice > 1 ? cap / slice : 1;
  c.rows = slice <= cap ? r0 : (r1 > 0 && cap / r1 > 1 ? cap / r1 : 1);
  c.n_i = (I + c.per - 1) / c.per;
  c.n_a = (r0 + c.rows - 1) / c.rows;
  return c;
}
// Job j (< n_i * n_a) of the task.
__host__ __device__ inline CopyJob copy_job_at(const CopyTask& t, const CopyCut& c, int j) {
  const int qi = j / c.n_a, qa = j - qi * c.n_a;
  CopyJob job;
  job.src = t.src;
  job.dst = t.dst;
  job.r0 = t.r0;
  job.I = t.I;
  job.r1 = t.r1;
  job.swap = t.swap;
  job.i0 = qi * c.per;
  job.i1 = job.i0 + c.per < t.I ? job.i0 + c.per : t.I;
  job.a0 = qa * c.rows;
  job.a1 = job.a0 + c.rows < t.r0 ? job.a0 + c.rows : t.r0;
  return job;
}

cudaError_t launch_batched(const void* table, const int32_t* order, const int32_t* tile, int n,
                           const CopyJob* jobs, int n_jobs, int* counters, double* out, int64_t* out_log2,
                           int32_t* status, int dtype, int grid, cudaStream_t s);

// Largest cluster size (<= want) the sweep kernel for this rank tile can run with.
int sweep_cluster_size(int rmax, int elem_bytes, int want);

extern std::atomic<uint64_t> g_launches;
inline void count_launch(uint64_t n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

}  // namespace ttc
