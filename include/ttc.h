/*
 * ttc.h -- C ABI of the GB300 (sm_103a) tensor-train contraction library.
 *
 * The library contracts two tensors held in tensor-train (TT) format along a
 * set of common modes, as in the Tensor-Train Contraction Product (TTCP) of
 * Kisil, Calvi, Konstantinidis, Xu and Mandic, "Reducing Computational
 * Complexity of Tensor Contractions via Tensor-Train Networks"
 * (arXiv 2109.00626).
 *
 * Data model (Def. 7 / Eq. 9): a TT of order N is N cores; core k holds
 *   G_k[r][i][r'],  r < R_k, i < I_k, r' < R_{k+1},  R_0 = R_N = 1,
 * contiguous and row-major in device memory (right rank fastest), and
 *   X[i_0..i_{N-1}] = G_0[:,i_0,:] G_1[:,i_1,:] ... G_{N-1}[:,i_{N-1},:].
 *
 * Conventions common to every call
 *   - Mode k of X is contracted with mode k of Y (same position).  The paper's
 *     TCP (Eq. 8) contracts one mode pair; a set S of pairs is contracted pair
 *     after pair, which is order independent.
 *   - Descriptors (tt_desc) and masks live in HOST memory; core pointers are
 *     DEVICE pointers.  The caller owns every buffer; the library allocates
 *     nothing on any call below except tt_batch_plan (host memory, released by
 *     tt_plan_free) and never synchronises the stream.
 *   - Every compute call is asynchronous on `stream` (NULL = legacy default
 *     stream) and returns a tt_error synchronously: argument and shape errors
 *     are detected on the host before anything is enqueued.
 *   - Conditions found on the device (non-finite values, overflow of the
 *     output after undoing the scaling, a wait that ran out) are OR-ed into the
 *     int32 word `*status_dev` (TT_STATUS_* bits).  The library never clears
 *     it: zero it before the call.  No call traps or faults on bad data.
 *   - Scaling.  Environments are kept as mantissa * 2^e with an exact power of
 *     two folded out whenever their largest entry leaves [2^-s, 2^s]
 *     (s = 32 for float32/bfloat16 arithmetic, 256 for float64), so long
 *     contractions neither overflow nor underflow.  Results may be returned
 *     split as (mantissa, int64 log2 scale).
 */
#ifndef TTC_H
#define TTC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st* tt_stream;

/* Storage type of TT cores. */
typedef enum { TT_F64 = 0, TT_F32 = 1, TT_BF16 = 2 } tt_dtype;

/* Arithmetic used for the core products.
 *   TT_P_NATIVE  products and sums in the storage type (float64 or float32;
 *                for bfloat16 storage: bfloat16 products, float32 sums).
 *   TT_P_BF16    float32 operands rounded to bfloat16, float32 sums (tensor cores).
 *   TT_P_BF16X3  float32 operands split as hi + lo bfloat16 pairs; the
 *                products hi*hi + hi*lo + lo*hi are summed in float32 (tensor
 *                cores), the lo*lo term is dropped.
 *   TT_P_TF32X3  float32 operands split as hi = tf32(x) (rounded to nearest)
 *                and lo = x - hi; all four products hi*hi + hi*lo + lo*hi +
 *                lo*lo summed in float32 (tensor cores, kind::tf32).
 *   TT_P_TF32    float32 operands rounded to tf32, float32 sums (tensor cores). */
typedef enum { TT_P_NATIVE = 0, TT_P_TF32X3 = 1, TT_P_BF16 = 2, TT_P_BF16X3 = 3, TT_P_TF32 = 4 } tt_prec;

/* Layout of a partial contraction's result (see tt_partial_shape). */
typedef enum { TT_LAYOUT_CHAIN = 0, TT_LAYOUT_MERGED = 1 } tt_layout;

/* Return codes. */
typedef enum {
  TT_OK = 0,
  TT_ERR_ARG = -1,         /* NULL pointer, bad enum, order <= 0 or > TT_MAX_ORDER     */
  TT_ERR_SHAPE = -2,       /* ranks do not chain, R_0/R_N != 1, I_k != J_k on S,      */
                           /* orders differ, output shape differs from tt_partial_shape */
  TT_ERR_DTYPE = -3,       /* dtype / precision combination not provided              */
  TT_ERR_LAYOUT = -4,      /* chain layout asked for a contracted set that is not an */
                           /* end block                                              */
  TT_ERR_TOO_LARGE = -5,   /* a rank, mode size or merged core exceeds a stated cap  */
  TT_ERR_WS = -6,          /* workspace smaller than tt_workspace_bytes              */
  TT_ERR_CUDA = -7,        /* a CUDA runtime call failed (launch, attribute query)   */
  TT_ERR_UNSUPPORTED = -8  /* valid request outside what this build implements       */
} tt_error;

/* Bits OR-ed into *status_dev by kernels. */
enum {
  TT_STATUS_NONFINITE = 1, /* an environment or result held Inf/NaN                  */
  TT_STATUS_OVERFLOW = 2,  /* undoing the power-of-two scaling left the float range  */
  TT_STATUS_TIMEOUT = 4    /* a bounded device-side wait gave up                     */
};

#define TT_MAX_ORDER 64

/* One TT operand.  All arrays are host memory; cores[k] is a device pointer to
 * R_k * I_k * R_{k+1} elements of `dtype`, contiguous, row-major. */
typedef struct {
  int32_t order;          /* N >= 1                                              */
  const int32_t* modes;   /* [N]   I_k >= 1                                      */
  const int32_t* ranks;   /* [N+1] R_0 = R_N = 1, R_k >= 1                       */
  void* const* cores;     /* [N]   device pointers                               */
  int32_t dtype;          /* tt_dtype                                           */
} tt_desc;

/* Operation selectors for tt_workspace_bytes. */
enum { TT_OP_FULL = 0, TT_OP_PARTIAL = 1, TT_OP_BACKWARD = 2 };

/* Bytes of device workspace `op` needs for these operands (0 is possible).
 * `mask` (host, [N], 1 = contracted) is ignored for TT_OP_FULL and may be NULL
 * there; for TT_OP_BACKWARD a NULL mask means the full contraction.
 * Returns TT_OK and sets *bytes, or an error code. */
int tt_workspace_bytes(int op, const tt_desc* x, const tt_desc* y, const uint8_t* mask, int layout,
                       int prec, size_t* bytes);

/* Full contraction z = <X, Y> = sum over all indices of X[i] Y[i]
 * (Fig. 1b: contraction along every mode to a scalar; the all-mode
 * generalisation of Algorithm 2 step 4).  X and Y have the same order and mode
 * sizes; ranks are independent.
 *   ws, ws_bytes device workspace.  For float32/float64 products with a
 *                workspace of tt_workspace_bytes(TT_OP_FULL) bytes and order
 *                >= 2, the environment is swept from both ends at once and
 *                the halves meet in the middle (half the dependent steps);
 *                when every rank of Y is 1 (the sum of X's entries, and the
 *                like; X's ranks <= 1024) X's cores are instead folded with
 *                y into matrices M_k = sum_i y_k[i] X_k[:, i, :] in the
 *                workspace and z is a chain of vector-matrix products, its
 *                last one in float64; with ws NULL or smaller the
 *                contraction runs as one sweep.  The tensor-core forms need
 *                their workspace (TT_ERR_WS).
 *   out_dev      device double.  If out_log2_dev is NULL it receives z;
 *                otherwise it receives a mantissa m and *out_log2_dev an int64 e
 *                with z = m * 2^e (use this form when |z| may leave the double
 *                range).
 *   status_dev   device int32, see TT_STATUS_*.
 * Precision: TT_P_NATIVE for F64/F32/BF16 storage; TT_P_BF16, TT_P_BF16X3,
 * TT_P_TF32 and TT_P_TF32X3 for F32 storage.  The final sum of the last mode
 * is accumulated in float64.  The bfloat16 forms run on the tensor cores and
 * need order >= 3, every interior rank of X equal to 128 or 256 and every
 * interior rank of Y a multiple of 64 up to 256; the tf32 forms run the whole
 * sweep (from both ends with the workspace) on the tensor cores and need every
 * rank of both operands <= 64 (TT_ERR_UNSUPPORTED otherwise). */
int tt_contract_full(const tt_desc* x, const tt_desc* y, int prec, double* out_dev,
                     int64_t* out_log2_dev, int32_t* status_dev, void* ws, size_t ws_bytes,
                     tt_stream stream);

/* Shape of the result of a partial contraction over S = {k : mask[k] != 0}
 * (host only, synchronous).  Z has the free modes of X ascending, then the
 * free modes of Y ascending (Eq. 8's order); m = number of free modes >= 1.
 *
 * TT_LAYOUT_CHAIN (S a leading block {0..s-1} or a trailing block
 *   {N-s..N-1}; Algorithm 2 steps 4-6): a TT of order 2m.
 *   leading : cores Gx_{N-1}^T .. Gx_{s+1}^T, C, Gy_s .. Gy_{N-1}
 *             with K = left environment over S and
 *             C[a'][i][b] = sum_a Gx_s[a][i][a'] K[a][b];
 *   trailing: cores Gx_0 .. Gx_{m-2}, C, Gy_{m-1}^T .. Gy_0^T
 *             with K = right environment over S and
 *             C[a][i][b] = sum_a' Gx_{m-1}[a][i][a'] K[a'][b];
 *   G^T exchanges the two rank legs of a core (the paper's T[1;3]).
 * TT_LAYOUT_MERGED (any S): a TT of m cores over the free positions
 *   f_0 < .. < f_{m-1}; core t is [r_t][I_{f_t}][J_{f_t}][r_{t+1}] (stored as
 *   [r_t][I*J][r_{t+1}], i major) holding Gx_{f_t} (x) Gy_{f_t} with pair rank
 *   index a*R^y + b, the environments of the contracted modes folded in.
 *
 * Outputs (host): *z_order = number of cores; z_modes[z_order] = mode size of
 * each core (I*J for merged); z_ranks[z_order+1]; z_perm[2m]: axis p of the
 * represented tensor is axis z_perm[p] of Eq. 8's Z (chain axes follow the
 * cores; merged axes are i_{f_0}, j_{f_0}, i_{f_1}, ...).  Arrays must hold
 * 2*N (+1 for ranks) entries. */
int tt_partial_shape(const tt_desc* x, const tt_desc* y, const uint8_t* mask, int layout,
                     int32_t* z_order, int32_t* z_modes, int32_t* z_ranks, int32_t* z_perm);

/* Partial contraction Z = X x_S Y (Eq. 8 over every pair in S; Algorithm 2
 * steps 4-6 for the chain layout).  `z` describes caller-allocated output
 * cores of exactly the shape tt_partial_shape reports, same dtype as X.
 * An output core may alias the input core it is a plain copy of (chain: the
 * Gy_k of a leading block, the Gx_k of a trailing block); then nothing is
 * copied for it.
 *   z_log2_dev  optional device int64: if non-NULL the power-of-two scale of
 *               the environment is stored there and left out of C (Z = Z_stored
 *               * 2^e); if NULL it is folded into C.  The merged layout always
 *               folds its scales into the cores and stores e = 0.
 * Merged layout: the contracted run after a free core acts on that core's
 * right rank leg; an interior run as its transfer matrix (the run swept from
 * every basis environment, R^x R^y sweeps, each with its own power-of-two
 * scale; a row more than 2^250 (F32) / 2^2000 (F64) below the largest
 * contributes zero), a trailing run as its right environment.  The m output
 * cores are built concurrently: the call forks from `stream` onto up to three
 * library-owned streams of the current device and joins back into `stream`
 * with events, so the result is ordered on `stream` like any other call.  The
 * first merged-layout call on a device creates those streams and four events
 * (never destroyed), so it should be made outside any stream capture.  A
 * captured stream captures the whole fork and join; until that capture ends
 * the auxiliary streams belong to it, so no other merged-layout call on the
 * device may run meanwhile.  Calls are serialised by a host mutex while they
 * enqueue.  TT_ERR_TOO_LARGE when a merged core, its run's transfer matrix or
 * the intermediate P (R^x I R^y' x the next pair rank) exceeds 2^30 entries,
 * or a rank exceeds 128 (F32) / 64 (F64).
 * Precision: TT_P_NATIVE (F64/F32); for the chain layout also TT_P_TF32 and
 * TT_P_TF32X3 on F32 storage with every rank <= 64 (the sweep and the
 * boundary core C on the tensor cores). */
int tt_contract_partial(const tt_desc* x, const tt_desc* y, const uint8_t* mask, int layout,
                        int prec, const tt_desc* z, int64_t* z_log2_dev, int32_t* status_dev,
                        void* ws, size_t ws_bytes, tt_stream stream);

/* The chain-layout partial contraction that also leaves, in `ws`, what its
 * backward pass (tt_contract_backward_k with the same ws) would otherwise
 * recompute: K, the environment over the contracted block (Algorithm 2 step
 * 4), with its scale, and for a leading block every left environment of the
 * block (L_0 .. L_{s-1}, with their scales), which the adjoint's gradient
 * launch reads.
 *   ws, ws_bytes  device workspace of at least tt_workspace_bytes(TT_OP_BACKWARD,
 *                 x, y, mask, TT_LAYOUT_CHAIN, prec) bytes, owned by the caller,
 *                 kept unchanged until the backward call (TT_ERR_WS if short).
 * Everything else as tt_contract_partial with TT_LAYOUT_CHAIN. */
int tt_contract_partial_k(const tt_desc* x, const tt_desc* y, const uint8_t* mask, int prec,
                          const tt_desc* z, int64_t* z_log2_dev, int32_t* status_dev, void* ws,
                          size_t ws_bytes, tt_stream stream);

/* Partial contraction of TTs of different orders over mode pairs: mode
 * xmodes[t] of X (order N) is contracted with mode ymodes[t] of Y (order M),
 * t < n_pairs (Eq. 8 applied to each pair, e.g. Example 1's x_3^2).  The
 * xmodes form a block at one end of X, the ymodes one at one end of Y, and
 * walking both trains from those ends inward meets the pairs in the same
 * order (leading against leading, leading against trailing, ...); else
 * TT_ERR_LAYOUT.  Result: one TT (chain layout) of (N - s) + (M - s) cores,
 * s = n_pairs: an operand whose block is the trailing one is read backwards
 * with its rank legs swapped, so both blocks lead; K is the environment over
 * the pairs; the cores are X's free cores walked from its far end back
 * (legs swapped), C = X's boundary core joined with K, then Y's free cores
 * (Algorithm 2 steps 4-6).  When X has no free mode the roles exchange: Y's
 * free cores walked back, the last of them joined with K^T.
 * tt_pairs_shape (host only, synchronous) reports the output shape and
 * z_perm: axis p of the represented tensor is axis z_perm[p] of Eq. 8's Z
 * (X's free modes ascending, then Y's).  Arrays hold N + M (+1 for ranks)
 * entries.  Mode sizes must agree on every pair (TT_ERR_SHAPE); repeated or
 * out-of-range modes, n_pairs < 1, or every mode of both operands contracted
 * (use tt_contract_full): TT_ERR_ARG.
 * tt_contract_pairs: `z` describes caller-allocated output cores of exactly
 * that shape, same dtype; z_log2_dev as in tt_contract_partial.  Precision:
 * TT_P_NATIVE (F64/F32), TT_P_TF32 and TT_P_TF32X3 (F32, ranks <= 64).
 * Asynchronous on `stream`; no allocation. */
int tt_pairs_shape(const tt_desc* x, const tt_desc* y, int n_pairs, const int32_t* xmodes, const int32_t* ymodes,
                   int32_t* z_order, int32_t* z_modes, int32_t* z_ranks, int32_t* z_perm);
int tt_contract_pairs(const tt_desc* x, const tt_desc* y, int n_pairs, const int32_t* xmodes,
                      const int32_t* ymodes, int prec, const tt_desc* z, int64_t* z_log2_dev,
                      int32_t* status_dev, tt_stream stream);

/* Partial contraction over any contracted set S (Eq. 8 applied to each k in
 * S) in factored form: the merged (TT-matrix) result kept as its Kronecker
 * factors.  With f_0 < ... < f_{m-1} the free positions,
 *   Z[i_F; j_F] = T_0 W_{f_0}[i_0, j_0] T_1 ... W_{f_{m-1}}[i_{m-1}, j_{m-1}] T_m,
 *   W_f[i, j][(a, b), (a', b')] = Gx_f[a][i][a'] Gy_f[b][j][b']  (pair index a R^y + b),
 * i_F in X's free modes, j_F in Y's (Eq. 8's order).  W_f is the operands'
 * own free cores (never formed or copied); T_t is the contracted run between
 * free positions as a matrix over pair indices: T_0 = the left environment
 * of the modes before f_0 (1 x R^x R^y at f_0), T_m = the right environment
 * of the modes after f_{m-1} (R^x R^y at f_{m-1}+1 x 1), and T_t for
 * 0 < t < m the transfer matrix of the modes strictly between f_{t-1} and
 * f_t: row (a, b) is the run swept from the basis environment e_a e_b^T,
 * R^x R^y at f_{t-1}+1 x R^x R^y at f_t.  A run with no mode is the identity
 * and stores nothing (rows = cols = 0).  Row r of T_t is stored as mantissas
 * scaled by 2^{log2_t[r]} (int64; an all-zero row has a large negative
 * scale).  Caps: ranks as tt_contract_full, every T_t at most 2^30 entries
 * (TT_ERR_TOO_LARGE); S = all modes: TT_ERR_ARG.
 * tt_factored_shape (host only) fills `f`: the free positions, each T_t's
 * shape and its byte offsets in one output arena (entries, then rows + 1
 * int64: the row scales and a scratch slot), and the arena size.
 * f->ws_bytes: the device workspace tt_contract_factored needs (0 unless an
 * interior run has R^x R^y >= 256 rows: those are swept for all rows at once
 * as plain GEMMs on cuBLAS, float32 / float64 arithmetic, in chunks that bound
 * the intermediate; smaller runs use one CTA per row).
 * tt_contract_factored: out_dev = a device arena of f->bytes (16-byte
 * aligned); `f` must be the shape of these operands and S (TT_ERR_SHAPE);
 * ws of at least f->ws_bytes (TT_ERR_WS).  The runs are computed one after
 * another on `stream`; no allocation, except that the first call on a
 * stream that takes the GEMM path creates a cuBLAS handle bound to that
 * stream (so that call belongs outside a stream capture); calls on different
 * streams may run concurrently. */
typedef struct {
  int32_t n_free;
  int32_t free_pos[TT_MAX_ORDER];
  int32_t rows[TT_MAX_ORDER + 1];
  int32_t cols[TT_MAX_ORDER + 1];
  size_t off_t[TT_MAX_ORDER + 1];
  size_t off_log2[TT_MAX_ORDER + 1];
  size_t bytes;
  size_t ws_bytes;
} tt_factored;
int tt_factored_shape(const tt_desc* x, const tt_desc* y, const uint8_t* mask, tt_factored* f);
int tt_contract_factored(const tt_desc* x, const tt_desc* y, const uint8_t* mask, const tt_factored* f,
                         void* out_dev, int32_t* status_dev, void* ws, size_t ws_bytes, tt_stream stream);

/* TT decomposition of a dense tensor: the TT-SVD of Section II (Algorithm 1),
 * whose result satisfies ||X - TT(X)||_F <= eps ||X||_F.  x_dev: device,
 * row-major, modes[0] x ... x modes[order-1] (F64 or F32).  Modes are taken
 * left to right: at mode k the unfactored part is a matrix of
 * (r_{k-1} I_k) rows; its SVD (one-sided Jacobi, in the storage type, singular
 * values and norms in float64) keeps the smallest rank r_k >= 1 whose dropped
 * singular values have 2-norm <= eps ||X||_F / sqrt(order - 1), then at most
 * max_rank (0: no cap); core k is the r_k leading left singular vectors
 * (left-orthonormal for k < order - 1), the last core carries the rest.
 * tt_svd_workspace (host only): cap_ranks[order + 1] = the largest ranks the
 * call can return (min of the two unfolding sizes, capped by max_rank) and
 * *ws_bytes; TT_ERR_TOO_LARGE when the shorter side of an unfolding exceeds
 * 512 or the tensor exceeds 2^31 - 1 entries.  tt_svd: cores_dev[k] holds at
 * least cap_ranks[k] * modes[k] * cap_ranks[k+1] elements and receives core k
 * contiguous with its chosen ranks, [r_k][I_k][r_{k+1}]; the chosen ranks go
 * to ranks_dev[order + 1] (device int32; read them after the stream has
 * reached the call).  A non-finite norm sets TT_STATUS_NONFINITE and writes no
 * core.  One cluster launch runs the decomposition (up to 16 CTAs: an SVD
 * whose vectors and rotations fit one CTA's shared memory runs there, larger
 * ones are spread over the cluster by columns; latency-bound: meant for
 * tensors of up to a few million entries).  Asynchronous on `stream`; no
 * allocation. */
int tt_svd_workspace(int order, const int32_t* modes, int dtype, int32_t max_rank, int32_t* cap_ranks,
                     size_t* ws_bytes);
int tt_svd(const void* x_dev, int order, const int32_t* modes, int dtype, double eps, int32_t max_rank,
           void* const* cores_dev, int32_t* ranks_dev, int32_t* status_dev, void* ws, size_t ws_bytes,
           tt_stream stream);

/* TT rounding: the tensor x represents, re-expressed with smaller ranks
 * within eps ||X||_F (the TT-SVD's truncation rule of Section II applied to a
 * TT, e.g. a merged-layout result viewed as a TT of modes I J).  One cluster
 * launch (SVDs as in tt_svd) runs two sweeps of single-core SVDs (one-sided
 * Jacobi, the storage type): right
 * to left making the cores right-orthonormal (only exactly-zero singular
 * values dropped), then left to right keeping, per core, the smallest rank
 * whose dropped singular values have 2-norm <= eps ||X||_F / sqrt(order - 1),
 * then at most max_rank (0: no cap).  cores_out[k] (device) holds at least
 * x's core k (ranks never grow) and receives core k contiguous with the new
 * ranks, which go to ranks_dev[order + 1] (device int32).  F64 / F32; every
 * unfolding's shorter side <= 512 (TT_ERR_TOO_LARGE).  tt_round_workspace
 * (host only) gives the workspace.  Asynchronous on `stream`; no allocation. */
int tt_round_workspace(const tt_desc* x, int32_t max_rank, size_t* ws_bytes);
int tt_round(const tt_desc* x, double eps, int32_t max_rank, void* const* cores_out, int32_t* ranks_dev,
             int32_t* status_dev, void* ws, size_t ws_bytes, tt_stream stream);

/* Dense mode permutation (Alg. 2 steps 1-2: the paired modes brought to the
 * front before the decomposition): out has axis t = axis axes[t] of in
 * (both device, row-major, F64 or F32, distinct buffers).  TT_ERR_ARG for a
 * repeated or out-of-range axis.  Asynchronous on `stream`; no allocation. */
int tt_dense_permute(const void* in_dev, int order, const int32_t* modes, const int32_t* axes, int dtype,
                     void* out_dev, tt_stream stream);

/* ---------------------------------------------------------------------------
 * Batched contraction of many independent pairs in one persistent launch.
 * ------------------------------------------------------------------------- */
typedef struct tt_plan tt_plan;

typedef struct {
  int32_t n_pairs;
  const tt_desc* x;              /* [n_pairs]                                       */
  const tt_desc* y;              /* [n_pairs]                                       */
  const uint8_t* const* mask;    /* [n_pairs]; NULL entry (or NULL array) = full    */
  const tt_desc* z;              /* [n_pairs] chain-layout outputs of partial pairs */
                                 /* (entries of full pairs are ignored; may be NULL */
                                 /* when every pair is full)                        */
  int32_t prec;                  /* TT_P_NATIVE                                     */
} tt_batch;

/* Validate every pair, order the work longest-first, plan each pair's sweep
 * and size the device tables.  The plan of a contracted mode is its
 * evaluation order (E B_i first or A_i^T E first, whichever a cost model of
 * the kernel rates faster) and how many mode slices one panel of the kernel's
 * products takes.  Each pair gets a tile configuration (reported by
 * tt_plan_info as 0..11 = panel-budget level + 3 * replica-cap index): the
 * panel budget is a quarter, half or all of the kernel's buffer (level 0, 1,
 * 2), the replica cap limits the thread groups that split the second product
 * of a slice panel to none, 1, 2 or 4; autotuned per (rank, mode size)
 * bucket (tt_autotune), else 2 (full budget, no cap).  Host only,
 * synchronous, allocates host memory (freed by tt_plan_free).  Returns the
 * bytes of the packed device table (*packed_bytes) and of the workspace
 * (*ws_bytes).  TT_ERR_TOO_LARGE: a swept rank above 128 (F32) / 64 (F64), or
 * a free core copied into a chain output with a right rank above 4096 (F32) /
 * 2048 (F64). */
int tt_batch_plan(const tt_batch* batch, tt_plan** plan, size_t* packed_bytes, size_t* ws_bytes);

/* Write the packed table into host memory `packed_host` (packed_bytes long);
 * the caller copies it to device memory once and passes that copy below. */
int tt_batch_pack(const tt_plan* plan, void* packed_host, size_t packed_bytes);

/* Enqueue the batched contraction.  out_dev: device double[n_pairs], the value
 * of each full pair (mantissa if out_log2_dev is non-NULL, which then receives
 * int64[n_pairs] scales); entries of partial pairs are set to 0.  Partial
 * pairs write their chain-layout cores into the batch's z descriptors (scale
 * folded in).  No allocation, no synchronisation: the call can be captured in
 * a CUDA graph and replayed. */
int tt_contract_batched(const tt_plan* plan, const void* packed_dev, double* out_dev,
                        int64_t* out_log2_dev, int32_t* status_dev, void* ws, size_t ws_bytes,
                        tt_stream stream);

/* The same batched contraction for callers that cannot allocate device
 * memory where they contract -- a plugin inside a framework that owns every
 * device allocation, or a loop that must not allocate once running -- and so
 * have no workspace to pass.  (The paper has no counterpart to this call.)
 * The work-queue counter lives in a fixed array inside the library instead:
 * TT_NOALLOC_SCRATCH_BYTES bytes of static device memory that every GPU which
 * loads the library holds until the process exits.  Plans whose workspace
 * (tt_batch_plan's *ws_bytes) exceeds that size are rejected with
 * TT_ERR_WS.  The call allocates and frees nothing; it zeroes what must
 * start at zero and otherwise behaves like tt_contract_batched.  Each call
 * made outside a stream capture looks up the array's device address on the
 * current device (so a context re-created after cudaDeviceReset is followed);
 * a call made during a capture reuses the address found by the last call
 * outside one, so the first call on a device comes before any capture.  Every call
 * shares the one array, which keeps the last call's contents: calls whose
 * executions overlap on the GPU race with each other. */
#define TT_NOALLOC_SCRATCH_BYTES 256
int tt_contract_batched_noalloc(const tt_plan* plan, const void* packed_dev, double* out_dev,
                                int64_t* out_log2_dev, int32_t* status_dev, tt_stream stream);

/* Number of pairs and the tile configuration chosen for pair p (for tests and
 * reports); returns TT_ERR_ARG for p out of range. */
int tt_plan_info(const tt_plan* plan, int32_t p, int32_t* n_pairs, int32_t* tile_config);

void tt_plan_free(tt_plan* plan);

/* Tile autotuner for the batched launch.  For every (rank bucket <= 16, <= 32,
 * <= 64, <= 128) x (mode-size bucket <= 4, <= 8, <= 16, <= 32, > 32) it times
 * each of the 12 tile configurations (see tt_batch_plan) on a batch of
 * order-6 full contractions of that rank and mode size filling the GPU (two
 * per SM), with seeded random cores that are distinct per pair up to 2 GiB
 * (so they stream from memory, not from L2), the median of three launches
 * after a warm-up; a configuration other than 2 is chosen only when it is at
 * least 3 % faster than configuration 2.  Writes text lines
 * "dtype rank_bucket mode_bucket config" to `cache_path`.  tt_batch_plan reads the file named by the environment
 * variable TTC_AUTOTUNE_CACHE (without it, configuration 2 is used).
 * Synchronous; unlike every other call it allocates (and frees) device memory
 * and must not be called during stream capture. */
int tt_autotune(int dtype, const char* cache_path);

/* ---------------------------------------------------------------------------
 * Adjoint.
 * ------------------------------------------------------------------------- */
/* Gradients of a full or partial contraction with respect to every core of
 * both operands.
 *   mask == NULL     full contraction; cot_dev = device double, the cotangent
 *                    of z; dz ignored.
 *   mask != NULL     chain-layout partial contraction; dz describes the
 *                    cotangent of every output core (device, same shapes as
 *                    the output), cot_dev ignored.
 *   gx, gy           caller-allocated gradient cores, shapes of x and y.
 *   ckpt_stride      >= 0, not otherwise used: every left environment is
 *                    kept (N of them, and N right environments: the
 *                    gradients of all modes are formed by one launch after
 *                    the backward sweep; TT_ERR_ARG when negative).
 * For a full contraction, dz/dGx_k[:,i,:] = L_k Gy_k[:,i,:] F_{k+1}^T and
 * dz/dGy_k[:,i,:] = L_k^T Gx_k[:,i,:] F_{k+1}, where L_k / F_{k+1} are the left
 * / right environments; a chain-layout partial contraction reduces to this with
 * the cotangent of its K as the boundary environment.  A full contraction whose
 * y has every rank 1 (e.g. the sum of x's entries, y = all ones) takes a vector
 * path: the environments are vectors, all of them kept (ckpt_stride unused),
 * and x's ranks may go up to 1024.
 * Precision: TT_P_NATIVE (F64/F32). */
int tt_contract_backward(const tt_desc* x, const tt_desc* y, const uint8_t* mask, int layout,
                         int prec, const double* cot_dev, const tt_desc* dz, const tt_desc* gx,
                         const tt_desc* gy, int32_t ckpt_stride, int32_t* status_dev, void* ws,
                         size_t ws_bytes, tt_stream stream);

/* tt_contract_backward of a chain-layout partial contraction run with
 * tt_contract_partial_k: `ws` is the workspace that call filled (same x, y,
 * mask), so K is not swept again and, for a leading block, the adjoint starts
 * from the left environments that call stored.  Arguments as
 * tt_contract_backward (mask required, TT_LAYOUT_CHAIN). */
int tt_contract_backward_k(const tt_desc* x, const tt_desc* y, const uint8_t* mask, int prec,
                           const tt_desc* dz, const tt_desc* gx, const tt_desc* gy,
                           int32_t* status_dev, void* ws, size_t ws_bytes, tt_stream stream);

/* ---------------------------------------------------------------------------
 * Misc.
 * ------------------------------------------------------------------------- */
/* Static text for a tt_error code. */
const char* tt_error_string(int code);

/* Number of kernel launches the library has enqueued since load (all calls,
 * all threads); used to report how many of this library's kernels ran. */
uint64_t tt_launch_count(void);

/* Self-test of the device-side bounded waits (the paper has no counterpart):
 * one CTA runs the bounded mbarrier wait that the pipelined kernels use, with
 * a limit of `limit_cycles` SM clock cycles (0 .. 10^9, the kernels' own
 * limit), on a barrier whose phase completes before the wait (complete != 0)
 * or never does (complete == 0).  A wait that runs out sets TT_STATUS_TIMEOUT
 * in *status_dev (device int32); nothing asynchronous is in flight, so the
 * kernel returns normally either way.  TT_ERR_ARG for a NULL status or a limit
 * out of range. */
int tt_selftest_wait(int complete, int64_t limit_cycles, int32_t* status_dev, tt_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* TTC_H */
