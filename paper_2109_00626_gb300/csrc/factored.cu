// Partial contraction over any contracted set S in factored form: the merged
// (TT-matrix) result of Eq. 8 kept as its Kronecker factors.  With
// f_0 < ... < f_{m-1} the free positions,
//   Z[i_F; j_F] = T_0 W_{f_0}[i_0, j_0] T_1 ... W_{f_{m-1}}[i_{m-1}, j_{m-1}] T_m,
//   W_f[i, j][(a, b), (a', b')] = Gx_f[a][i][a'] Gy_f[b][j][b'],
// where W_f is never formed (the operands' own free cores are its factors)
// and T_t is the contracted run between free positions as a matrix over pair
// indices a R^y + b: T_0 = E_L (1 x R^x R^y, the left environment of the
// contracted modes before f_0), T_m = E_R (R^x R^y x 1, the right
// environment after f_{m-1}), and for 0 < t < m the transfer matrix of the
// modes strictly between f_{t-1} and f_t (row (a, b) = the run swept from the
// basis environment e_a e_b^T).  An empty run is the identity and is not
// stored.  The output holds R^4-sized run matrices instead of merged cores of
// R^x R^y I J R^x' R^y' entries, so it exists at ranks where the merged layout
// does not.
//
// The end environments come from the environment sweeps (sweep_body.cuh);
// interior runs from transfer_kernel (merged.cu) when small, else from plain
// GEMMs over all rows at once (below); each row keeps its own power-of-two
// scale.
#include <cublas_v2.h>
#include <limits.h>
#include <string.h>

#include <map>
#include <mutex>
#include <utility>

#include "host_plan.h"
#include "ttc_device.cuh"

namespace ttc {

// Interior runs with at least this many rows (pair ranks R^x R^y at the
// run's start) are swept for all rows at once as plain GEMMs: with E_q the
// environment of row q (R^x x R^y),
//   T[(q, c)][(i, v)] = sum_d E_q[c][d] Gy[d][i][v]          (one GEMM, K = R^y)
//   E'_q[u][v] = sum_{c,i} Gx[c][i][u] T[(q, c)][(i, v)]      (a strided batch over q, K = R^x I)
// on cuBLAS (SGEMM / DGEMM, no reduced-precision math), in chunks of rows
// that bound the intermediate T; each row is renormalised by a power of two
// after every mode.  The first mode of the run, from the basis environment
// e_a e_b^T, is E_q[u][v] = sum_i Gx[a][i][u] Gy[b][i][v] (run_first_kernel).
// Smaller runs use transfer_kernel, one CTA per row.
constexpr int kGemmRunRows = 256;

static int sm_count_dev() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}
constexpr int64_t kGemmChunkElems = int64_t(1) << 26;  // intermediate T per chunk

template <typename T>
__global__ void run_first_kernel(const T* __restrict__ gx, const T* __restrict__ gy, int ry, int I, int rx2, int ry2,
                                 int64_t n, T* __restrict__ e) {
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < n;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int v = static_cast<int>(idx % ry2);
    const int64_t r = idx / ry2;
    const int u = static_cast<int>(r % rx2);
    const int q = static_cast<int>(r / rx2);
    const int a = q / ry, b = q - a * ry;
    const T* xa = gx + static_cast<int64_t>(a) * I * rx2 + u;
    const T* yb = gy + static_cast<int64_t>(b) * I * ry2 + v;
    T acc = T(0);
    for (int i = 0; i < I; ++i) acc = fma(xa[static_cast<int64_t>(i) * rx2], yb[static_cast<int64_t>(i) * ry2], acc);
    e[idx] = acc;
  }
}

// Row q of e (n_row entries) scaled by 2^-m, m its largest binary exponent,
// and m added to log2[q]; an all-zero row gets the zero marker (and keeps
// it); non-finite entries set TT_STATUS_NONFINITE.  One block per row.
template <typename T>
__global__ void renorm_rows_kernel(T* __restrict__ e, int64_t n_row, int rows, int64_t* __restrict__ log2,
                                   int32_t* status) {
  __shared__ int red[8];
  __shared__ int bad_s;
  for (int q = blockIdx.x; q < rows; q += gridDim.x) {
    T* row = e + static_cast<int64_t>(q) * n_row;
    int m = INT_MIN, bad = 0;
    for (int64_t k = threadIdx.x; k < n_row; k += blockDim.x) {
      const T v = row[k];
      if (!isfinite(v)) bad = 1;
      else if (v != T(0)) m = max(m, exp2_bits(v));
    }
    if (threadIdx.x == 0) bad_s = 0;
    m = __reduce_max_sync(0xffffffffu, m);
    bad = __reduce_or_sync(0xffffffffu, bad);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    if (bad) bad_s = 1;
    __syncthreads();
    m = INT_MIN;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) m = max(m, red[w]);
    const int64_t cur = log2[q];
    if (m == INT_MIN || cur == kMergedZeroExp) {
      if (threadIdx.x == 0) log2[q] = kMergedZeroExp;
    } else {
      for (int64_t k = threadIdx.x; k < n_row; k += blockDim.x) row[k] = mul_pow2<T>(row[k], -m);
      if (threadIdx.x == 0) log2[q] = cur + m;
    }
    if (threadIdx.x == 0 && bad_s) atomicOr(status, TT_STATUS_NONFINITE);
    __syncthreads();
  }
}

// One cuBLAS handle per (device, stream), created on the first GEMM-path
// call on that stream (it allocates cuBLAS's own workspace, so that first
// call belongs outside a stream capture) and bound to the stream for good:
// calls on different streams may run at the same time without sharing a
// cuBLAS workspace.  The table is guarded by a lock.
static std::mutex g_blas_mu;
static std::map<std::pair<int, cudaStream_t>, cublasHandle_t> g_blas;

static cublasHandle_t blas_handle(cudaStream_t s) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  const auto key = std::make_pair(dev, s);
  auto it = g_blas.find(key);
  if (it != g_blas.end()) return it->second;
  cublasHandle_t h = nullptr;
  if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return nullptr;
  if (cublasSetMathMode(h, CUBLAS_DEFAULT_MATH) != CUBLAS_STATUS_SUCCESS || cublasSetStream(h, s) != CUBLAS_STATUS_SUCCESS) {
    cublasDestroy(h);
    return nullptr;
  }
  g_blas.emplace(key, h);
  return h;
}

// Row-major C (M x N) = E (M x K) Gy (K x N): column-major C^T = Gy^T E^T.
static cublasStatus_t gemm_rm(cublasHandle_t h, int dtype, int M, int N, int K, const void* a, const void* b, void* c) {
  if (dtype == TT_F64) {
    const double one = 1.0, zero = 0.0;
    return cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, N, M, K, &one, static_cast<const double*>(b), N,
                       static_cast<const double*>(a), K, &zero, static_cast<double*>(c), N);
  }
  const float one = 1.f, zero = 0.f;
  return cublasSgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, N, M, K, &one, static_cast<const float*>(b), N,
                     static_cast<const float*>(a), K, &zero, static_cast<float*>(c), N);
}

// For q < batch, row-major C_q (M x N) = Gx^T (M x K) T_q (K x N), Gx stored
// row-major K x M, T_q = t + q K N, C_q = c + q M N.  Column-major:
// C_q^T (N x M) = T_q^T (N x K) Gx (K x M).
static cublasStatus_t gemm_at_b_batched(cublasHandle_t h, int dtype, int M, int N, int K, const void* gx,
                                        const void* t, void* c, int batch) {
  const long long st = static_cast<long long>(K) * N, sc = static_cast<long long>(M) * N;
  if (dtype == TT_F64) {
    const double one = 1.0, zero = 0.0;
    return cublasDgemmStridedBatched(h, CUBLAS_OP_N, CUBLAS_OP_T, N, M, K, &one, static_cast<const double*>(t), N,
                                     st, static_cast<const double*>(gx), M, 0, &zero, static_cast<double*>(c), N, sc,
                                     batch);
  }
  const float one = 1.f, zero = 0.f;
  return cublasSgemmStridedBatched(h, CUBLAS_OP_N, CUBLAS_OP_T, N, M, K, &one, static_cast<const float*>(t), N, st,
                                   static_cast<const float*>(gx), M, 0, &zero, static_cast<float*>(c), N, sc, batch);
}

// Workspace of the GEMM path for the interior run k0 .. k1-1: two
// environment buffers (rows x the largest R^x R^y inside the run) and one
// chunk of the intermediate T.
static size_t gemm_run_ws(const tt_desc* x, const tt_desc* y, int k0, int k1, int64_t rows) {
  const size_t eb = static_cast<size_t>(elem_bytes(x->dtype));
  int64_t emax = 1, tmax = 1;
  for (int k = k0; k < k1; ++k) {
    emax = std::max<int64_t>(emax, static_cast<int64_t>(x->ranks[k + 1]) * y->ranks[k + 1]);
    if (k > k0) {
      const int64_t per = static_cast<int64_t>(x->ranks[k]) * x->modes[k] * y->ranks[k + 1];
      const int64_t q = std::max<int64_t>(1, std::min<int64_t>(rows, kGemmChunkElems / per));
      tmax = std::max(tmax, q * per);
    }
  }
  return 2 * align256(static_cast<size_t>(rows * emax) * eb) + align256(static_cast<size_t>(tmax) * eb);
}

template <typename T>
static int gemm_run(const tt_desc* x, const tt_desc* y, int k0, int k1, int rows, void* out, int64_t* lg,
                    char* ws, int32_t* status, cudaStream_t s) {
  const int dtype = x->dtype;
  const size_t eb = sizeof(T);
  int64_t emax = 1;
  for (int k = k0; k < k1; ++k) emax = std::max<int64_t>(emax, static_cast<int64_t>(x->ranks[k + 1]) * y->ranks[k + 1]);
  T* eb0 = reinterpret_cast<T*>(ws);
  T* eb1 = reinterpret_cast<T*>(ws + align256(static_cast<size_t>(rows * emax) * eb));
  T* tbuf = reinterpret_cast<T*>(ws + 2 * align256(static_cast<size_t>(rows * emax) * eb));
  const int sms = sm_count_dev();
  if (cudaMemsetAsync(lg, 0, sizeof(int64_t) * rows, s) != cudaSuccess) return TT_ERR_CUDA;
  // first mode from the basis environments
  {
    const int ry = y->ranks[k0], rx2 = x->ranks[k0 + 1], ry2 = y->ranks[k0 + 1];
    const int64_t n = static_cast<int64_t>(rows) * rx2 * ry2;
    T* dst = k1 == k0 + 1 ? static_cast<T*>(out) : eb0;
    run_first_kernel<T><<<static_cast<int>(std::min<int64_t>(8 * sms, (n + 255) / 256)), 256, 0, s>>>(
        static_cast<const T*>(x->cores[k0]), static_cast<const T*>(y->cores[k0]), ry, x->modes[k0], rx2, ry2, n, dst);
    renorm_rows_kernel<T><<<std::min(rows, 8 * sms), 256, 0, s>>>(dst, static_cast<int64_t>(rx2) * ry2, rows, lg,
                                                                 status);
    count_launch(2);
    if (cudaGetLastError() != cudaSuccess) return TT_ERR_CUDA;
  }
  if (k1 == k0 + 1) return TT_OK;
  std::lock_guard<std::mutex> lock(g_blas_mu);
  cublasHandle_t h = blas_handle(s);
  if (h == nullptr) return TT_ERR_CUDA;
  T* cur = eb0;
  T* nxt = eb1;
  for (int k = k0 + 1; k < k1; ++k) {
    const int rx = x->ranks[k], ry = y->ranks[k], I = x->modes[k], rx2 = x->ranks[k + 1], ry2 = y->ranks[k + 1];
    T* dst = k + 1 == k1 ? static_cast<T*>(out) : nxt;
    const int64_t per = static_cast<int64_t>(rx) * I * ry2;
    const int Q = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(rows, kGemmChunkElems / per)));
    for (int q0 = 0; q0 < rows; q0 += Q) {
      const int nq = std::min(Q, rows - q0);
      if (gemm_rm(h, dtype, nq * rx, I * ry2, ry, cur + static_cast<int64_t>(q0) * rx * ry, y->cores[k], tbuf) !=
          CUBLAS_STATUS_SUCCESS)
        return TT_ERR_CUDA;
      if (gemm_at_b_batched(h, dtype, rx2, ry2, rx * I, x->cores[k], tbuf, dst + static_cast<int64_t>(q0) * rx2 * ry2,
                            nq) != CUBLAS_STATUS_SUCCESS)
        return TT_ERR_CUDA;
      count_launch(2);
    }
    renorm_rows_kernel<T><<<std::min(rows, 8 * sms), 256, 0, s>>>(dst, static_cast<int64_t>(rx2) * ry2, rows, lg,
                                                                 status);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return TT_ERR_CUDA;
    T* sw = cur;
    cur = nxt;
    nxt = sw;
  }
  return TT_OK;
}

// log2[1 .. n-1] = log2[0]: the right environment has one scale for all rows.
__global__ void broadcast_log2_kernel(int64_t* log2, int n) {
  for (int i = 1 + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) log2[i] = log2[0];
}

static int factored_plan(const tt_desc* x, const tt_desc* y, const uint8_t* mask, tt_factored* f) {
  int rc = check_pair(x, y, mask);
  if (rc != TT_OK) return rc;
  if (mask == nullptr || f == nullptr) return TT_ERR_ARG;
  if (x->dtype == TT_BF16) return TT_ERR_UNSUPPORTED;
  const int n = x->order;
  memset(f, 0, sizeof(*f));
  int m = 0;
  for (int k = 0; k < n; ++k)
    if (!mask[k]) f->free_pos[m++] = k;
  if (m == 0) return TT_ERR_ARG;  // every mode contracted: tt_contract_full
  f->n_free = m;
  int rmax = 1;
  for (int k = 0; k <= n; ++k) rmax = std::max({rmax, x->ranks[k], y->ranks[k]});
  if (rmax > rank_cap(x->dtype)) return TT_ERR_TOO_LARGE;
  const size_t eb = static_cast<size_t>(elem_bytes(x->dtype));
  auto pr = [&](int k) { return static_cast<int64_t>(x->ranks[k]) * y->ranks[k]; };
  size_t off = 0;
  for (int t = 0; t <= m; ++t) {
    const int k0 = t == 0 ? 0 : f->free_pos[t - 1] + 1;  // the run's modes k0 .. k1-1
    const int k1 = t == m ? n : f->free_pos[t];
    if (k1 <= k0) continue;  // identity
    const int64_t rows = t == 0 ? 1 : pr(k0);
    const int64_t cols = t == m ? 1 : pr(k1);
    if (rows * cols > kMergedCoreCap) return TT_ERR_TOO_LARGE;
    f->rows[t] = static_cast<int32_t>(rows);
    f->cols[t] = static_cast<int32_t>(cols);
    f->off_t[t] = off;
    off += align256(static_cast<size_t>(rows * cols) * eb);
    f->off_log2[t] = off;
    off += align256(static_cast<size_t>(rows + 1) * sizeof(int64_t));  // + one scratch slot
    if (t > 0 && t < m && rows >= kGemmRunRows) f->ws_bytes = std::max(f->ws_bytes, gemm_run_ws(x, y, k0, k1, rows));
  }
  f->bytes = std::max<size_t>(off, 256);
  return TT_OK;
}

}  // namespace ttc

using namespace ttc;

extern "C" int tt_factored_shape(const tt_desc* x, const tt_desc* y, const uint8_t* mask, tt_factored* f) {
  return factored_plan(x, y, mask, f);
}

extern "C" int tt_contract_factored(const tt_desc* x, const tt_desc* y, const uint8_t* mask, const tt_factored* f,
                                    void* out_dev, int32_t* status_dev, void* ws, size_t ws_bytes, tt_stream stream) {
  if (f == nullptr || out_dev == nullptr || status_dev == nullptr) return TT_ERR_ARG;
  tt_factored g;
  int rc = factored_plan(x, y, mask, &g);
  if (rc != TT_OK) return rc;
  // the caller's shape must be this contraction's (not one for other operands or another S)
  bool same = g.n_free == f->n_free && g.bytes == f->bytes && g.ws_bytes == f->ws_bytes;
  for (int t = 0; same && t < g.n_free; ++t) same = g.free_pos[t] == f->free_pos[t];
  for (int t = 0; same && t <= g.n_free; ++t)
    same = g.rows[t] == f->rows[t] && g.cols[t] == f->cols[t] && g.off_t[t] == f->off_t[t] &&
           g.off_log2[t] == f->off_log2[t];
  if (!same) return TT_ERR_SHAPE;
  if (g.ws_bytes > 0 && (ws == nullptr || ws_bytes < g.ws_bytes)) return TT_ERR_WS;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* out = static_cast<char*>(out_dev);
  const int n = x->order, m = g.n_free;
  const int bits = x->dtype == TT_F64 ? kRenormBitsF64 : kRenormBitsF32;
  for (int t = 0; t <= m && rc == TT_OK; ++t) {
    if (g.rows[t] == 0) continue;
    const int k0 = t == 0 ? 0 : g.free_pos[t - 1] + 1;
    const int k1 = t == m ? n : g.free_pos[t];
    void* tm = out + g.off_t[t];
    int64_t* lg = reinterpret_cast<int64_t*>(out + g.off_log2[t]);
    if (t == 0 || t == m) {
      // an environment: one sweep from the end of the train
      SweepParams p;
      memset(&p, 0, sizeof(p));
      if (t == 0) fill_left(p, x, y, k0, k1);
      else fill_right(p, x, y, k0, k1);
      p.rx0 = 1;
      p.ry0 = 1;
      p.renorm_bits = bits;
      p.e_out = tm;
      p.e_out_log2 = lg;
      p.status = status_dev;
      rc = launch_sweep(p, x->dtype, s);
      if (rc == TT_OK && g.rows[t] > 1) {
        broadcast_log2_kernel<<<std::min(64, (g.rows[t] + 255) / 256), 256, 0, s>>>(lg, g.rows[t]);
        count_launch();
        if (cudaGetLastError() != cudaSuccess) rc = TT_ERR_CUDA;
      }
    } else if (g.rows[t] >= kGemmRunRows) {
      rc = x->dtype == TT_F64 ? gemm_run<double>(x, y, k0, k1, g.rows[t], tm, lg, static_cast<char*>(ws), status_dev, s)
                              : gemm_run<float>(x, y, k0, k1, g.rows[t], tm, lg, static_cast<char*>(ws), status_dev, s);
    } else {
      // an interior run: its transfer matrix, a scale per row; the slot after
      // the row scales takes the largest (the kernel's running maximum)
      if (cudaMemsetAsync(lg + g.rows[t], 0xC0, sizeof(int64_t), s) != cudaSuccess) return TT_ERR_CUDA;
      TransferParams tp;
      memset(&tp, 0, sizeof(tp));
      SweepParams sp;
      memset(&sp, 0, sizeof(sp));
      fill_left(sp, x, y, k0, k1);
      tp.n_steps = sp.n_steps;
      memcpy(tp.step, sp.step, sizeof(tp.step));
      tp.m = tm;
      tp.mexp = lg;
      tp.emax = lg + g.rows[t];
      tp.status = status_dev;
      if (launch_transfer(tp, x->dtype, s) != cudaSuccess) rc = TT_ERR_CUDA;
    }
  }
  return rc;
}
