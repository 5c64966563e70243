// Partial contraction over any contracted set, merged (TT-matrix) layout.
//
// With free positions f_0 < ... < f_{m-1}, output core t is the Kronecker pair
//   W_t[(a,b)][i][j][(a',b')] = Gx_{f_t}[a][i][a'] Gy_{f_t}[b][j][b']
// (pair rank index a*R^y + b).  The left environment E_L of the contracted
// modes before f_0 is folded into W_0:
//   W_0[0][i][j][(a',b')] = sum_a Gx[a][i][a'] V[a][j][b'],  V = E_L Gy (per j).
// The contracted run between f_t and f_{t+1} (or after f_{m-1}) acts on the
// right leg of W_t: every row (r, i, j) of W_t, read as an R^x' x R^y'
// environment, is swept through the run with the shared sweep body (one
// persistent kernel over all rows), which leaves R^x_{f_{t+1}} R^y_{f_{t+1}}
// (or 1) entries per row.  The Kronecker expansion is bound by HBM writes.
#include "sweep_body.cuh"

namespace ttc {

// W[(a*ry + b)][i][j][(a2*ry2 + b2)] = gx[a][i][a2] gy[b][j][b2]
template <typename T>
__global__ void __launch_bounds__(256) kron_kernel(const __grid_constant__ KronParams p) {
  const T* gx = static_cast<const T*>(p.gx);
  const T* gy = static_cast<const T*>(p.gy);
  T* w = static_cast<T*>(p.out);
  const int64_t ncol = static_cast<int64_t>(p.rx2) * p.ry2;
  const int64_t n = static_cast<int64_t>(p.rx) * p.ry * p.I * p.J * ncol;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t c = e % ncol;
    int64_t r = e / ncol;
    const int j = static_cast<int>(r % p.J);
    r /= p.J;
    const int i = static_cast<int>(r % p.I);
    r /= p.I;
    const int b = static_cast<int>(r % p.ry), a = static_cast<int>(r / p.ry);
    const int a2 = static_cast<int>(c / p.ry2), b2 = static_cast<int>(c % p.ry2);
    w[e] = gx[(static_cast<int64_t>(a) * p.I + i) * p.rx2 + a2] * gy[(static_cast<int64_t>(b) * p.J + j) * p.ry2 + b2];
  }
}

// V[a][j][b2] = sum_b E_L[a][b] gy[b][j][b2]   (then W_0 from V)
template <typename T>
__global__ void __launch_bounds__(256) kron0_v_kernel(const __grid_constant__ KronParams p) {
  const T* el = static_cast<const T*>(p.el);
  const T* gy = static_cast<const T*>(p.gy);
  T* v = static_cast<T*>(p.tmp);
  const int64_t n = static_cast<int64_t>(p.rx) * p.J * p.ry2;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int b2 = static_cast<int>(e % p.ry2);
    const int64_t r = e / p.ry2;
    const int j = static_cast<int>(r % p.J), a = static_cast<int>(r / p.J);
    T s = T(0);
    for (int b = 0; b < p.ry; ++b) s = fma(el[a * p.ry + b], gy[(static_cast<int64_t>(b) * p.J + j) * p.ry2 + b2], s);
    v[e] = s;
  }
}

// W_0[i][j][(a2*ry2 + b2)] = 2^e * sum_a gx[a][i][a2] V[a][j][b2]
template <typename T>
__global__ void __launch_bounds__(256) kron0_w_kernel(const __grid_constant__ KronParams p) {
  const T* gx = static_cast<const T*>(p.gx);
  const T* v = static_cast<const T*>(p.tmp);
  T* w = static_cast<T*>(p.out);
  const int64_t lg = p.el_log2 != nullptr ? *p.el_log2 : 0;
  const int64_t ncol = static_cast<int64_t>(p.rx2) * p.ry2;
  const int64_t n = static_cast<int64_t>(p.I) * p.J * ncol;
  int bits = 0;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t c = e % ncol;
    const int64_t r = e / ncol;
    const int j = static_cast<int>(r % p.J), i = static_cast<int>(r / p.J);
    const int a2 = static_cast<int>(c / p.ry2), b2 = static_cast<int>(c % p.ry2);
    T s = T(0);
    for (int a = 0; a < p.rx; ++a)
      s = fma(gx[(static_cast<int64_t>(a) * p.I + i) * p.rx2 + a2], v[(static_cast<int64_t>(a) * p.J + j) * p.ry2 + b2], s);
    const T s0 = s;
    s = scale_pow2_sat<T>(s, lg);
    if (isfinite(s0) && !isfinite(s)) bits |= TT_STATUS_OVERFLOW;
    if (!isfinite(s)) bits |= TT_STATUS_NONFINITE;
    w[e] = s;
  }
  if (bits) set_status(p.status, bits);
}

// Every row of a merged core swept through a contracted run (C = 1 per row).
template <typename T, int RM>
__global__ void __launch_bounds__(512, 1) rows_sweep_kernel(const __grid_constant__ SweepParams p, RowIO io) {
  extern __shared__ __align__(16) unsigned char smem[];
  for (int64_t row = blockIdx.x; row < io.n_rows; row += gridDim.x) {
    SweepOut o{nullptr, nullptr, p.status};
    o.e_in = static_cast<const char*>(io.in) + row * io.in_stride_bytes;
    o.e_out = static_cast<char*>(io.out) + row * io.out_stride_bytes;
    o.fold_e_out = 1;
    SweepState<T, RM, false> st;
    if (sweep_body<T, RM, false>(p, o, smem, 1, 0, st)) sweep_tail<T, RM, false>(p, o, smem, 1, 0, st);
    __syncthreads();
  }
}

template <typename T>
static cudaError_t kron_impl(const KronParams& p, int which, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = sms * 8;
  count_launch();
  if (which == 0) kron_kernel<T><<<grid, 256, 0, s>>>(p);
  else if (which == 1) kron0_v_kernel<T><<<grid, 256, 0, s>>>(p);
  else kron0_w_kernel<T><<<grid, 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_kron(const KronParams& p, int which, int dtype, cudaStream_t s) {
  return dtype == TT_F64 ? kron_impl<double>(p, which, s) : kron_impl<float>(p, which, s);
}

template <typename T, int RM>
static cudaError_t rows_impl(const SweepParams& p, const RowIO& io, cudaStream_t s) {
  const size_t smem = SweepCfg<T, RM, false>::SMEM;
  cudaError_t err = cudaFuncSetAttribute(rows_sweep_kernel<T, RM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, rows_sweep_kernel<T, RM>, SweepCfg<T, RM, false>::NT, smem);
  if (err != cudaSuccess) return err;
  int64_t grid = static_cast<int64_t>(sms) * std::max(per, 1);
  grid = std::min<int64_t>(grid, io.n_rows);
  count_launch();
  rows_sweep_kernel<T, RM><<<static_cast<unsigned>(grid), SweepCfg<T, RM, false>::NT, smem, s>>>(p, io);
  return cudaGetLastError();
}

cudaError_t launch_rows_sweep(const SweepParams& p, const RowIO& io, int dtype, int rmax, cudaStream_t s) {
  if (dtype == TT_F64) {
    if (rmax <= 32) return rows_impl<double, 32>(p, io, s);
    return rows_impl<double, 64>(p, io, s);
  }
  if (rmax <= 32) return rows_impl<float, 32>(p, io, s);
  if (rmax <= 64) return rows_impl<float, 64>(p, io, s);
  return rows_impl<float, 128>(p, io, s);
}

}  // namespace ttc
