// Host side of the batched contraction: plan (validation, LPT order, tile
// choice), packing of the device table, launch, and the tile autotuner.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <numeric>
#include <vector>

#include "host_plan.h"

struct tt_plan {
  int n_pairs = 0;
  int dtype = TT_F32;
  std::vector<ttc::SweepParams> table;
  std::vector<int32_t> order;
  std::vector<int32_t> tile;
  std::vector<double> cost;
  std::vector<ttc::CopyJob> jobs;
  size_t off_order = 0, off_tile = 0, off_jobs = 0, packed_bytes = 0;
  size_t ws_bytes = 256;  // device workspace the launch needs (the work-queue counter)
};

namespace ttc {

// Autotuned tile configuration (plan_engine_steps) per (dtype, rank bucket,
// mode bucket); -1 = not tuned.
constexpr int kRankBuckets = 4, kModeBuckets = 5;
struct TuneTable {
  int cfg[2][kRankBuckets][kModeBuckets];
  bool loaded = false;
  char path[512] = {0};  // the cache file it was read from ("" = none)
};

static int rank_bucket(int r) { return r <= 16 ? 0 : (r <= 32 ? 1 : (r <= 64 ? 2 : 3)); }
static int mode_bucket(int I) { return I <= 4 ? 0 : (I <= 8 ? 1 : (I <= 16 ? 2 : (I <= 32 ? 3 : 4))); }
static const int kRankOf[kRankBuckets] = {16, 32, 64, 128};  // representative sizes the tuner times
static const int kModeOf[kModeBuckets] = {4, 8, 16, 32, 48};
constexpr size_t kTuneBytes = size_t(2) << 30;  // distinct synthetic cores per bucket (well above L2)
constexpr float kTuneMargin = 0.97f;            // a configuration must beat the default by 3 %

// Seeded values for the tuner's synthetic cores: SplitMix64 (Steele, Lea and
// Flood 2014) of the element index, mapped to [-1, 1) and scaled.
template <typename T>
__global__ void tune_fill_kernel(T* dst, size_t n, uint64_t seed, double sc) {
  for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    uint64_t z = seed + (e + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    dst[e] = static_cast<T>((static_cast<double>(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0) * sc);
  }
}

// Read again whenever TTC_AUTOTUNE_CACHE names another file (or after tt_autotune).
static TuneTable& tune_table() {
  static TuneTable t;
  const char* path = getenv("TTC_AUTOTUNE_CACHE");
  if (t.loaded && strncmp(t.path, path != nullptr ? path : "", sizeof(t.path) - 1) != 0) t.loaded = false;
  if (!t.loaded) {
    for (auto& a : t.cfg)
      for (auto& b : a)
        for (int& c : b) c = -1;
    snprintf(t.path, sizeof(t.path), "%s", path != nullptr ? path : "");
    if (path != nullptr) {
      FILE* f = fopen(path, "r");
      if (f != nullptr) {
        int d, rb, ib, cfg;
        while (fscanf(f, "%d %d %d %d", &d, &rb, &ib, &cfg) == 4)
          if (d >= 0 && d < 2 && rb >= 0 && rb < kRankBuckets && ib >= 0 && ib < kModeBuckets && cfg >= 0 &&
              cfg < kTileConfigs)
            t.cfg[d][rb][ib] = cfg;
        fclose(f);
      }
    }
    t.loaded = true;
  }
  return t;
}

// Tile configuration of a pair's engine plan: the autotuned value of its
// (rank, mode) bucket, else the default (full panel budget, no replica cap).
static int choose_config(const SweepParams& p, int dtype) {
  const int d = dtype == TT_F64 ? 1 : 0;
  const int tuned = tune_table().cfg[d][rank_bucket(sweep_max_rank(p))][mode_bucket(sweep_max_mode(p))];
  return tuned >= 0 ? tuned : kDefaultTileConfig;
}

}  // namespace ttc

using namespace ttc;

extern "C" {

int tt_batch_plan(const tt_batch* b, tt_plan** plan_out, size_t* packed_bytes, size_t* ws_bytes) {
  if (b == nullptr || plan_out == nullptr || packed_bytes == nullptr || ws_bytes == nullptr) return TT_ERR_ARG;
  if (b->n_pairs < 1 || b->x == nullptr || b->y == nullptr) return TT_ERR_ARG;
  if (b->prec != TT_P_NATIVE) return TT_ERR_UNSUPPORTED;
  const int n = b->n_pairs;
  tt_plan* plan = new tt_plan();
  plan->n_pairs = n;
  plan->dtype = b->x[0].dtype;
  plan->table.resize(n);
  plan->tile.resize(n);
  plan->cost.resize(n);
  for (int i = 0; i < n; ++i) {
    const tt_desc* x = &b->x[i];
    const tt_desc* y = &b->y[i];
    const uint8_t* mask = b->mask != nullptr ? b->mask[i] : nullptr;
    int rc = check_pair(x, y, mask);
    if (rc == TT_OK && x->dtype != plan->dtype) rc = TT_ERR_DTYPE;
    if (rc == TT_OK && x->dtype == TT_BF16) rc = TT_ERR_UNSUPPORTED;
    if (rc == TT_OK) {
      if (mask == nullptr) {
        build_full(x, y, nullptr, nullptr, nullptr, &plan->table[i]);
      } else {
        ChainPlan cp;
        rc = chain_plan(x, y, mask, &cp);
        if (rc == TT_OK && b->z == nullptr) rc = TT_ERR_ARG;
        if (rc == TT_OK) rc = check_chain_output(x, cp, &b->z[i]);
        if (rc == TT_OK) rc = build_partial(x, y, cp, &b->z[i], nullptr, nullptr, &plan->table[i]);
      }
    }
    if (rc == TT_OK && sweep_max_rank(plan->table[i]) > rank_cap(plan->dtype)) rc = TT_ERR_TOO_LARGE;
    if (rc == TT_OK && plan->table[i].emit.enabled) {
      const EmitParams& em = plan->table[i].emit;
      for (int t = 0; t < em.n_copies; ++t)
        if (em.copy[t].r1 > kCopyJobBytes / elem_bytes(plan->dtype)) rc = TT_ERR_TOO_LARGE;
    }
    if (rc != TT_OK) {
      delete plan;
      return rc;
    }
    plan->tile[i] = choose_config(plan->table[i], plan->dtype);
    plan_engine_steps(plan->table[i], plan->dtype, plan->tile[i]);
    plan->cost[i] = sweep_flops(plan->table[i]);
  }
  // longest processing time first
  plan->order.resize(n);
  std::iota(plan->order.begin(), plan->order.end(), 0);
  std::stable_sort(plan->order.begin(), plan->order.end(),
                   [&](int a, int c) { return plan->cost[a] > plan->cost[c]; });
  // free-core copies cut into jobs of at most kCopyJobBytes (copy_cut)
  const int eb = elem_bytes(plan->dtype);
  for (int i = 0; i < n; ++i) {
    const EmitParams& em = plan->table[plan->order[i]].emit;
    if (!em.enabled) continue;
    for (int t = 0; t < em.n_copies; ++t) {
      const CopyTask& tk = em.copy[t];
      const CopyCut cut = copy_cut(tk.r0, tk.I, tk.r1, eb);
      for (int j = 0; j < cut.n_i * cut.n_a; ++j) plan->jobs.push_back(copy_job_at(tk, cut, j));
    }
  }
  plan->off_order = align256(sizeof(SweepParams) * n);
  plan->off_tile = plan->off_order + align256(sizeof(int32_t) * n);
  plan->off_jobs = plan->off_tile + align256(sizeof(int32_t) * n);
  plan->packed_bytes = plan->off_jobs + align256(sizeof(CopyJob) * std::max<size_t>(1, plan->jobs.size()));
  *packed_bytes = plan->packed_bytes;
  *ws_bytes = 256;  // work-queue counter
  *plan_out = plan;
  return TT_OK;
}

int tt_batch_pack(const tt_plan* plan, void* packed_host, size_t packed_bytes) {
  if (plan == nullptr || packed_host == nullptr || packed_bytes < plan->packed_bytes) return TT_ERR_ARG;
  char* base = static_cast<char*>(packed_host);
  memset(base, 0, plan->packed_bytes);
  memcpy(base, plan->table.data(), sizeof(SweepParams) * plan->n_pairs);
  memcpy(base + plan->off_order, plan->order.data(), sizeof(int32_t) * plan->n_pairs);
  memcpy(base + plan->off_tile, plan->tile.data(), sizeof(int32_t) * plan->n_pairs);
  if (!plan->jobs.empty()) memcpy(base + plan->off_jobs, plan->jobs.data(), sizeof(CopyJob) * plan->jobs.size());
  return TT_OK;
}

int tt_contract_batched(const tt_plan* plan, const void* packed_dev, double* out_dev, int64_t* out_log2_dev,
                        int32_t* status_dev, void* ws, size_t ws_bytes, tt_stream stream) {
  if (plan == nullptr || packed_dev == nullptr || out_dev == nullptr) return TT_ERR_ARG;
  if (ws == nullptr || ws_bytes < 256) return TT_ERR_WS;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const char* base = static_cast<const char*>(packed_dev);
  if (cudaMemsetAsync(ws, 0, 2 * sizeof(int), s) != cudaSuccess) return TT_ERR_CUDA;
  if (cudaMemsetAsync(out_dev, 0, sizeof(double) * plan->n_pairs, s) != cudaSuccess) return TT_ERR_CUDA;
  const cudaError_t err =
      launch_batched(base, reinterpret_cast<const int32_t*>(base + plan->off_order),
                     reinterpret_cast<const int32_t*>(base + plan->off_tile), plan->n_pairs,
                     reinterpret_cast<const CopyJob*>(base + plan->off_jobs), static_cast<int>(plan->jobs.size()),
                     static_cast<int*>(ws), out_dev, out_log2_dev, status_dev, plan->dtype, 0, s);
  return err == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

int tt_plan_info(const tt_plan* plan, int32_t p, int32_t* n_pairs, int32_t* tile_config) {
  if (plan == nullptr) return TT_ERR_ARG;
  if (n_pairs != nullptr) *n_pairs = plan->n_pairs;
  if (p < 0 || p >= plan->n_pairs) return TT_ERR_ARG;
  if (tile_config != nullptr) *tile_config = plan->tile[p];
  return TT_OK;
}

void tt_plan_free(tt_plan* plan) { delete plan; }

int tt_autotune(int dtype, const char* cache_path) {
  if (cache_path == nullptr) return TT_ERR_ARG;
  if (dtype != TT_F32 && dtype != TT_F64) return TT_ERR_DTYPE;
  const int d = dtype == TT_F64 ? 1 : 0;
  const int eb = dtype == TT_F64 ? 8 : 4;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int order = 6;
  const int npairs = 2 * sms;
  FILE* f = fopen(cache_path, "w");
  if (f == nullptr) return TT_ERR_ARG;
  int rc = TT_OK;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  void* cores = nullptr;
  void* dev_table = nullptr;
  int* counter = nullptr;
  double* out = nullptr;
  // every buffer is released here, on success and on every error path
  auto release = [&]() {
    if (cores != nullptr) cudaFree(cores);
    if (dev_table != nullptr) cudaFree(dev_table);
    if (counter != nullptr) cudaFree(counter);
    if (out != nullptr) cudaFree(out);
    cores = dev_table = nullptr;
    counter = nullptr;
    out = nullptr;
  };
  if (cudaStreamCreate(&s) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    rc = TT_ERR_CUDA;
  }
  for (int rb = 0; rb < kRankBuckets && rc == TT_OK; ++rb) {
    if (dtype == TT_F64 && kRankOf[rb] > 64) break;  // float64 ranks stop at 64
    for (int ib = 0; ib < kModeBuckets && rc == TT_OK; ++ib) {
      const int R = kRankOf[rb];
      const int I = kModeOf[ib];
      // Synthetic full contractions of order 6 at the bucket's rank and mode
      // size, one per CTA slot.  Pairs own distinct cores (up to kTuneBytes
      // of them, then reused in turn) so that, as in a real batch, the cores
      // stream from memory rather than from L2.
      const size_t core_bytes = static_cast<size_t>(R) * I * R * eb;
      const size_t pair_bytes = 2 * order * core_bytes;
      const int ndist = static_cast<int>(std::max<size_t>(1, std::min<size_t>(npairs, kTuneBytes / pair_bytes)));
      if (cudaMalloc(&cores, pair_bytes * ndist) != cudaSuccess) {
        rc = TT_ERR_CUDA;
        release();
        break;
      }
      const double sc = 1.0 / std::sqrt(static_cast<double>(I) * R);
      const size_t nel = pair_bytes * ndist / eb;
      const uint64_t seed = 0x2109006260ull + 977ull * (rb * kModeBuckets + ib);
      if (eb == 8) tune_fill_kernel<double><<<4 * sms, 256, 0, s>>>(static_cast<double*>(cores), nel, seed, sc);
      else tune_fill_kernel<float><<<4 * sms, 256, 0, s>>>(static_cast<float*>(cores), nel, seed, sc);
      std::vector<SweepParams> base(ndist);
      for (int k = 0; k < ndist; ++k) {
        int32_t modes[order], ranks[order + 1];
        void* px[order];
        void* py[order];
        char* pb = static_cast<char*>(cores) + k * pair_bytes;
        for (int c = 0; c < order; ++c) {
          modes[c] = I;
          ranks[c] = c == 0 ? 1 : R;
          px[c] = pb + c * core_bytes;
          py[c] = pb + (order + c) * core_bytes;
        }
        ranks[order] = 1;
        tt_desc x{order, modes, ranks, px, dtype};
        tt_desc y{order, modes, ranks, py, dtype};
        build_full(&x, &y, nullptr, nullptr, nullptr, &base[k]);
      }
      std::vector<SweepParams> tab(npairs);
      std::vector<int32_t> ord(npairs), tl(npairs);
      std::iota(ord.begin(), ord.end(), 0);
      if (cudaMalloc(&dev_table, sizeof(SweepParams) * npairs + 8 * npairs + 256) != cudaSuccess ||
          cudaMalloc(&counter, 256) != cudaSuccess || cudaMalloc(&out, sizeof(double) * npairs) != cudaSuccess) {
        rc = TT_ERR_CUDA;
        release();
        break;
      }
      char* tb = static_cast<char*>(dev_table);
      cudaMemcpyAsync(tb + sizeof(SweepParams) * npairs, ord.data(), 4 * npairs, cudaMemcpyHostToDevice, s);
      float ms[kTileConfigs];
      for (int cfg = 0; cfg < kTileConfigs && rc == TT_OK; ++cfg) {
        for (int k = 0; k < npairs; ++k) {
          tab[k] = base[k % ndist];
          plan_engine_steps(tab[k], dtype, cfg);
        }
        std::fill(tl.begin(), tl.end(), cfg);
        cudaMemcpyAsync(tb, tab.data(), sizeof(SweepParams) * npairs, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(tb + sizeof(SweepParams) * npairs + 4 * npairs, tl.data(), 4 * npairs,
                        cudaMemcpyHostToDevice, s);
        float times[4];
        for (int rep = 0; rep < 4; ++rep) {
          cudaMemsetAsync(counter, 0, 8, s);
          cudaEventRecord(e0, s);
          launch_batched(tb, reinterpret_cast<int32_t*>(tb + sizeof(SweepParams) * npairs),
                         reinterpret_cast<int32_t*>(tb + sizeof(SweepParams) * npairs + 4 * npairs), npairs, nullptr,
                         0, counter, out, nullptr, nullptr, dtype, 0, s);
          cudaEventRecord(e1, s);
          cudaEventSynchronize(e1);
          cudaEventElapsedTime(&times[rep], e0, e1);
        }
        if (cudaGetLastError() != cudaSuccess) {
          rc = TT_ERR_CUDA;
          break;
        }
        // median of the three launches after the first
        std::sort(times + 1, times + 4);
        ms[cfg] = times[2];
      }
      release();
      if (rc != TT_OK) break;
      // another configuration replaces the default only when it is clearly
      // faster (timing noise must not move a bucket off a good default)
      int best = kDefaultTileConfig;
      for (int cfg = 0; cfg < kTileConfigs; ++cfg)
        if (ms[cfg] < kTuneMargin * ms[kDefaultTileConfig] && ms[cfg] < ms[best]) best = cfg;
      // a bucket is written only when every configuration of it was timed without error
      fprintf(f, "%d %d %d %d\n", d, rb, ib, best);
    }
  }
  release();
  fclose(f);
  if (e0 != nullptr) cudaEventDestroy(e0);
  if (e1 != nullptr) cudaEventDestroy(e1);
  if (s != nullptr) cudaStreamDestroy(s);
  tune_table().loaded = false;  // pick the new cache up on the next plan
  return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched contraction without a caller-provided workspace.
//
// Some callers cannot hand this library a device buffer at the point where
// they contract: a plugin inside a framework that owns every device
// allocation, or a loop that must not allocate once it is running.  For them
// the work-queue counter lives in a fixed array inside the library instead of
// in `ws`.  The array is static device memory: every GPU that loads the library
// holds one copy of kNoAllocScratchBytes bytes until the process exits.
// ---------------------------------------------------------------------------
namespace ttc {

constexpr size_t kNoAllocScratchBytes = TT_NOALLOC_SCRATCH_BYTES;
static_assert(kNoAllocScratchBytes >= 2 * sizeof(int), "the work-queue counter must fit the fixed array");
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
static void* g_noalloc_addr[kMaxDevices];  // device address of g_noalloc_scratch, per device
static std::mutex g_noalloc_mu;

// Device address of the scratch array on the current device.  The host-side
// name g_noalloc_scratch is only a stand-in.  Outside a stream capture the
// address is looked up on every call, with the device current (a new context
// after cudaDeviceReset may place the array elsewhere); a call being captured
// uses the address its device's last uncaptured call found.
static int noalloc_scratch(cudaStream_t s, void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TT_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return TT_ERR_UNSUPPORTED;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return TT_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (cap == cudaStreamCaptureStatusNone || g_noalloc_addr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return TT_ERR_CUDA;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return TT_OK;
}

}  // namespace ttc

extern "C" int tt_contract_batched_noalloc(const tt_plan* plan, const void* packed_dev, double* out_dev,
                                           int64_t* out_log2_dev, int32_t* status_dev, tt_stream stream) {
  if (plan == nullptr || packed_dev == nullptr || out_dev == nullptr) return TT_ERR_ARG;
  if (plan->ws_bytes > TT_NOALLOC_SCRATCH_BYTES) return TT_ERR_WS;  // plan needs more than the fixed array
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  void* scratch = nullptr;
  const int rc = noalloc_scratch(s, &scratch);
  if (rc != TT_OK) return rc;
  const char* base = static_cast<const char*>(packed_dev);
  // the counter must start at zero on every call; the array keeps the last call's contents
  if (cudaMemsetAsync(scratch, 0, 2 * sizeof(int), s) != cudaSuccess) return TT_ERR_CUDA;
  if (cudaMemsetAsync(out_dev, 0, sizeof(double) * plan->n_pairs, s) != cudaSuccess) return TT_ERR_CUDA;
  const cudaError_t err =
      launch_batched(base, reinterpret_cast<const int32_t*>(base + plan->off_order),
                     reinterpret_cast<const int32_t*>(base + plan->off_tile), plan->n_pairs,
                     reinterpret_cast<const CopyJob*>(base + plan->off_jobs), static_cast<int>(plan->jobs.size()),
                     static_cast<int*>(scratch), out_dev, out_log2_dev, status_dev, plan->dtype, 0, s);
  return err == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}
