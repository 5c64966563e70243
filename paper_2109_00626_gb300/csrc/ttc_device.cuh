// Device helpers shared by the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace ttc {

// Load N consecutive elements (16-byte aligned when N * sizeof(T) >= 16).
template <typename T, int N>
__device__ __forceinline__ void ld_vec(T (&r)[N], const T* __restrict__ p) {
  if constexpr (std::is_same<T, float>::value && N % 4 == 0) {
#pragma unroll
    for (int j = 0; j < N; j += 4) {
      const float4 v = *reinterpret_cast<const float4*>(p + j);
      r[j] = v.x;
      r[j + 1] = v.y;
      r[j + 2] = v.z;
      r[j + 3] = v.w;
    }
  } else if constexpr (std::is_same<T, float>::value && N % 2 == 0) {
#pragma unroll
    for (int j = 0; j < N; j += 2) {
      const float2 v = *reinterpret_cast<const float2*>(p + j);
      r[j] = v.x;
      r[j + 1] = v.y;
    }
  } else if constexpr (std::is_same<T, double>::value && N % 2 == 0) {
#pragma unroll
    for (int j = 0; j < N; j += 2) {
      const double2 v = *reinterpret_cast<const double2*>(p + j);
      r[j] = v.x;
      r[j + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < N; ++j) r[j] = p[j];
  }
}

template <typename T>
__device__ __forceinline__ T ldg(const T* p) {
  return __ldg(p);
}

// Ampere-style asynchronous global -> shared copies (any 4/8-byte aligned
// element, or 16-byte chunks); completion through commit/wait groups.
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem) {
  if constexpr (sizeof(T) == 8) cp_async8(smem, gmem);
  else cp_async4(smem, gmem);
}

// n / d for 0 <= n < 2^16, 1 <= d < 2^16 without the integer divide: the
// float product n * rcp(d) is within n * 2^-23 of n / d, which is below the
// 1 / d gap to the next integer whenever n / d is not one; an exact quotient
// that rounds just below is fixed by the single correction step.
__device__ __forceinline__ int udiv16(int n, int d) {
  int q = __float2int_rz(__int2float_rn(n) * __frcp_rn(__int2float_rn(d)));
  q += (q + 1) * d <= n ? 1 : 0;
  return q;
}

__device__ __forceinline__ void set_status(int32_t* status, int bits) {
  if (status != nullptr && bits != 0) atomicOr(status, bits);
}

template <typename T>
__device__ __forceinline__ bool finite_val(T v) {
  return isfinite(v);
}

// Exact multiplication by 2^e for |e| well inside the exponent range of T.
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }
__device__ __forceinline__ double pow2d(int e) {
  return __longlong_as_double(static_cast<long long>(1023 + e) << 52);
}
template <typename T>
__device__ __forceinline__ T pow2(int e);
template <>
__device__ __forceinline__ float pow2<float>(int e) {
  return pow2f(e);
}
template <>
__device__ __forceinline__ double pow2<double>(int e) {
  return pow2d(e);
}

// x * 2^e, exact for |e| up to about twice the exponent range of T (two steps).
template <typename T>
__device__ __forceinline__ T mul_pow2(T x, int e) {
  const int e1 = e / 2;
  return x * pow2<T>(e1) * pow2<T>(e - e1);
}

// s * 2^e saturated to +-Inf / signed zero outside the range of T.
template <typename T>
__device__ __forceinline__ T scale_pow2_sat(T s, int64_t e) {
  constexpr int64_t lim = sizeof(T) == 4 ? 250 : 2000;
  if (s == T(0) || !isfinite(s)) return s;
  if (e > lim) return s > T(0) ? T(INFINITY) : T(-INFINITY);
  if (e < -lim) return s * T(0);
  return mul_pow2<T>(s, static_cast<int>(e));
}

// Binary exponent e with 2^(e-1) <= |v| < 2^e of a finite non-zero v, read
// from its IEEE-754 bits (no float64 arithmetic, which runs at a small
// fraction of the float32 rate here); subnormals are given the smallest
// normal exponent, which only changes the power of two a rescale picks.
__device__ __forceinline__ int exp2_bits(float v) { return max((__float_as_int(v) >> 23) & 0xff, 1) - 126; }
__device__ __forceinline__ int exp2_bits(double v) {
  return max(static_cast<int>((__double_as_longlong(v) >> 52) & 0x7ff), 1) - 1022;
}

// Binary exponent e with 2^(e-1) <= |v| < 2^e (v finite, non-zero).
__device__ __forceinline__ int exp2_of(double v) {
  int e;
  frexp(v, &e);
  return e;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_or(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Elements [0, n) of the sum of `parts` consecutive arrays of n elements
// (added in order: part 0, then 1, ...), each handed to f(idx, value) by the
// block's NT threads.  A thread keeps 16 elements' loads of a part in flight,
// so the sum costs about `parts` memory latencies, not one per element and part.
template <typename T, int NT, typename F>
__device__ __forceinline__ void sum_parts(const T* __restrict__ src, int n, int parts, F f) {
  constexpr int B = 16;
  for (int base = threadIdx.x; base < n; base += NT * B) {
    T acc[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int idx = base + u * NT;
      acc[u] = idx < n ? src[idx] : T(0);
    }
    for (int g = 1; g < parts; ++g) {
      const T* sg = src + static_cast<int64_t>(g) * n;
#pragma unroll
      for (int u = 0; u < B; ++u) {
        const int idx = base + u * NT;
        if (idx < n) acc[u] += sg[idx];
      }
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int idx = base + u * NT;
      if (idx < n) f(idx, acc[u]);
    }
  }
}

}  // namespace ttc
