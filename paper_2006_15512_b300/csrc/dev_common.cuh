// Device helpers shared by the CUDA translation units of the library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace wmc {
namespace dev {

constexpr int kThreads = 256;
constexpr int kMaxQ = 1024;
constexpr unsigned long long kNoMin = ~0ull;

// --------------------------------------------------------------- helpers

__device__ __forceinline__ int pow2_exp_of(unsigned long long bits, float) {
  if (bits == 0) return 0;
  int e = (int)((bits >> 23) & 0xff) - 127;
  e = e < -126 ? -126 : e;
  return e > 126 ? 126 : e;
}
__device__ __forceinline__ int pow2_exp_of(unsigned long long bits, double) {
  if (bits == 0) return 0;
  int e = (int)((bits >> 52) & 0x7ff) - 1023;
  e = e < -1022 ? -1022 : e;
  return e > 1022 ? 1022 : e;
}
__device__ __forceinline__ float pow2_scale(int e, float) { return __int_as_float((127 - e) << 23); }
__device__ __forceinline__ double pow2_scale(int e, double) {
  return __longlong_as_double((long long)(1023 - e) << 52);
}
__device__ __forceinline__ unsigned long long abs_bits(float x) {
  return (unsigned long long)(__float_as_uint(x) & 0x7fffffffu);
}
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ bool below_normal(float x) { return fabsf(x) < 1.17549435e-38f; }
__device__ __forceinline__ bool below_normal(double x) { return fabs(x) < 2.2250738585072014e-308; }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }

// insert a zero bit at position p
__device__ __forceinline__ uint32_t insert0(uint32_t x, int p) {
  uint32_t lo = x & ((1u << p) - 1u);
  return ((x >> p) << (p + 1)) | lo;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <typename T> __device__ __forceinline__ T from_bits(unsigned long long b);
template <> __device__ __forceinline__ float from_bits<float>(unsigned long long b) {
  return __uint_as_float((uint32_t)b);
}
template <> __device__ __forceinline__ double from_bits<double>(unsigned long long b) {
  return __longlong_as_double((long long)b);
}

}  // namespace dev
}  // namespace wmc
