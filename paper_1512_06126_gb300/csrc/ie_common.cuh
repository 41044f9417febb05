// Common device helpers for the GB300 integral-equation library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

namespace ie {

template <typename T> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };
template <typename T> using C = typename cplx<T>::type;

template <typename T> __host__ __device__ __forceinline__ C<T> mk(T re, T im) { C<T> c; c.x = re; c.y = im; return c; }
template <typename V> __host__ __device__ __forceinline__ V cadd(V a, V b) { a.x += b.x; a.y += b.y; return a; }
template <typename V> __host__ __device__ __forceinline__ V csub(V a, V b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename V> __host__ __device__ __forceinline__ V cmul(V a, V b) {
  V c; c.x = a.x * b.x - a.y * b.y; c.y = a.x * b.y + a.y * b.x; return c;
}
// acc += a * b
template <typename V> __host__ __device__ __forceinline__ void cfma(V &acc, V a, V b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfma(float2 &acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(a.y, b.x, acc.y);
}
template <typename V> __host__ __device__ __forceinline__ V cconj(V a) { a.y = -a.y; return a; }
template <typename V, typename S> __host__ __device__ __forceinline__ V cscale(V a, S s) { a.x *= s; a.y *= s; return a; }
template <typename V> __host__ __device__ __forceinline__ V cneg(V a) { a.x = -a.x; a.y = -a.y; return a; }

// FP64 <-> FP32 conversions from the bits with integer operations (GB300 runs FP64
// instructions, conversions included, at a small fraction of the FP32 rate).
// d2f_bits: rounded to nearest (ties away from zero) within FP32's normal range, zero
// below it, Inf above it, NaN kept.  f2d_bits: exact for normal and zero FP32 values
// (FP32 subnormals become zero), Inf and NaN kept.
__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const uint32_t sgn = (uint32_t)(u >> 32) & 0x80000000u;
  const unsigned long long a = (u & 0x7FFFFFFFFFFFFFFFull) + (1ull << 28);  // half an FP32 ulp
  const uint32_t e = (uint32_t)(a >> 52);                                   // after the carry
  const uint32_t m = (uint32_t)(a >> 29) & 0x7FFFFFu;
  const bool nan = (u & 0x7FFFFFFFFFFFFFFFull) > 0x7FF0000000000000ull;
  uint32_t f = sgn | ((e - 896u) << 23) | m;
  f = e < 897u ? sgn : f;
  f = e > 1150u ? (sgn | (nan ? 0x7FC00000u : 0x7F800000u)) : f;
  return __uint_as_float(f);
}
__device__ __forceinline__ double f2d_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu;
  const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long man = (unsigned long long)(u & 0x7FFFFFu) << 29;
  const unsigned long long bits =
      e == 0u ? sgn : (e == 0xFFu ? sgn | 0x7FF0000000000000ull | man : sgn | ((unsigned long long)(e + 896u) << 52) | man);
  return __longlong_as_double((long long)bits);
}
template <typename T> __device__ __forceinline__ C<T> to_prec(float2 v);
template <> __device__ __forceinline__ float2 to_prec<float>(float2 v) { return v; }
template <> __device__ __forceinline__ double2 to_prec<double>(float2 v) {
  return make_double2(f2d_bits(v.x), f2d_bits(v.y));
}
__device__ __forceinline__ float2 to_f32(float2 v) { return v; }
__device__ __forceinline__ float2 to_f32(double2 v) { return make_float2(d2f_bits(v.x), d2f_bits(v.y)); }

// Count of kernels launched by the library (all launchers increment it).
void count_launches(long long n);
long long launches();

// Maximum number of radix stages in an FFT plan.
constexpr int kMaxStages = 20;

// A mixed-radix Stockham plan for one transform length L.
struct FftPlan {
  int L;
  int n_stages;
  int radix[kMaxStages];
};

}  // namespace ie
