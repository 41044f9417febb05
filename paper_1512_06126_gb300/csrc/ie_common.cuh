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
