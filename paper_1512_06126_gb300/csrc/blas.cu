// Krylov kernels for restarted GMRES (the iterative method of Sect. 3.3 (ii)):
// classical Gram-Schmidt with selective reorthogonalisation, norms, scaling and the
// basis update.  All right-hand sides advance in lockstep; each has its own Krylov
// space.  Vectors are c128 (the FP64 solver) or c64 (the inner solver of the mixed
// precision refinement); the Hessenberg entries, norms and every cross-thread sum are
// FP64.  c64 kernels form short per-thread sums (at most 64 terms) in FP32 and
// combine them in FP64.
//
// Layout: a basis vector block is V[i][r][n] (basis index i, right-hand side r,
// element n), so basis vector i of right-hand side r starts at V + (i*R + r)*n.
#include "blas.cuh"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace ie {
namespace {

constexpr int kT = 256;
constexpr int kEPT = 4;            // elements per thread in the reductions
constexpr int kChunk = kT * kEPT;  // elements per block

// Sum over the block; the total is valid in thread 0 only.
__device__ __forceinline__ double2 block_reduce(double2 v, double2 *sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double2 r = make_double2(0.0, 0.0);
  if (wid == 0) {
    r = lane < (kT / 32) ? sh[lane] : make_double2(0.0, 0.0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      r.x += __shfl_down_sync(0xffffffffu, r.x, o);
      r.y += __shfl_down_sync(0xffffffffu, r.y, o);
    }
  }
  __syncthreads();
  return r;
}

__device__ __forceinline__ float mad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double mad(double a, double b, double c) { return fma(a, b, c); }
template <typename T> __device__ __forceinline__ C<T> to_c(double2 v) { return mk<T>((T)v.x, (T)v.y); }

// w[r] -= sum_{i<k1} h[r * ldh + i] * V_i[r]   (sign = -1), or x[r] += ... (sign = +1)
template <typename T>
__global__ void maxpy_kernel(const C<T> *__restrict__ V, const double2 *__restrict__ h, C<T> *__restrict__ w, int k1,
                             int R, long long n, int ldh, double sign) {
  __shared__ C<T> hs[64];
  const int r = blockIdx.y;
  if (threadIdx.x < k1) hs[threadIdx.x] = to_c<T>(h[(long long)r * ldh + threadIdx.x]);
  __syncthreads();
  const T sg = (T)sign;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    C<T> acc = mk<T>(0, 0);
    for (int i = 0; i < k1; ++i) {
      const C<T> a = V[((long long)i * R + r) * n + idx];
      const C<T> c = hs[i];
      acc.x = mad(c.x, a.x, acc.x);
      acc.x = mad(-c.y, a.y, acc.x);
      acc.y = mad(c.x, a.y, acc.y);
      acc.y = mad(c.y, a.x, acc.y);
    }
    C<T> v = w[(long long)r * n + idx];
    v.x += sg * acc.x;
    v.y += sg * acc.y;
    w[(long long)r * n + idx] = v;
  }
}

// (FP64 sums also for c64 vectors: the norms set the thresholds and the first basis
// vector of every cycle)
template <typename T>
__global__ void __launch_bounds__(kT) norm_partial(const C<T> *__restrict__ w, double *__restrict__ part, long long n,
                                                   int nb) {
  __shared__ double2 sh[kT / 32];
  const int r = blockIdx.y;
  double acc = 0.0;
  for (long long idx = blockIdx.x * (long long)kT + threadIdx.x; idx < n; idx += (long long)nb * kT) {
    const C<T> v = w[(long long)r * n + idx];
    acc = fma((double)v.x, (double)v.x, acc);
    acc = fma((double)v.y, (double)v.y, acc);
  }
  const double2 s = block_reduce(make_double2(acc, 0.0), sh);
  if (threadIdx.x == 0) part[(long long)r * nb + blockIdx.x] = s.x;
}

__global__ void norm_final(const double *__restrict__ part, double *__restrict__ out, int nb) {
  __shared__ double2 sh[kT / 32];
  const int r = blockIdx.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += kT) acc += part[(long long)r * nb + b];
  const double2 s = block_reduce(make_double2(acc, 0.0), sh);
  if (threadIdx.x == 0) out[r] = sqrt(s.x);
}

// dst[r] = src[r] / nrm[r]  (dst may alias src)
template <typename T>
__global__ void scale_kernel(const C<T> *__restrict__ src, C<T> *__restrict__ dst, const double *__restrict__ nrm,
                             long long n, const int *__restrict__ flag) {
  const int r = blockIdx.y;
  if (flag && !flag[r]) return;
  const T s = (T)(nrm[r] > 0.0 ? 1.0 / nrm[r] : 0.0);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    C<T> v = src[(long long)r * n + idx];
    dst[(long long)r * n + idx] = mk<T>(v.x * s, v.y * s);
  }
}

// out = a - b
template <typename T>
__global__ void sub_kernel(const C<T> *__restrict__ a, const C<T> *__restrict__ b, C<T> *__restrict__ out,
                           long long n) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const C<T> u = a[idx], v = b[idx];
    out[idx] = mk<T>(u.x - v.x, u.y - v.y);
  }
}

// y += x  (x c128 or c64, y c128)
template <typename T>
__global__ void add_kernel(const C<T> *__restrict__ x, double2 *__restrict__ y, long long n) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const C<T> u = x[idx];
    double2 v = y[idx];
    v.x += (double)u.x;
    v.y += (double)u.y;
    y[idx] = v;
  }
}

// y = x rounded to c64
__global__ void round_kernel(const double2 *__restrict__ x, float2 *__restrict__ y, long long n) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const double2 u = x[idx];
    y[idx] = make_float2((float)u.x, (float)u.y);
  }
}

// ---------------------------------------------------------------------------
// Classical Gram-Schmidt with selective reorthogonalisation.  In FP64 the arithmetic
// sets the pace (the vector length times the basis size in complex FMAs per pass); in
// FP32 the passes are bound by the basis reads from HBM, so both are organised to keep
// every SM busy with loads in flight and no wave tail:
//   dot pass: one warp per unit (right-hand side r, chunk c of kCh<T> elements, basis
//     vector i), units of one chunk consecutive so that the chunk of x comes from HBM
//     once and from L2 for the other vectors; part(r, i, c) = sum_chunk conj(V_i) x and,
//     with the i = 0 unit, npart(r, c) = sum_chunk |x|^2.  The grid is sized so that
//     every warp gets the same number of units.
//   sub pass: persistent blocks per right-hand side stream x -= sum_i h_i V_i over
//     chunks of kT * kSubEPT elements (the same number of chunks per block), one basis
//     vector at a time, and leave one partial of |x|^2 per block.
// A right-hand side whose flag (if given) is 0 is skipped.
// ---------------------------------------------------------------------------
template <typename T> struct GsShape;
template <> struct GsShape<float> { static constexpr int kCh = 512; static constexpr int kSubEPT = 8; };
template <> struct GsShape<double> { static constexpr int kCh = 2048; static constexpr int kSubEPT = 8; };

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
// lane 0 gets the warp's sum: FP32 vectors reduce in FP32 (32 lane sums of at most 32
// products each, ~1e-6 of the sum of magnitudes) and convert once; FP64 in FP64
__device__ __forceinline__ double warp_total(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return (double)v;
}
__device__ __forceinline__ double warp_total(double v) { return warp_sum(v); }

// one unit of the dot pass (a warp): (ax, ay) = sum conj(v) x over the chunk, nn = sum |x|^2
template <typename T, bool NORM>
__device__ __forceinline__ void dot_unit(const C<T> *__restrict__ vi, const C<T> *__restrict__ xr, long long lim,
                                         int lane, double &ax, double &ay, double &nn) {
  constexpr int PER = GsShape<T>::kCh / 32;
  const C<T> zero = mk<T>(0, 0);
  T ax0 = 0, ay0 = 0, ax1 = 0, ay1 = 0, n0 = 0, n1 = 0;
#pragma unroll 8
  for (int j = 0; j < PER; j += 2) {
    const int l0 = j * 32 + lane, l1 = l0 + 32;
    const C<T> a0 = l0 < lim ? __ldg(vi + l0) : zero, a1 = l1 < lim ? __ldg(vi + l1) : zero;
    const C<T> b0 = l0 < lim ? __ldg(xr + l0) : zero, b1 = l1 < lim ? __ldg(xr + l1) : zero;
    ax0 = mad(a0.x, b0.x, ax0);
    ax0 = mad(a0.y, b0.y, ax0);
    ay0 = mad(a0.x, b0.y, ay0);
    ay0 = mad(-a0.y, b0.x, ay0);
    ax1 = mad(a1.x, b1.x, ax1);
    ax1 = mad(a1.y, b1.y, ax1);
    ay1 = mad(a1.x, b1.y, ay1);
    ay1 = mad(-a1.y, b1.x, ay1);
    if (NORM) {
      n0 = mad(b0.x, b0.x, n0);
      n0 = mad(b0.y, b0.y, n0);
      n1 = mad(b1.x, b1.x, n1);
      n1 = mad(b1.y, b1.y, n1);
    }
  }
  ax = warp_total(ax0 + ax1);
  ay = warp_total(ay0 + ay1);
  if (NORM) nn = warp_total(n0 + n1);
}

template <typename T>
__global__ void __launch_bounds__(kT) cgs_dot_kernel(const C<T> *__restrict__ V, const C<T> *__restrict__ x,
                                                     double2 *__restrict__ part, double *__restrict__ npart,
                                                     const int *__restrict__ flag, int k1, int R, long long n,
                                                     int nch) {
  constexpr int CH = GsShape<T>::kCh;
  if (flag) {  // nothing to do unless some right-hand side is flagged
    int any = 0;
    for (int r = 0; r < R; ++r) any |= flag[r];
    if (!any) return;
  }
  const int lane = threadIdx.x & 31;
  const int nw = gridDim.x * (kT / 32);
  const int units = R * nch * k1;  // < 2^31 for every grid the library accepts
  for (int u = blockIdx.x * (kT / 32) + (threadIdx.x >> 5); u < units; u += nw) {
    const int i = u % k1, rc = u / k1;
    const int c = rc % nch, r = rc / nch;
    if (flag && !flag[r]) continue;
    const long long e0 = (long long)c * CH;
    const C<T> *vi = V + ((long long)i * R + r) * n + e0;
    const C<T> *xr = x + (long long)r * n + e0;
    double ax, ay, nn = 0.0;
    if (i == 0)
      dot_unit<T, true>(vi, xr, n - e0, lane, ax, ay, nn);
    else
      dot_unit<T, false>(vi, xr, n - e0, lane, ax, ay, nn);
    if (lane == 0) {
      part[((long long)r * k1 + i) * nch + c] = make_double2(ax, ay);
      if (i == 0) npart[(long long)r * nch + c] = nn;
    }
  }
}

// x[r] -= sum_{i<k1} h[r * ldh + i] V_i[r]; npart[r * nbs + block] = the block's part of
// |x'|^2.  With vout: a right-hand side whose oflag is 0 instead gets vout[r] = x' /
// nrm[r] (the next basis vector, normalised by the norm known in advance) and no norm
// partial; one whose oflag is 1 gets x' in x as above.
template <typename T>
__global__ void __launch_bounds__(kT) cgs_sub_kernel(const C<T> *__restrict__ V, C<T> *__restrict__ x,
                                                     const double2 *__restrict__ h, double *__restrict__ npart,
                                                     const int *__restrict__ flag, int k1, int R, long long n,
                                                     int nbs, int ldh, C<T> *__restrict__ vout,
                                                     const double *__restrict__ nrm, const int *__restrict__ oflag) {
  constexpr int EPT = GsShape<T>::kSubEPT;
  __shared__ C<T> hs[64];
  __shared__ double2 shn[kT / 32];
  const int r = blockIdx.y;
  if (flag && !flag[r]) return;
  const bool scaled = vout && !oflag[r];
  const int tid = threadIdx.x;
  if (tid < k1) hs[tid] = to_c<T>(h[(long long)r * ldh + tid]);
  __syncthreads();
  const T sc = (T)(scaled && nrm[r] > 0.0 ? 1.0 / nrm[r] : 0.0);
  C<T> *xr = x + (long long)r * n;
  C<T> *vr = vout ? vout + (long long)r * n : nullptr;
  T nacc = 0;
  for (long long c0 = (long long)blockIdx.x * kT * EPT; c0 < n; c0 += (long long)nbs * kT * EPT) {
    C<T> v[EPT];
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
      const long long e = c0 + j * kT + tid;
      v[j] = e < n ? xr[e] : mk<T>(0, 0);
    }
    // one basis vector at a time (8 loads in flight per thread): unrolling over vectors
    // costs registers and occupancy and measured slower (5.1 against 6.0 TB/s at k1 = 10)
#pragma unroll 1
    for (int i = 0; i < k1; ++i) {
      const C<T> hv = hs[i];
      const C<T> *vi = V + ((long long)i * R + r) * n + c0 + tid;
#pragma unroll
      for (int j = 0; j < EPT; ++j) {
        if (c0 + j * kT + tid < n) {
          const C<T> a = __ldg(vi + j * kT);
          v[j].x = mad(-hv.x, a.x, v[j].x);
          v[j].x = mad(hv.y, a.y, v[j].x);
          v[j].y = mad(-hv.x, a.y, v[j].y);
          v[j].y = mad(-hv.y, a.x, v[j].y);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
      const long long e = c0 + j * kT + tid;
      if (e < n) {
        if (scaled) {
          vr[e] = mk<T>(v[j].x * sc, v[j].y * sc);
        } else {
          xr[e] = v[j];
          nacc = mad(v[j].x, v[j].x, nacc);
          nacc = mad(v[j].y, v[j].y, nacc);
        }
      }
    }
  }
  if (scaled) return;
  const double2 sres = block_reduce(make_double2((double)nacc, 0.0), shn);
  if (tid == 0) npart[(long long)r * nbs + blockIdx.x] = sres.x;
}

// The test: ||x'||^2 = ||x||^2 - sum_i |h_i|^2 before the subtraction (x' = x - V h is the
// part of x orthogonal to the basis), flag[r] = 1 where ||x'|| < ||x|| / 16.  The test is
// that of Daniel, Gragg, Kaufman and Stewart with a looser threshold than their
// 1/sqrt(2): one projection leaves x' orthogonal to V up to about eps ||x|| / ||x'||,
// so below 1/16 cancellation the loss stays under ~16 eps per step: ~4e-15 in FP64,
// far below what restarted GMRES to 1e-7 can notice, and ~2e-6 in FP32, below the
// relative tolerance (>= 1e-4) of the inner solves that run in FP32.  The difference of
// squares is as accurate as the sums (FP64 ~1e-13, FP32 ~1e-6 of ||x||^2), i.e. at
// worst 256 times less relative to ||x'||^2.  For this operator the product A v_k is
// dominated by v_k, so 1/sqrt(2) would trigger the second projection in nearly every
// iteration, doubling the work.
//
// First projection, after the dot pass: block (i < k1, r) sums the chunk partials of
// h1[r][i] (and zeroes h2[r][i]), block (k1, r) those of ||w||^2 (kept in nrm[R + r]);
// the last of the k1 + 1 blocks of r to finish (a ticket counter, reset by it) runs the
// test below on r.
__global__ void __launch_bounds__(kT) cgs_hsum_kernel(const double2 *__restrict__ part,
                                                      const double *__restrict__ npart, double2 *__restrict__ h,
                                                      double2 *__restrict__ h2, double *__restrict__ nrm,
                                                      int *__restrict__ flag, unsigned *__restrict__ tick, int k1,
                                                      int R, int nch, int ldh) {
  __shared__ double2 sh[kT / 32];
  __shared__ int last;
  const int i = blockIdx.x, r = blockIdx.y, tid = threadIdx.x;
  double2 acc = make_double2(0.0, 0.0);
  if (i < k1) {
#pragma unroll 4
    for (int c = tid; c < nch; c += kT) {
      const double2 v = part[((long long)r * k1 + i) * nch + c];
      acc.x += v.x;
      acc.y += v.y;
    }
  } else {
#pragma unroll 4
    for (int c = tid; c < nch; c += kT) acc.x += npart[(long long)r * nch + c];
  }
  acc = block_reduce(acc, sh);
  if (tid == 0) {
    if (i < k1) {
      h[(long long)r * ldh + i] = acc;
      h2[(long long)r * ldh + i] = make_double2(0.0, 0.0);
    } else {
      nrm[R + r] = acc.x;
    }
    __threadfence();
    last = atomicAdd(&tick[r], 1u) == (unsigned)k1;
  }
  __syncthreads();
  if (!last) return;
  double a1 = 0.0;
  for (int j = tid; j < k1; j += kT) {
    const double2 v = __ldcg(&h[(long long)r * ldh + j]);
    a1 = fma(v.x, v.x, a1);
    a1 = fma(v.y, v.y, a1);
  }
  const double2 sa = block_reduce(make_double2(a1, 0.0), sh);
  if (tid == 0) {
    const double s0 = __ldcg(&nrm[R + r]);
    const double n0 = sqrt(s0);
    const double d = s0 - sa.x;
    const double n1 = d > 0.0 ? sqrt(d) : 0.0;
    nrm[r] = n1;
    flag[r] = n1 < 0.0625 * n0 ? 1 : 0;
    if (flag[r]) atomicAdd(&flag[32], 1);  // second projections so far
    tick[r] = 0u;
  }
}

// The second projection of every flagged right-hand side r in one cooperative launch
// (the grid is co-resident), which returns at once when no flag is set:
//   h2 = V^H w' (dot units), w'' = w' - V h2, nrm = ||w''||, vnext = w'' / nrm.
// The per-block norm partials go to npart[r * gridDim.x + block] (gridDim.x <= 1024).
// the split copy of one basis entry (defined with the double-float helpers below)
__device__ __forceinline__ float4 dsplit4(double2 v);

template <typename T>
__global__ void __launch_bounds__(kT) cgs_second_kernel(const C<T> *__restrict__ V, C<T> *__restrict__ w,
                                                        C<T> *__restrict__ vnext, double2 *__restrict__ h2,
                                                        double2 *__restrict__ part, double *__restrict__ npart,
                                                        double *__restrict__ nrm, const int *__restrict__ flag,
                                                        int k1, int R, long long n, int ldh, int nch,
                                                        float4 *__restrict__ vsnext) {
  int any = 0;
  for (int r = 0; r < R; ++r) any |= flag[r];
  if (!any) return;  // the same decision in every block: no block reaches a grid barrier
  cg::grid_group grid = cg::this_grid();
  __shared__ C<T> hs[64];
  __shared__ double2 shn[kT / 32];
  const int tid = threadIdx.x, lane = tid & 31;
  const int nw = gridDim.x * (kT / 32), gw = blockIdx.x * (kT / 32) + (tid >> 5);
  constexpr int CH = GsShape<T>::kCh;
  // h2 partials
  const int units = R * nch * k1;
  for (int u = gw; u < units; u += nw) {
    const int i = u % k1, rc = u / k1;
    const int c = rc % nch, r = rc / nch;
    if (!flag[r]) continue;
    const long long e0 = (long long)c * CH;
    double ax, ay, nn = 0.0;
    dot_unit<T, false>(V + ((long long)i * R + r) * n + e0, w + (long long)r * n + e0, n - e0, lane, ax, ay, nn);
    if (lane == 0) part[((long long)r * k1 + i) * nch + c] = make_double2(ax, ay);
  }
  grid.sync();
  // h2[r][i]: one warp per (r, i)
  for (int p = gw; p < R * k1; p += nw) {
    const int r = p / k1, i = p % k1;
    if (!flag[r]) continue;
    double ax = 0.0, ay = 0.0;
    for (int c = lane; c < nch; c += 32) {
      const double2 v = __ldcg(&part[((long long)r * k1 + i) * nch + c]);
      ax += v.x;
      ay += v.y;
    }
    ax = warp_sum(ax);
    ay = warp_sum(ay);
    if (lane == 0) h2[(long long)r * ldh + i] = make_double2(ax, ay);
  }
  grid.sync();
  // w'' = w' - V h2 and the block's part of ||w''||^2
  for (int r = 0; r < R; ++r) {
    if (!flag[r]) continue;
    __syncthreads();
    if (tid < k1) hs[tid] = to_c<T>(__ldcg(&h2[(long long)r * ldh + tid]));
    __syncthreads();
    T nacc = 0;
    for (long long e = (long long)blockIdx.x * kT + tid; e < n; e += (long long)gridDim.x * kT) {
      C<T> v = w[(long long)r * n + e];
      for (int i = 0; i < k1; ++i) {
        const C<T> a = V[((long long)i * R + r) * n + e], hv = hs[i];
        v.x = mad(-hv.x, a.x, v.x);
        v.x = mad(hv.y, a.y, v.x);
        v.y = mad(-hv.x, a.y, v.y);
        v.y = mad(-hv.y, a.x, v.y);
      }
      w[(long long)r * n + e] = v;
      nacc = mad(v.x, v.x, nacc);
      nacc = mad(v.y, v.y, nacc);
    }
    const double2 sres = block_reduce(make_double2((double)nacc, 0.0), shn);
    if (tid == 0) npart[(long long)r * gridDim.x + blockIdx.x] = sres.x;
  }
  grid.sync();
  // nrm = ||w''|| (every block sums the partials itself) and vnext = w'' / nrm
  for (int r = 0; r < R; ++r) {
    if (!flag[r]) continue;
    double a = 0.0;
    for (int b = tid; b < (int)gridDim.x; b += kT) a += __ldcg(&npart[(long long)r * gridDim.x + b]);
    const double2 sr = block_reduce(make_double2(a, 0.0), shn);  // the total in thread 0
    if (tid == 0) shn[0].x = sqrt(sr.x);
    __syncthreads();
    const double nr = shn[0].x;
    __syncthreads();
    if (blockIdx.x == 0 && tid == 0) nrm[r] = nr;
    const T sc = (T)(nr > 0.0 ? 1.0 / nr : 0.0);
    for (long long e = (long long)blockIdx.x * kT + tid; e < n; e += (long long)gridDim.x * kT) {
      const C<T> v = w[(long long)r * n + e];
      const C<T> vs = mk<T>(v.x * sc, v.y * sc);
      vnext[(long long)r * n + e] = vs;
      if constexpr (sizeof(T) == 8) {
        if (vsnext) vsnext[(long long)r * n + e] = dsplit4(vs);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Gram-Schmidt passes for FP64 vectors in double-float arithmetic (the inner solves of
// IE_MIXED_FP64K).  GB300 runs FP64 at about 1/64 of the FP32 rate, so the FP64 dot and
// subtract passes are bound by the FP64 pipe, not by their basis reads.  Here every FP64
// number x is taken as hi + lo (hi: x's leading 24 significant bits, lo: the next 23,
// so x = hi + lo up to 2^-46 |x|), split with integer operations on its bits, and the
// products go through the compensated scheme of Ogita, Rump and Oishi: TwoProduct by
// FMA, TwoSum into a second FP32 accumulator, the cross terms hi lo added to it (lo lo
// dropped).  A dot product is then as accurate as one in twice FP32 precision (about
// 2^-46 relative to the sum of magnitudes, against 2^-53 in FP64); the vectors stay
// FP64 in memory and the partial sums are combined in FP64.  Same chunking, partial
// layout and flags as cgs_dot_kernel / cgs_sub_kernel.
// ---------------------------------------------------------------------------
struct Df {
  float s, c;  // value s + c
};

// x = hi + lo + O(2^-46 |x|) for 2^-103 <= |x| < 2^127, from the bits of x with integer
// operations only (no FP64 instruction): below that range hi = lo = 0 (a relative
// contribution below 2^-103 of a unit vector); above it, and for Inf and NaN, hi is
// non-finite (Inf, or NaN where the leading 20 + 3 significand bits are not all zero,
// as in every NaN that arithmetic produces) and lo = 0, so that a non-finite vector
// still fails every test downstream
__device__ __forceinline__ void dsplit(double x, float &hi, float &lo) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const uint32_t uh = (uint32_t)(u >> 32), ul = (uint32_t)u;
  const uint32_t sgn = uh & 0x80000000u;
  const uint32_t e = (uh >> 20) & 0x7FFu;                    // biased FP64 exponent
  const uint32_t mh = ((uh & 0xFFFFFu) << 3) | (ul >> 29);  // significand bits 1..23
  const uint32_t ml = (ul >> 6) & 0x7FFFFFu;                // bits 24..46
  uint32_t h = sgn | ((e - 896u) << 23) | mh;
  // 0.m24..m46 = (1.m24..m46 - 1) exactly, times 2^(e - 1023 - 23) with the sign
  float l = __fmul_rn(__fsub_rn(__uint_as_float(0x3F800000u | ml), 1.0f), __uint_as_float(sgn | ((e - 919u) << 23)));
  const bool small = e < 920u, big = e > 1150u;
  h = small ? sgn : h;
  h = big ? (sgn | 0x7F800000u | mh) : h;
  l = (small || big) ? 0.0f : l;
  hi = __uint_as_float(h);
  lo = l;
}

// (re hi, re lo, im hi, im lo) of a complex FP64 value: its entry in the split copy of
// the Krylov basis that the double-float passes read
__device__ __forceinline__ float4 dsplit4(double2 v) {
  float4 q;
  dsplit(v.x, q.x, q.y);
  dsplit(v.y, q.z, q.w);
  return q;
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
}

// acc += (ah + al)(bh + bl)
__device__ __forceinline__ void df_fma(Df &acc, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float pe = __fmaf_rn(ah, bh, -p);
  pe = __fmaf_rn(ah, bl, pe);
  pe = __fmaf_rn(al, bh, pe);
  float t, e;
  two_sum(acc.s, p, t, e);
  acc.s = t;
  acc.c = __fadd_rn(acc.c, __fadd_rn(e, pe));
}

// a finite float as a double, built from its bits (no FP64 conversion instruction;
// FP32 subnormals, which carry no weight here, become zero)
__device__ __forceinline__ double f2d(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu;
  const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long bits =
      e == 0u ? sgn
              : (e == 0xFFu ? sgn | 0x7FF0000000000000ull | ((unsigned long long)(u & 0x7FFFFFu) << 29)
                            : sgn | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29));
  return __longlong_as_double((long long)bits);
}
// the value s + c: one FP64 addition
__device__ __forceinline__ double df_value(const Df &a) { return f2d(a.s) + f2d(a.c); }
// (s + c)(bh + bl) as a double-float
__device__ __forceinline__ Df df_mul(const Df &a, float bh, float bl) {
  Df r = {0.f, 0.f};
  df_fma(r, a.s, a.c, bh, bl);
  return r;
}

// a += b for double-floats (b given by its two parts)
__device__ __forceinline__ void df_add(Df &a, float bs, float bc) {
  float t, e;
  two_sum(a.s, bs, t, e);
  a.s = t;
  a.c = __fadd_rn(a.c, __fadd_rn(bc, e));
}
// sum over the warp in double-float (FP32 shuffles; the total in every lane)
__device__ __forceinline__ void df_warp_sum(Df &a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float bs = __shfl_xor_sync(0xffffffffu, a.s, o), bc = __shfl_xor_sync(0xffffffffu, a.c, o);
    df_add(a, bs, bc);
  }
}

// Warp sums of four double-floats at once by recursive halving: at the first two levels
// each lane sends the half of its values that its partner keeps, so the four totals
// cost six double-float additions and twelve shuffles per lane instead of twenty and
// forty.  Returns, in every lane, the total of a0 (lanes 0-7), a1 (8-15), b0 (16-23)
// or b1 (24-31).
__device__ __forceinline__ Df df_warp_sum4(const Df &a0, const Df &a1, const Df &b0, const Df &b1) {
  const int lane = threadIdx.x & 31;
  const bool u16 = (lane & 16) != 0, u8 = (lane & 8) != 0;
  Df k0 = u16 ? b0 : a0, k1 = u16 ? b1 : a1;
  const Df s0 = u16 ? a0 : b0, s1 = u16 ? a1 : b1;
  {
    const float p0 = __shfl_xor_sync(0xffffffffu, s0.s, 16), q0 = __shfl_xor_sync(0xffffffffu, s0.c, 16);
    const float p1 = __shfl_xor_sync(0xffffffffu, s1.s, 16), q1 = __shfl_xor_sync(0xffffffffu, s1.c, 16);
    df_add(k0, p0, q0);
    df_add(k1, p1, q1);
  }
  Df k = u8 ? k1 : k0;
  const Df sk = u8 ? k0 : k1;
  df_add(k, __shfl_xor_sync(0xffffffffu, sk.s, 8), __shfl_xor_sync(0xffffffffu, sk.c, 8));
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    const float bs = __shfl_xor_sync(0xffffffffu, k.s, o), bc = __shfl_xor_sync(0xffffffffu, k.c, o);
    df_add(k, bs, bc);
  }
  return k;
}

// Both double-float passes take chunks of kT * kDfEPT elements, kDfEPT per thread, and
// walk the basis one vector at a time with the next vector's loads already in flight
// (the dot pass keeps its chunk of x split in registers).  At 128 x 128 x 32 with two
// right-hand sides this ran the dot pass at 3.2-3.4 TB/s and the subtract pass at
// 4.3-4.4 TB/s for basis sizes 4-20, against 2.0-2.4 and 3.2-3.3 TB/s for groups of
// four basis vectors per warp (dot) and eight elements per thread without the
// pipelining (subtract); at that rate both are bound by the issue of the double-float
// arithmetic (about 100 instructions per complex element and basis vector).
constexpr int kDfEPT = 4;
constexpr int kDfCh = kT * kDfEPT;  // elements per chunk

// part(r, i, c) = sum_chunk conj(V_i) x and npart(r, c) = sum_chunk |x|^2, chunk c of
// kDfCh elements; grid (nbs, R), each block the same number of chunks
__global__ void __launch_bounds__(kT) cgs_dot_df_kernel(const float4 *__restrict__ Vs, const double2 *__restrict__ x,
                                                        double2 *__restrict__ part, double *__restrict__ npart, int k1,
                                                        int R, long long n, int nbs, int nch) {
  constexpr int EPT = kDfEPT;
  __shared__ double2 red[kT / 32][65];  // per warp: the k1 dot products, then |x|^2 in slot 64
  const int r = blockIdx.y, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const double2 *xr = x + (long long)r * n;
  const double2 z2 = make_double2(0.0, 0.0);
  for (long long c0 = (long long)blockIdx.x * kDfCh; c0 < n; c0 += (long long)nbs * kDfCh) {
    const int c = (int)(c0 / kDfCh);
    float xs[EPT][4];  // (re hi, re lo, im hi, im lo)
    Df nn = {0.f, 0.f};
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
      const long long e = c0 + j * kT + tid;
      const double2 v = e < n ? __ldg(xr + e) : z2;
      dsplit(v.x, xs[j][0], xs[j][1]);
      dsplit(v.y, xs[j][2], xs[j][3]);
      df_fma(nn, xs[j][0], xs[j][1], xs[j][0], xs[j][1]);
      df_fma(nn, xs[j][2], xs[j][3], xs[j][2], xs[j][3]);
    }
    df_warp_sum(nn);
    if (lane == 0) red[wid][64] = make_double2(df_value(nn), 0.0);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 vn[EPT];
    {
      const float4 *v0 = Vs + (long long)r * n + c0 + tid;
#pragma unroll
      for (int j = 0; j < EPT; ++j) vn[j] = c0 + j * kT + tid < n ? __ldg(v0 + j * kT) : z4;
    }
    Df pre = {0.f, 0.f}, pim = {0.f, 0.f};  // an even basis vector's sums, awaiting its partner
#pragma unroll 1
    for (int i = 0; i < k1; ++i) {
      float4 vc[EPT];
#pragma unroll
      for (int j = 0; j < EPT; ++j) vc[j] = vn[j];
      if (i + 1 < k1) {
        const float4 *v1 = Vs + ((long long)(i + 1) * R + r) * n + c0 + tid;
#pragma unroll
        for (int j = 0; j < EPT; ++j) vn[j] = c0 + j * kT + tid < n ? __ldg(v1 + j * kT) : z4;
      }
      Df are = {0.f, 0.f}, aim = {0.f, 0.f};
#pragma unroll
      for (int j = 0; j < EPT; ++j) {
        const float vrh = vc[j].x, vrl = vc[j].y, vih = vc[j].z, vil = vc[j].w;
        // conj(v) x = (vr xr + vi xi) + i (vr xi - vi xr)
        df_fma(are, vrh, vrl, xs[j][0], xs[j][1]);
        df_fma(are, vih, vil, xs[j][2], xs[j][3]);
        df_fma(aim, vrh, vrl, xs[j][2], xs[j][3]);
        df_fma(aim, -vih, -vil, xs[j][0], xs[j][1]);
      }
      if (!(i & 1) && i + 1 < k1) {
        pre = are;
        pim = aim;
        continue;
      }
      // the pair (i - 1, i), or the last vector alone
      const int i0 = (i & 1) ? i - 1 : i;
      const Df z = {0.f, 0.f};
      const Df tot = (i & 1) ? df_warp_sum4(pre, pim, are, aim) : df_warp_sum4(are, aim, z, z);
      if ((lane & 7) == 0 && (i0 + (lane >> 4)) <= i) {
        double *dst = reinterpret_cast<double *>(&red[wid][i0 + (lane >> 4)]) + ((lane >> 3) & 1);
        *dst = df_value(tot);
      }
    }
    __syncthreads();
    if (tid <= k1) {
      const int i = tid < k1 ? tid : 64;
      double sx = 0.0, sy = 0.0;
#pragma unroll
      for (int w = 0; w < kT / 32; ++w) {
        sx += red[w][i].x;
        sy += red[w][i].y;
      }
      if (tid < k1) part[((long long)r * k1 + tid) * nch + c] = make_double2(sx, sy);
      else npart[(long long)r * nch + c] = sx;
    }
    __syncthreads();
  }
}

// x[r] -= sum_{i<k1} h[r * ldh + i] V_i[r] in double-float (neg = 0: x += ...); otherwise
// as cgs_sub_kernel (vout, nrm, oflag: the normalised next basis vector where no second
// projection runs; npart may be NULL when no norm is wanted)
__global__ void __launch_bounds__(kT) cgs_sub_df_kernel(const float4 *__restrict__ Vs, double2 *__restrict__ x,
                                                        const double2 *__restrict__ h, double *__restrict__ npart,
                                                        int k1, int R, long long n, int nbs, int ldh,
                                                        double2 *__restrict__ vout, float4 *__restrict__ vsout,
                                                        const double *__restrict__ nrm,
                                                        const int *__restrict__ oflag, int neg) {
  constexpr int EPT = kDfEPT;
  __shared__ float4 hs[64];  // -h split: (-hr hi, -hr lo, -hi hi, -hi lo)
  __shared__ double2 shn[kT / 32];
  const int r = blockIdx.y;
  const bool scaled = vout && !oflag[r];
  const int tid = threadIdx.x;
  if (tid < k1) {
    const double2 hv = h[(long long)r * ldh + tid];
    float a, b, c, d;
    dsplit(neg ? -hv.x : hv.x, a, b);
    dsplit(neg ? -hv.y : hv.y, c, d);
    hs[tid] = make_float4(a, b, c, d);
  }
  __syncthreads();
  const double sc = scaled && nrm[r] > 0.0 ? 1.0 / nrm[r] : 0.0;
  float sch, scl;
  dsplit(sc, sch, scl);
  double2 *xr = x + (long long)r * n;
  double2 *vr = vout ? vout + (long long)r * n : nullptr;
  Df nacc = {0.f, 0.f};
  for (long long c0 = (long long)blockIdx.x * kDfCh; c0 < n; c0 += (long long)nbs * kDfCh) {
    Df ar[EPT], ai[EPT];
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
      const long long e = c0 + j * kT + tid;
      const double2 v = e < n ? xr[e] : make_double2(0.0, 0.0);
      dsplit(v.x, ar[j].s, ar[j].c);
      dsplit(v.y, ai[j].s, ai[j].c);
    }
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 vn[EPT];
    {
      const float4 *v0 = Vs + (long long)r * n + c0 + tid;
#pragma unroll
      for (int j = 0; j < EPT; ++j) vn[j] = c0 + j * kT + tid < n ? __ldg(v0 + j * kT) : z4;
    }
#pragma unroll 1
    for (int i = 0; i < k1; ++i) {
      const float4 hv = hs[i];  // -h
      float4 vc[EPT];
#pragma unroll
      for (int j = 0; j < EPT; ++j) vc[j] = vn[j];
      if (i + 1 < k1) {
        const float4 *v1 = Vs + ((long long)(i + 1) * R + r) * n + c0 + tid;
#pragma unroll
        for (int j = 0; j < EPT; ++j) vn[j] = c0 + j * kT + tid < n ? __ldg(v1 + j * kT) : z4;
      }
#pragma unroll
      for (int j = 0; j < EPT; ++j) {
        const float vrh = vc[j].x, vrl = vc[j].y, vih = vc[j].z, vil = vc[j].w;
        // x += (-h) v: re += (-hr) vr - (-hi) vi, im += (-hr) vi + (-hi) vr
        df_fma(ar[j], hv.x, hv.y, vrh, vrl);
        df_fma(ar[j], -hv.z, -hv.w, vih, vil);
        df_fma(ai[j], hv.x, hv.y, vih, vil);
        df_fma(ai[j], hv.z, hv.w, vrh, vrl);
      }
    }
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
      const long long e = c0 + j * kT + tid;
      if (e < n) {
        if (scaled) {
          const double2 v = make_double2(df_value(df_mul(ar[j], sch, scl)), df_value(df_mul(ai[j], sch, scl)));
          vr[e] = v;
          if (vsout) vsout[(long long)r * n + e] = dsplit4(v);
        } else {
          xr[e] = make_double2(df_value(ar[j]), df_value(ai[j]));
          df_fma(nacc, ar[j].s, ar[j].c, ar[j].s, ar[j].c);
          df_fma(nacc, ai[j].s, ai[j].c, ai[j].s, ai[j].c);
        }
      }
    }
  }
  if (scaled || !npart) return;
  const double2 sres = block_reduce(make_double2(df_value(nacc), 0.0), shn);
  if (tid == 0) npart[(long long)r * nbs + blockIdx.x] = sres.x;
}

// vs = the split copy of v (dsplit4 of every entry)
__global__ void __launch_bounds__(kT) split_vec_kernel(const double2 *__restrict__ v, float4 *__restrict__ vs,
                                                       long long n) {
  for (long long e = blockIdx.x * (long long)kT + threadIdx.x; e < n; e += (long long)gridDim.x * kT)
    vs[e] = dsplit4(v[e]);
}

// chunks of the dot pass per right-hand side
template <typename T> int cgs_nch(long long n) {
  return (int)((n + GsShape<T>::kCh - 1) / GsShape<T>::kCh);
}

// resident blocks per SM of the two passes (occupancy of the compiled kernels)
template <typename T> int sub_per_sm() {
  static int v = 0;
  if (v == 0 && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, cgs_sub_kernel<T>, kT, 0) != cudaSuccess || v < 1)) {
    cudaGetLastError();
    v = 1;
  }
  return v;
}
template <typename T> int dot_per_sm() {
  static int v = 0;
  if (v == 0 && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, cgs_dot_kernel<T>, kT, 0) != cudaSuccess || v < 1)) {
    cudaGetLastError();
    v = 1;
  }
  return v;
}

// blocks per right-hand side of the sub pass: at most one wave of the GPU over all R,
// every block the same number of chunks
template <typename T> int cgs_nbs(long long n, int R) {
  const long long chunks = (n + (long long)kT * GsShape<T>::kSubEPT - 1) / ((long long)kT * GsShape<T>::kSubEPT);
  long long maxb = ((long long)sub_per_sm<T>() * sm_count()) / R;
  if (maxb < 1) maxb = 1;
  const long long per = (chunks + maxb - 1) / maxb;
  return (int)((chunks + per - 1) / per);
}

// blocks of the dot pass: at most one wave, every warp the same number of units
template <typename T> int cgs_dot_blocks(long long units) {
  const long long maxw = (long long)dot_per_sm<T>() * sm_count() * (kT / 32);
  const long long per = (units + maxw - 1) / maxw;
  const long long warps = (units + per - 1) / per;
  const long long b = (warps + kT / 32 - 1) / (kT / 32);
  return (int)(b < 1 ? 1 : b);
}

// grid of the element-wise kernels (grid-stride loops): up to eight 256-thread blocks
// per SM
int blocks_for(long long n) {
  long long g = (n + kT - 1) / kT;
  const long long cap = 8LL * sm_count();
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

int mdot_nb(long long n) { return (int)((n + kChunk - 1) / kChunk); }

template <typename T>
void gmres_maxpy(const C<T> *V, const double2 *h, C<T> *w, int k1, int R, long long n, int ldh, double sign,
                 cudaStream_t s) {
  count_launches(1);
  maxpy_kernel<T><<<dim3(blocks_for(n), R), kT, 0, s>>>(V, h, w, k1, R, n, ldh, sign);
}

template <typename T>
void gmres_norm(const C<T> *w, double *part, double *out, int R, long long n, cudaStream_t s) {
  int nb = mdot_nb(n);
  if (nb > 1024) nb = 1024;
  count_launches(2);
  norm_partial<T><<<dim3(nb, R), kT, 0, s>>>(w, part, n, nb);
  norm_final<<<R, kT, 0, s>>>(part, out, nb);
}

// blocks per right-hand side of the double-float passes: at most one wave of the GPU
// over all R (at the smaller occupancy of the two kernels), every block the same
// number of kDfCh-element chunks
int df_blocks(long long n, int R) {
  static int per = 0;
  if (per == 0) {
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, cgs_dot_df_kernel, kT, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, cgs_sub_df_kernel, kT, 0) != cudaSuccess) {
      cudaGetLastError();
      a = b = 1;
    }
    per = a < b ? a : b;
    if (per < 1) per = 1;
  }
  const long long chunks = (n + kDfCh - 1) / kDfCh;
  long long maxb = ((long long)per * sm_count()) / R;
  if (maxb < 1) maxb = 1;
  const long long each = (chunks + maxb - 1) / maxb;
  return (int)((chunks + each - 1) / each);
}

template <typename T> int second_blocks() {
  static int v = 0;
  if (v == 0) {
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, cgs_second_kernel<T>, kT, 0) != cudaSuccess || per < 1) {
      cudaGetLastError();
      per = 1;
    }
    // two blocks per SM at most: the launch is cheap when nothing is flagged (the usual
    // case) and still streams at full width when something is
    v = (per < 2 ? per : 2) * sm_count();
    if (v > 1024) v = 1024;
  }
  return v;
}

template <typename T>
int gmres_orthogonalize(const C<T> *V, C<T> *w, C<T> *vnext, double2 *h1, double2 *h2, double2 *part, double *npart,
                        double *nrm, int *flag, int k1, int R, long long n, int ldh, cudaStream_t s, bool df,
                        const float4 *Vs, float4 *vs_next) {
  if (k1 < 1 || k1 > 64 || R < 1 || R > 16) return -1;
  df = df && sizeof(T) == 8 && Vs && vs_next;
  const int nch = cgs_nch<T>(n), nbs = cgs_nbs<T>(n, R);
  // the double-float dot pass uses shorter chunks (more of them: gs_partial_blocks
  // allows the count of the c64 chunking, the largest); np1 starts past either
  const int nch_max = gs_partial_blocks(n);
  int nch_used = nch;
  double *np0 = npart, *np1 = npart + (long long)R * nch_max;
  unsigned *tick = reinterpret_cast<unsigned *>(flag + 16);
  count_launches(4);
  // first projection: h1 = V^H w and ||w||; ||w'|| from the difference of squares
  if constexpr (sizeof(T) == 8) {
    if (df) {
      nch_used = (int)((n + kDfCh - 1) / kDfCh);
      const int nbd = df_blocks(n, R);
      cgs_dot_df_kernel<<<dim3(nbd, R), kT, 0, s>>>(Vs, w, part, np0, k1, R, n, nbd, nch_used);
    }
  }
  if (!df) {
    const int gd = cgs_dot_blocks<T>((long long)R * nch * k1);
    cgs_dot_kernel<T><<<gd, kT, 0, s>>>(V, w, part, np0, nullptr, k1, R, n, nch);
  }
  cgs_hsum_kernel<<<dim3(k1 + 1, R), kT, 0, s>>>(part, np0, h1, h2, nrm, flag, tick, k1, R, nch_used, ldh);
  // w' = w - V h1, written normalised into vnext where no second projection is needed
  if constexpr (sizeof(T) == 8) {
    if (df) {
      const int nbd = df_blocks(n, R);
      cgs_sub_df_kernel<<<dim3(nbd, R), kT, 0, s>>>(Vs, w, h1, np1, k1, R, n, nbd, ldh, vnext, vs_next, nrm, flag, 1);
    }
  }
  if (!df) cgs_sub_kernel<T><<<dim3(nbs, R), kT, 0, s>>>(V, w, h1, np1, nullptr, k1, R, n, nbs, ldh, vnext, nrm, flag);
  // second projection where the first cancelled too much (h2 = 0 elsewhere)
  const C<T> *Va = V;
  C<T> *wa = w, *va = vnext;
  double2 *h2a = h2, *pa = part;
  double *npa = np1, *nrma = nrm;
  const int *fa = flag;
  int k1a = k1, Ra = R, ldha = ldh, ncha = nch;
  long long na = n;
  float4 *vsa = df ? vs_next : nullptr;
  void *args[] = {&Va, &wa, &va, &h2a, &pa, &npa, &nrma, &fa, &k1a, &Ra, &na, &ldha, &ncha, &vsa};
  if (cudaLaunchCooperativeKernel((const void *)cgs_second_kernel<T>, dim3(second_blocks<T>()), dim3(kT), args, 0, s) !=
      cudaSuccess)
    return -1;
  return 0;
}

// ---------------------------------------------------------------------------
// Givens rotations and the least-squares solution of GMRES on the device, one thread
// per right-hand side (the Hessenberg columns never leave the GPU).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double zabs(double2 a) { return hypot(a.x, a.y); }

// new cycle: g = (||r_0||, 0, ...), active where ||r_0|| > thr, no columns yet
__global__ void givens_init_kernel(GivensState st, const double *nrm, int R, int ldh) {
  const int r = threadIdx.x;
  __shared__ int cnt;
  if (r == 0) cnt = 0;
  __syncthreads();
  if (r < R) {
    for (int i = 0; i < ldh; ++i) st.g[(long long)r * ldh + i] = make_double2(i == 0 ? nrm[r] : 0.0, 0.0);
    const int act = nrm[r] > st.thr[r] ? 1 : 0;
    st.active[r] = act;
    st.kr[r] = 0;
    st.brk[r] = 0;
    if (act) atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (r == 0) *st.n_active = cnt;
}

// column k of the Hessenberg matrix (h1 + h2 above the diagonal, nrm below) for every
// active right-hand side: previous rotations, the new rotation, the residual estimate
// |g_{k+1}|; a right-hand side leaves the iteration when the estimate reaches thr or
// the new vector vanished (breakdown).  One warp per right-hand side: the lanes stage
// the column and the rotations in shared memory, lane 0 runs the recurrence from there.
constexpr int kGivWarps = 16;
// A: the arithmetic of the recurrence (FP32 for the c64 inner solves, whose tolerance is
// at least 1e-4; FP64 otherwise); the state stays FP64 in memory.
template <typename A>
__global__ void __launch_bounds__(kGivWarps * 32) givens_kernel(GivensState st, const double2 *h1, const double2 *h2,
                                                               const double *nrm, int k, int R, int m, int ldh) {
  using Z = C<A>;
  __shared__ Z col_s[kGivWarps][64];
  __shared__ Z sn_s[kGivWarps][64];
  __shared__ A cs_s[kGivWarps][64];
  __shared__ int cnt;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int r = wid; r < R; r += nwarp) {
    if (!st.active[r]) continue;
    Z *cs_col = col_s[wid];
    for (int i = lane; i <= k; i += 32) {
      const double2 a = h1[(long long)r * ldh + i], b = h2[(long long)r * ldh + i];
      cs_col[i] = mk<A>((A)(a.x + b.x), (A)(a.y + b.y));
    }
    for (int i = lane; i < k; i += 32) {
      cs_s[wid][i] = (A)st.cs[(long long)r * m + i];
      const double2 v = st.sn[(long long)r * m + i];
      sn_s[wid][i] = mk<A>((A)v.x, (A)v.y);
    }
    __syncwarp();
    if (lane == 0) {
      const A hk1 = (A)nrm[r];
      Z bi_next = cs_col[0];
      for (int i = 0; i < k; ++i) {
        const A ci = cs_s[wid][i];
        const Z si = sn_s[wid][i];
        const Z ai = bi_next, bi = cs_col[i + 1];
        const Z sb = cmul(si, bi), na = cmul(cconj(si), ai);
        cs_col[i] = mk<A>(ci * ai.x + sb.x, ci * ai.y + sb.y);
        bi_next = mk<A>(-na.x + ci * bi.x, -na.y + ci * bi.y);
      }
      const Z a = bi_next;
      const A aa = hypot(a.x, a.y);
      const A rho = hypot(aa, hk1);
      A ck;
      Z sk;
      if (aa == (A)0) {
        ck = (A)0;
        sk = mk<A>((A)1, (A)0);
      } else {
        ck = aa / rho;
        sk = mk<A>(a.x / aa * hk1 / rho, a.y / aa * hk1 / rho);
      }
      cs_col[k] = mk<A>(ck * a.x + sk.x * hk1, ck * a.y + sk.y * hk1);
      st.cs[(long long)r * m + k] = (double)ck;
      st.sn[(long long)r * m + k] = make_double2((double)sk.x, (double)sk.y);
      double2 *gr = st.g + (long long)r * ldh;
      const Z gk = mk<A>((A)gr[k].x, (A)gr[k].y);
      const Z gn = cmul(cconj(sk), gk);
      gr[k + 1] = make_double2(-(double)gn.x, -(double)gn.y);
      gr[k] = make_double2((double)(ck * gk.x), (double)(ck * gk.y));
      st.kr[r] = k + 1;
      int act = 1;
      if (hk1 == (A)0) {
        act = 0;
        st.brk[r] = 1;
      }
      if (hypot(gn.x, gn.y) <= (A)st.thr[r]) act = 0;
      st.active[r] = act;
    }
    __syncwarp();
    double2 *col = st.Rm + ((long long)r * m + k) * ldh;
    for (int i = lane; i <= k; i += 32) col[i] = make_double2((double)cs_col[i].x, (double)cs_col[i].y);
    __syncwarp();
  }
  __syncthreads();
  if ((int)threadIdx.x < R && st.active[threadIdx.x]) atomicAdd(&cnt, 1);
  __syncthreads();
  if (threadIdx.x == 0) *st.n_active = cnt;
}

// y = R^-1 g over the kr columns of each right-hand side; yd[r * ldh + i] (zero beyond kr)
__global__ void backsub_kernel(GivensState st, double2 *yd, int R, int m, int ldh) {
  const int r = threadIdx.x;
  if (r >= R) return;
  const int kr = st.kr[r];
  double2 *y = yd + (long long)r * ldh;
  for (int i = kr; i < ldh; ++i) y[i] = make_double2(0.0, 0.0);
  for (int i = kr - 1; i >= 0; --i) {
    double2 acc = st.g[(long long)r * ldh + i];
    for (int j = i + 1; j < kr; ++j) {
      const double2 p = zmul(st.Rm[((long long)r * m + j) * ldh + i], y[j]);
      acc.x -= p.x;
      acc.y -= p.y;
    }
    const double2 d = st.Rm[((long long)r * m + i) * ldh + i];
    const double dd = d.x * d.x + d.y * d.y;
    y[i] = dd == 0.0 ? make_double2(0.0, 0.0)
                     : make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd);
  }
}

// z[r] = Q^H (g_kr e_kr): the residual of the cycle's least-squares solution in the
// basis V_0..V_kr (the rotations applied in reverse, G_i^H (a, b) = (c a - s b,
// conj(s) a + c b)); zero beyond kr
__global__ void residual_coeffs_kernel(GivensState st, double2 *z, int R, int m, int ldh) {
  const int r = threadIdx.x;
  if (r >= R) return;
  const int kr = st.kr[r];
  double2 *zr = z + (long long)r * ldh;
  for (int i = 0; i < ldh; ++i) zr[i] = make_double2(0.0, 0.0);
  zr[kr] = st.g[(long long)r * ldh + kr];
  for (int i = kr - 1; i >= 0; --i) {
    const double c = st.cs[(long long)r * m + i];
    const double2 sn = st.sn[(long long)r * m + i];
    const double2 a = zr[i], b = zr[i + 1];
    const double2 sb = zmul(sn, b), sa = zmul(zconj(sn), a);
    zr[i] = make_double2(c * a.x - sb.x, c * a.y - sb.y);
    zr[i + 1] = make_double2(sa.x + c * b.x, sa.y + c * b.y);
  }
}

int gs_partial_blocks(long long n) { return cgs_nch<float>(n) > cgs_nch<double>(n) ? cgs_nch<float>(n) : cgs_nch<double>(n); }

void givens_init(const GivensState &st, const double *nrm, int R, int ldh, cudaStream_t s) {
  count_launches(1);
  givens_init_kernel<<<1, 32, 0, s>>>(st, nrm, R, ldh);
}

void givens_step(const GivensState &st, const double2 *h1, const double2 *h2, const double *nrm, int k, int R, int m,
                 int ldh, bool fp32, cudaStream_t s) {
  count_launches(1);
  const int warps = R < kGivWarps ? R : kGivWarps;
  const dim3 blk(32 * (warps > 0 ? warps : 1));
  if (fp32)
    givens_kernel<float><<<1, blk, 0, s>>>(st, h1, h2, nrm, k, R, m, ldh);
  else
    givens_kernel<double><<<1, blk, 0, s>>>(st, h1, h2, nrm, k, R, m, ldh);
}

void givens_residual(const GivensState &st, double2 *z, int R, int m, int ldh, cudaStream_t s) {
  count_launches(1);
  residual_coeffs_kernel<<<1, 32, 0, s>>>(st, z, R, m, ldh);
}

void givens_solve(const GivensState &st, double2 *yd, int R, int m, int ldh, cudaStream_t s) {
  count_launches(1);
  backsub_kernel<<<1, 32, 0, s>>>(st, yd, R, m, ldh);
}

void gmres_maxpy_df(const float4 *Vs, const double2 *h, double2 *x, int k1, int R, long long n, int ldh,
                    cudaStream_t s) {
  if (k1 < 0 || k1 > 64) return;
  const int nbd = df_blocks(n, R);
  count_launches(1);
  cgs_sub_df_kernel<<<dim3(nbd, R), kT, 0, s>>>(Vs, x, h, nullptr, k1, R, n, nbd, ldh, nullptr, nullptr, nullptr,
                                                nullptr, 0);
}

void gmres_split(const double2 *v, float4 *vs, long long n, cudaStream_t s) {
  count_launches(1);
  split_vec_kernel<<<blocks_for(n), kT, 0, s>>>(v, vs, n);
}

template <typename T>
void gmres_scale(const C<T> *src, C<T> *dst, const double *nrm, int R, long long n, cudaStream_t s) {
  count_launches(1);
  scale_kernel<T><<<dim3(blocks_for(n), R), kT, 0, s>>>(src, dst, nrm, n, nullptr);
}

template <typename T>
void vec_sub(const C<T> *a, const C<T> *b, C<T> *out, long long n, cudaStream_t s) {
  count_launches(1);
  sub_kernel<T><<<blocks_for(n), kT, 0, s>>>(a, b, out, n);
}

template <typename T>
void vec_add(const C<T> *x, double2 *y, long long n, cudaStream_t s) {
  count_launches(1);
  add_kernel<T><<<blocks_for(n), kT, 0, s>>>(x, y, n);
}

void vec_round(const double2 *x, float2 *y, long long n, cudaStream_t s) {
  count_launches(1);
  round_kernel<<<blocks_for(n), kT, 0, s>>>(x, y, n);
}

#define IE_BLAS_INSTANTIATE(T)                                                                                      \
  template void gmres_maxpy<T>(const C<T> *, const double2 *, C<T> *, int, int, long long, int, double,            \
                               cudaStream_t);                                                                       \
  template void gmres_norm<T>(const C<T> *, double *, double *, int, long long, cudaStream_t);                      \
  template int gmres_orthogonalize<T>(const C<T> *, C<T> *, C<T> *, double2 *, double2 *, double2 *, double *,      \
                                      double *, int *, int, int, long long, int, cudaStream_t, bool, const float4 *, \
                                      float4 *);                                                                   \
  template void gmres_scale<T>(const C<T> *, C<T> *, const double *, int, long long, cudaStream_t);                 \
  template void vec_sub<T>(const C<T> *, const C<T> *, C<T> *, long long, cudaStream_t);                           \
  template void vec_add<T>(const C<T> *, double2 *, long long, cudaStream_t);
IE_BLAS_INSTANTIATE(float)
IE_BLAS_INSTANTIATE(double)
#undef IE_BLAS_INSTANTIATE

}  // namespace ie
