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

namespace ie {
namespace {

constexpr int kT = 256;
constexpr int kEPT = 4;            // elements per thread in the reductions
constexpr int kChunk = kT * kEPT;  // elements per block

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
// sets the pace (the vector length times the basis size in complex FMAs per pass), so
// the passes are organised to spend the FP64 pipe on multiply-adds and little else; in
// FP32 the same passes are bound by the basis reads from HBM.
// A block owns a tile of kTile consecutive elements of one right-hand side.
//   dot pass: part_i = sum_tile conj(V_i) x  and  npart = sum_tile |x|^2
//   sub pass: x -= sum_i h_i V_i on the tile  and  npart = sum_tile |x|^2
// In the dot pass the tile of x sits in shared memory and warp j owns basis vectors
// j, j + 8, ...: each lane accumulates over 64 elements of the tile before a single
// warp reduction (in FP64) per (vector, tile).  With a per-right-hand-side flag the
// block of a right-hand side whose flag is 0 returns at once.
// ---------------------------------------------------------------------------
constexpr int kTileEPT = 8;
constexpr int kTile = kT * kTileEPT;  // 2048 elements

template <typename T>
__global__ void __launch_bounds__(kT) cgs_dot_kernel(const C<T> *__restrict__ V, const C<T> *__restrict__ x,
                                                     double2 *__restrict__ part, double *__restrict__ npart,
                                                     const int *__restrict__ flag, int k1, int R, long long n,
                                                     int nb) {
  __shared__ C<T> xw[kTile];
  __shared__ double2 shn[kT / 32];
  const int r = blockIdx.y;
  if (flag && !flag[r]) return;
  const long long t0 = (long long)blockIdx.x * kTile;
  const int tid = threadIdx.x;
  const C<T> *xr = x + (long long)r * n;
  const C<T> zero = mk<T>(0, 0);
  T nacc = 0;
#pragma unroll
  for (int j = 0; j < kTileEPT; ++j) {
    const long long e = t0 + j * kT + tid;
    const C<T> v = e < n ? xr[e] : zero;
    xw[j * kT + tid] = v;
    nacc = mad(v.x, v.x, nacc);
    nacc = mad(v.y, v.y, nacc);
  }
  const double2 sres = block_reduce(make_double2((double)nacc, 0.0), shn);  // also orders the xw stores
  if (tid == 0) npart[(long long)r * nb + blockIdx.x] = sres.x;
  const int lane = tid & 31, wid = tid >> 5;
  const long long lim = n - t0;  // elements of the tile inside the vector
  for (int i = wid; i < k1; i += kT / 32) {
    const C<T> *vi = V + ((long long)i * R + r) * n + t0;
    T ax0 = 0, ay0 = 0, ax1 = 0, ay1 = 0;
#pragma unroll 8
    for (int q = 0; q < kTile / 32; q += 2) {
      const int l0 = q * 32 + lane, l1 = l0 + 32;
      const C<T> a0 = l0 < lim ? __ldg(vi + l0) : zero;
      const C<T> a1 = l1 < lim ? __ldg(vi + l1) : zero;
      const C<T> b0 = xw[l0], b1 = xw[l1];
      ax0 = mad(a0.x, b0.x, ax0);
      ax0 = mad(a0.y, b0.y, ax0);
      ay0 = mad(a0.x, b0.y, ay0);
      ay0 = mad(-a0.y, b0.x, ay0);
      ax1 = mad(a1.x, b1.x, ax1);
      ax1 = mad(a1.y, b1.y, ax1);
      ay1 = mad(a1.x, b1.y, ay1);
      ay1 = mad(-a1.y, b1.x, ay1);
    }
    double ax = (double)ax0 + (double)ax1, ay = (double)ay0 + (double)ay1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ax += __shfl_down_sync(0xffffffffu, ax, o);
      ay += __shfl_down_sync(0xffffffffu, ay, o);
    }
    if (lane == 0) part[((long long)r * k1 + i) * nb + blockIdx.x] = make_double2(ax, ay);
  }
}

// x[r] -= sum_{i<k1} h[r * ldh + i] V_i[r] on the tile; npart = sum_tile |x|^2.
// With vout: a right-hand side whose oflag is 0 instead gets vout[r] = x' / nrm[r]
// (the next basis vector, normalised by the norm known in advance) and no norm
// partial; one whose oflag is 1 gets x' in x as above.  A right-hand side whose
// flag (if given) is 0 is skipped.
template <typename T>
__global__ void __launch_bounds__(kT) cgs_sub_kernel(const C<T> *__restrict__ V, C<T> *__restrict__ x,
                                                     const double2 *__restrict__ h, double *__restrict__ npart,
                                                     const int *__restrict__ flag, int k1, int R, long long n,
                                                     int nb, int ldh, C<T> *__restrict__ vout,
                                                     const double *__restrict__ nrm, const int *__restrict__ oflag) {
  __shared__ C<T> hs[64];
  __shared__ double2 shn[kT / 32];
  const int r = blockIdx.y;
  if (flag && !flag[r]) return;
  const bool scaled = vout && !oflag[r];
  const long long t0 = (long long)blockIdx.x * kTile;
  const int tid = threadIdx.x;
  C<T> *xr = x + (long long)r * n;
  if (tid < k1) hs[tid] = to_c<T>(h[(long long)r * ldh + tid]);
  __syncthreads();
  C<T> v[kTileEPT];
#pragma unroll
  for (int j = 0; j < kTileEPT; ++j) {
    const long long e = t0 + j * kT + tid;
    v[j] = e < n ? xr[e] : mk<T>(0, 0);
  }
  for (int i = 0; i < k1; ++i) {
    const C<T> hv = hs[i];
    const C<T> *vi = V + ((long long)i * R + r) * n;
#pragma unroll
    for (int j = 0; j < kTileEPT; ++j) {
      const long long e = t0 + j * kT + tid;
      if (e < n) {
        const C<T> a = __ldg(vi + e);
        v[j].x = mad(-hv.x, a.x, v[j].x);
        v[j].x = mad(hv.y, a.y, v[j].x);
        v[j].y = mad(-hv.x, a.y, v[j].y);
        v[j].y = mad(-hv.y, a.x, v[j].y);
      }
    }
  }
  if (scaled) {
    const T sc = (T)(nrm[r] > 0.0 ? 1.0 / nrm[r] : 0.0);
    C<T> *vr = vout + (long long)r * n;
#pragma unroll
    for (int j = 0; j < kTileEPT; ++j) {
      const long long e = t0 + j * kT + tid;
      if (e < n) vr[e] = mk<T>(v[j].x * sc, v[j].y * sc);
    }
    return;
  }
  T nacc = 0;
#pragma unroll
  for (int j = 0; j < kTileEPT; ++j) {
    const long long e = t0 + j * kT + tid;
    if (e < n) xr[e] = v[j];
    nacc = mad(v[j].x, v[j].x, nacc);
    nacc = mad(v[j].y, v[j].y, nacc);
  }
  const double2 sres = block_reduce(make_double2((double)nacc, 0.0), shn);
  if (tid == 0) npart[(long long)r * nb + blockIdx.x] = sres.x;
}

// Before the subtraction: ||x'||^2 = ||x||^2 - sum_i |h_i|^2 (x' = x - V h is the part
// of x orthogonal to the basis), flag[r] = 1 where ||x'|| < ||x|| / 16.  The test is
// that of Daniel, Gragg, Kaufman and Stewart with a looser threshold than their
// 1/sqrt(2): one projection leaves x' orthogonal to V up to about eps ||x|| / ||x'||,
// so below 1/16 cancellation the loss stays under ~16 eps per step: ~4e-15 in FP64,
// far below what restarted GMRES to 1e-7 can notice, and ~2e-6 in FP32, below the
// relative tolerance (>= 1e-4) of the inner solves that run in FP32.  The difference of
// squares is as accurate as the sums (FP64 ~1e-13, FP32 ~1e-6 of ||x||^2), i.e. at
// worst 256 times less relative to ||x'||^2.  For this operator the product A v_k is
// dominated by v_k, so 1/sqrt(2) would trigger the second projection in nearly every
// iteration, doubling the work.
__global__ void cgs_precheck_kernel(const double *__restrict__ npart0, const double2 *__restrict__ h,
                                    double *__restrict__ nrm, int *__restrict__ flag, int k1, int nb, int ldh) {
  __shared__ double2 sh[kT / 32];
  const int r = blockIdx.x;
  double a0 = 0.0, a1 = 0.0;
  for (int b = threadIdx.x; b < nb; b += kT) a0 += npart0[(long long)r * nb + b];
  for (int i = threadIdx.x; i < k1; i += kT) {
    const double2 v = h[(long long)r * ldh + i];
    a1 = fma(v.x, v.x, a1);
    a1 = fma(v.y, v.y, a1);
  }
  const double2 s = block_reduce(make_double2(a0, a1), sh);
  if (threadIdx.x == 0) {
    const double n0 = sqrt(s.x);
    const double d = s.x - s.y;
    const double n1 = d > 0.0 ? sqrt(d) : 0.0;
    nrm[r] = n1;
    flag[r] = n1 < 0.0625 * n0 ? 1 : 0;
  }
}

// after the second projection: nrm[r] = ||x''|| for the right-hand sides that had one
__global__ void cgs_renorm_kernel(const double *__restrict__ npart, double *__restrict__ nrm,
                                  const int *__restrict__ flag, int nb) {
  __shared__ double2 sh[kT / 32];
  const int r = blockIdx.x;
  if (!flag[r]) return;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += kT) acc += npart[(long long)r * nb + b];
  const double2 s = block_reduce(make_double2(acc, 0.0), sh);
  if (threadIdx.x == 0) nrm[r] = sqrt(s.x);
}

// out[r * ldh + i] = sum_b part[(r * k1 + i) * nb + b]; 0 where flag[r] == 0
__global__ void part_sum_kernel(const double2 *__restrict__ part, double2 *__restrict__ out,
                                const int *__restrict__ flag, int k1, int nb, int ldh) {
  __shared__ double2 sh[kT / 32];
  const int i = blockIdx.x, r = blockIdx.y;
  if (flag && !flag[r]) {
    if (threadIdx.x == 0) out[(long long)r * ldh + i] = make_double2(0.0, 0.0);
    return;
  }
  double2 acc = make_double2(0.0, 0.0);
  for (int b = threadIdx.x; b < nb; b += kT) {
    const double2 v = part[((long long)r * k1 + i) * nb + b];
    acc.x += v.x;
    acc.y += v.y;
  }
  const double2 t = block_reduce(acc, sh);
  if (threadIdx.x == 0) out[(long long)r * ldh + i] = t;
}

int cgs_nb(long long n) { return (int)((n + kTile - 1) / kTile); }

int blocks_for(long long n) {
  long long g = (n + kT - 1) / kT;
  if (g > 152LL * 32) g = 152LL * 32;
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

template <typename T>
int gmres_orthogonalize(const C<T> *V, C<T> *w, C<T> *vnext, double2 *h1, double2 *h2, double2 *part, double *npart,
                        double *nrm, int *flag, int k1, int R, long long n, int ldh, cudaStream_t s) {
  if (k1 < 1 || k1 > 64) return -1;
  const int nb = cgs_nb(n);
  double *np0 = npart, *np1 = npart + (long long)R * nb;
  const dim3 g(nb, R);
  count_launches(9);
  // first projection: h1 = V^H w and ||w||; ||w'|| from the difference of squares
  cgs_dot_kernel<T><<<g, kT, 0, s>>>(V, w, part, np0, nullptr, k1, R, n, nb);
  part_sum_kernel<<<dim3(k1, R), kT, 0, s>>>(part, h1, nullptr, k1, nb, ldh);
  cgs_precheck_kernel<<<R, kT, 0, s>>>(np0, h1, nrm, flag, k1, nb, ldh);
  // w' = w - V h1, written normalised into vnext where no second projection is needed
  cgs_sub_kernel<T><<<g, kT, 0, s>>>(V, w, h1, np1, nullptr, k1, R, n, nb, ldh, vnext, nrm, flag);
  // second projection where the first cancelled too much (h2 = 0 elsewhere)
  cgs_dot_kernel<T><<<g, kT, 0, s>>>(V, w, part, np0, flag, k1, R, n, nb);
  part_sum_kernel<<<dim3(k1, R), kT, 0, s>>>(part, h2, flag, k1, nb, ldh);
  cgs_sub_kernel<T><<<g, kT, 0, s>>>(V, w, h2, np1, flag, k1, R, n, nb, ldh, nullptr, nullptr, nullptr);
  cgs_renorm_kernel<<<R, kT, 0, s>>>(np1, nrm, flag, nb);
  scale_kernel<T><<<dim3(blocks_for(n), R), kT, 0, s>>>(w, vnext, nrm, n, flag);
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
// the new vector vanished (breakdown).
__global__ void givens_kernel(GivensState st, const double2 *h1, const double2 *h2, const double *nrm, int k, int R,
                              int m, int ldh) {
  const int r = threadIdx.x;
  __shared__ int cnt;
  if (r == 0) cnt = 0;
  __syncthreads();
  if (r < R && st.active[r]) {
    double2 *col = st.Rm + ((long long)r * m + k) * ldh;
    for (int i = 0; i <= k; ++i) {
      const double2 a = h1[(long long)r * ldh + i], b = h2[(long long)r * ldh + i];
      col[i] = make_double2(a.x + b.x, a.y + b.y);
    }
    const double hk1 = nrm[r];
    for (int i = 0; i < k; ++i) {
      const double ci = st.cs[(long long)r * m + i];
      const double2 si = st.sn[(long long)r * m + i];
      const double2 ai = col[i], bi = col[i + 1];
      const double2 t = make_double2(ci * ai.x + zmul(si, bi).x, ci * ai.y + zmul(si, bi).y);
      const double2 nb = zmul(zconj(si), ai);
      col[i + 1] = make_double2(-nb.x + ci * bi.x, -nb.y + ci * bi.y);
      col[i] = t;
    }
    const double2 a = col[k];
    const double aa = zabs(a);
    const double rho = hypot(aa, hk1);
    double ck;
    double2 sk;
    if (aa == 0.0) {
      ck = 0.0;
      sk = make_double2(1.0, 0.0);
    } else {
      ck = aa / rho;
      sk = make_double2(a.x / aa * hk1 / rho, a.y / aa * hk1 / rho);
    }
    col[k] = make_double2(ck * a.x + sk.x * hk1, ck * a.y + sk.y * hk1);
    st.cs[(long long)r * m + k] = ck;
    st.sn[(long long)r * m + k] = sk;
    double2 *gr = st.g + (long long)r * ldh;
    const double2 gk = gr[k];
    const double2 gn = zmul(zconj(sk), gk);
    gr[k + 1] = make_double2(-gn.x, -gn.y);
    gr[k] = make_double2(ck * gk.x, ck * gk.y);
    st.kr[r] = k + 1;
    int act = 1;
    if (hk1 == 0.0) {
      act = 0;
      st.brk[r] = 1;
    }
    if (zabs(gr[k + 1]) <= st.thr[r]) act = 0;
    st.active[r] = act;
  }
  __syncthreads();
  if (r < R && st.active[r]) atomicAdd(&cnt, 1);
  __syncthreads();
  if (r == 0) *st.n_active = cnt;
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

int gs_partial_blocks(long long n) { return cgs_nb(n); }

void givens_init(const GivensState &st, const double *nrm, int R, int ldh, cudaStream_t s) {
  count_launches(1);
  givens_init_kernel<<<1, 32, 0, s>>>(st, nrm, R, ldh);
}

void givens_step(const GivensState &st, const double2 *h1, const double2 *h2, const double *nrm, int k, int R, int m,
                 int ldh, cudaStream_t s) {
  count_launches(1);
  givens_kernel<<<1, 32, 0, s>>>(st, h1, h2, nrm, k, R, m, ldh);
}

void givens_solve(const GivensState &st, double2 *yd, int R, int m, int ldh, cudaStream_t s) {
  count_launches(1);
  backsub_kernel<<<1, 32, 0, s>>>(st, yd, R, m, ldh);
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
                                      double *, int *, int, int, long long, int, cudaStream_t);                     \
  template void gmres_scale<T>(const C<T> *, C<T> *, const double *, int, long long, cudaStream_t);                 \
  template void vec_sub<T>(const C<T> *, const C<T> *, C<T> *, long long, cudaStream_t);                           \
  template void vec_add<T>(const C<T> *, double2 *, long long, cudaStream_t);
IE_BLAS_INSTANTIATE(float)
IE_BLAS_INSTANTIATE(double)
#undef IE_BLAS_INSTANTIATE

}  // namespace ie
