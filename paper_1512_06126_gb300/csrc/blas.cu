// FP64 Krylov kernels for restarted GMRES with classical Gram-Schmidt applied
// twice (the orthogonalisation of FGMRES, Sect. 3.3 (ii) of the paper).  All
// right-hand sides advance in lockstep; each has its own Krylov space.
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

// part[(r * k1 + i) * nb + blk] = sum over the block's chunk of conj(V_i) * w
__global__ void __launch_bounds__(kT) mdot_partial(const double2 *__restrict__ V, const double2 *__restrict__ w,
                                                   double2 *__restrict__ part, int k1, int R, long long n, int nb) {
  __shared__ double2 sh[kT / 32];
  const int r = blockIdx.y;
  const long long base = (long long)blockIdx.x * kChunk;
  double2 wl[kEPT];
#pragma unroll
  for (int e = 0; e < kEPT; ++e) {
    const long long idx = base + e * kT + threadIdx.x;
    wl[e] = idx < n ? w[(long long)r * n + idx] : make_double2(0.0, 0.0);
  }
  for (int i = 0; i < k1; ++i) {
    const double2 *vi = V + ((long long)i * R + r) * n;
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll
    for (int e = 0; e < kEPT; ++e) {
      const long long idx = base + e * kT + threadIdx.x;
      if (idx < n) {
        const double2 a = vi[idx];
        acc.x = fma(a.x, wl[e].x, acc.x);
        acc.x = fma(a.y, wl[e].y, acc.x);
        acc.y = fma(a.x, wl[e].y, acc.y);
        acc.y = fma(-a.y, wl[e].x, acc.y);
      }
    }
    const double2 s = block_reduce(acc, sh);
    if (threadIdx.x == 0) part[((long long)r * k1 + i) * nb + blockIdx.x] = s;
  }
}

// out[r * ldh + i] (+)= sum_b part[(r * k1 + i) * nb + b]
__global__ void mdot_final(const double2 *__restrict__ part, double2 *__restrict__ out, int k1, int nb, int ldh,
                           int accumulate) {
  __shared__ double2 sh[kT / 32];
  const int i = blockIdx.x, r = blockIdx.y;
  double2 acc = make_double2(0.0, 0.0);
  for (int b = threadIdx.x; b < nb; b += kT) {
    const double2 v = part[((long long)r * k1 + i) * nb + b];
    acc.x += v.x;
    acc.y += v.y;
  }
  const double2 s = block_reduce(acc, sh);
  if (threadIdx.x == 0) {
    double2 *o = out + (long long)r * ldh + i;
    if (accumulate) { o->x += s.x; o->y += s.y; }
    else *o = s;
  }
}

// w[r] -= sum_{i<k1} h[r * ldh + i] * V_i[r]   (sign = -1), or x[r] += ... (sign = +1)
__global__ void maxpy_kernel(const double2 *__restrict__ V, const double2 *__restrict__ h, double2 *__restrict__ w,
                             int k1, int R, long long n, int ldh, double sign) {
  const int r = blockIdx.y;
  const double2 *hr = h + (long long)r * ldh;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    for (int i = 0; i < k1; ++i) {
      const double2 a = V[((long long)i * R + r) * n + idx];
      const double2 c = hr[i];
      acc.x = fma(c.x, a.x, acc.x);
      acc.x = fma(-c.y, a.y, acc.x);
      acc.y = fma(c.x, a.y, acc.y);
      acc.y = fma(c.y, a.x, acc.y);
    }
    double2 v = w[(long long)r * n + idx];
    v.x += sign * acc.x;
    v.y += sign * acc.y;
    w[(long long)r * n + idx] = v;
  }
}

__global__ void __launch_bounds__(kT) norm_partial(const double2 *__restrict__ w, double *__restrict__ part,
                                                   long long n, int nb) {
  __shared__ double2 sh[kT / 32];
  const int r = blockIdx.y;
  double acc = 0.0;
  for (long long idx = blockIdx.x * (long long)kT + threadIdx.x; idx < n; idx += (long long)nb * kT) {
    const double2 v = w[(long long)r * n + idx];
    acc = fma(v.x, v.x, acc);
    acc = fma(v.y, v.y, acc);
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
__global__ void scale_kernel(const double2 *__restrict__ src, double2 *__restrict__ dst, const double *__restrict__ nrm,
                             long long n) {
  const int r = blockIdx.y;
  const double s = nrm[r] > 0.0 ? 1.0 / nrm[r] : 0.0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    double2 v = src[(long long)r * n + idx];
    dst[(long long)r * n + idx] = make_double2(v.x * s, v.y * s);
  }
}

// out = a - b
__global__ void sub_kernel(const double2 *__restrict__ a, const double2 *__restrict__ b, double2 *__restrict__ out,
                           long long n) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const double2 u = a[idx], v = b[idx];
    out[idx] = make_double2(u.x - v.x, u.y - v.y);
  }
}

// y += x
__global__ void add_kernel(const double2 *__restrict__ x, double2 *__restrict__ y, long long n) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const double2 u = x[idx];
    double2 v = y[idx];
    v.x += u.x;
    v.y += u.y;
    y[idx] = v;
  }
}

// ---------------------------------------------------------------------------
// Classical Gram-Schmidt passes, tiled over the vector length.  A block owns a tile
// of kTile consecutive elements of one right-hand side:
//   MODE 0 (dot):       part_i = sum_tile conj(V_i) w
//   MODE 1 (sub + dot): w -= sum_i h_i V_i on the tile, then part_i = sum conj(V_i) w
//   MODE 2 (sub + norm): w -= sum_i h_i V_i on the tile, then part = sum |w|^2
// The tile of w sits in shared memory; for the dots, (basis vector, 256-element
// chunk) work units are spread over the warps, each lane streaming 8 elements, so a
// block keeps many independent loads in flight with few registers.
// ---------------------------------------------------------------------------
constexpr int kTileEPT = 8;
constexpr int kTile = kT * kTileEPT;  // 2048 elements
constexpr int kChunk256 = 256;

template <int MODE>
__global__ void __launch_bounds__(kT) cgs_tile_kernel(const double2 *__restrict__ V, double2 *__restrict__ w,
                                                      const double2 *__restrict__ h, double2 *__restrict__ part,
                                                      double *__restrict__ npart, int k1, int R, long long n, int nb,
                                                      int ldh) {
  __shared__ double2 xw[kTile];
  __shared__ double red[2 * 64];
  __shared__ double2 hs[64];
  __shared__ double2 shn[kT / 32];
  const int r = blockIdx.y;
  const long long t0 = (long long)blockIdx.x * kTile;
  const long long Rn = (long long)R * n;
  const int tid = threadIdx.x;
  const double2 *Vr = V + (long long)r * n;
  double2 *wr = w + (long long)r * n;
  if (tid < 2 * 64) red[tid] = 0.0;
  if (MODE != 0 && tid < k1) hs[tid] = h[(long long)r * ldh + tid];
  __syncthreads();
  double nacc = 0.0;
  if (MODE == 0) {
#pragma unroll
    for (int j = 0; j < kTileEPT; ++j) {
      const long long e = t0 + j * kT + tid;
      xw[j * kT + tid] = e < n ? wr[e] : make_double2(0.0, 0.0);
    }
  } else {
    double2 x[kTileEPT];
#pragma unroll
    for (int j = 0; j < kTileEPT; ++j) {
      const long long e = t0 + j * kT + tid;
      x[j] = e < n ? wr[e] : make_double2(0.0, 0.0);
    }
    for (int i = 0; i < k1; ++i) {
      const double2 hv = hs[i];
      const double2 *vi = Vr + (long long)i * Rn;
#pragma unroll
      for (int j = 0; j < kTileEPT; ++j) {
        const long long e = t0 + j * kT + tid;
        if (e < n) {
          const double2 a = __ldg(vi + e);
          x[j].x -= hv.x * a.x - hv.y * a.y;
          x[j].y -= hv.x * a.y + hv.y * a.x;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kTileEPT; ++j) {
      const long long e = t0 + j * kT + tid;
      if (e < n) wr[e] = x[j];
      xw[j * kT + tid] = x[j];
      nacc = fma(x[j].x, x[j].x, nacc);
      nacc = fma(x[j].y, x[j].y, nacc);
    }
  }
  if (MODE == 2) {
    const double2 sres = block_reduce(make_double2(nacc, 0.0), shn);
    if (tid == 0) npart[(long long)r * nb + blockIdx.x] = sres.x;
    return;
  }
  __syncthreads();
  const int lane = tid & 31, wid = tid >> 5;
  const int units = k1 * (kTile / kChunk256);
  for (int u = wid; u < units; u += kT / 32) {
    const int i = u / (kTile / kChunk256), c = u % (kTile / kChunk256);
    const double2 *vi = Vr + (long long)i * Rn;
    double ax = 0.0, ay = 0.0;
#pragma unroll
    for (int q = 0; q < kChunk256 / 32; ++q) {
      const int le = c * kChunk256 + q * 32 + lane;
      const long long e = t0 + le;
      if (e < n) {
        const double2 a = __ldg(vi + e);
        const double2 b = xw[le];
        ax = fma(a.x, b.x, ax);
        ax = fma(a.y, b.y, ax);
        ay = fma(a.x, b.y, ay);
        ay = fma(-a.y, b.x, ay);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ax += __shfl_down_sync(0xffffffffu, ax, o);
      ay += __shfl_down_sync(0xffffffffu, ay, o);
    }
    if (lane == 0) {
      atomicAdd(&red[2 * i], ax);
      atomicAdd(&red[2 * i + 1], ay);
    }
  }
  __syncthreads();
  if (tid < k1) part[((long long)r * k1 + tid) * nb + blockIdx.x] = make_double2(red[2 * tid], red[2 * tid + 1]);
}

// out[r * ldh + i] = sum_b part[(r * k1 + i) * nb + b]
__global__ void part_sum_kernel(const double2 *__restrict__ part, double2 *__restrict__ out, int k1, int nb,
                                int ldh) {
  __shared__ double2 sh[kT / 32];
  const int i = blockIdx.x, r = blockIdx.y;
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

void gmres_mdot(const double2 *V, const double2 *w, double2 *part, double2 *h_out, int k1, int R, long long n, int ldh,
                int accumulate, cudaStream_t s) {
  const int nb = mdot_nb(n);
  count_launches(2);
  mdot_partial<<<dim3(nb, R), kT, 0, s>>>(V, w, part, k1, R, n, nb);
  mdot_final<<<dim3(k1, R), kT, 0, s>>>(part, h_out, k1, nb, ldh, accumulate);
}

void gmres_maxpy(const double2 *V, const double2 *h, double2 *w, int k1, int R, long long n, int ldh, double sign,
                 cudaStream_t s) {
  count_launches(1);
  maxpy_kernel<<<dim3(blocks_for(n), R), kT, 0, s>>>(V, h, w, k1, R, n, ldh, sign);
}

void gmres_norm(const double2 *w, double *part, double *out, int R, long long n, cudaStream_t s) {
  int nb = mdot_nb(n);
  if (nb > 1024) nb = 1024;
  count_launches(2);
  norm_partial<<<dim3(nb, R), kT, 0, s>>>(w, part, n, nb);
  norm_final<<<R, kT, 0, s>>>(part, out, nb);
}

int gmres_cgs2(const double2 *V, double2 *w, double2 *h1, double2 *h2, double2 *part, double *npart, double *nrm,
               int k1, int R, long long n, int ldh, cudaStream_t s) {
  if (k1 < 1 || k1 > 64) return -1;
  const int nb = cgs_nb(n);
  count_launches(6);
  cgs_tile_kernel<0><<<dim3(nb, R), kT, 0, s>>>(V, w, nullptr, part, nullptr, k1, R, n, nb, ldh);
  part_sum_kernel<<<dim3(k1, R), kT, 0, s>>>(part, h1, k1, nb, ldh);
  cgs_tile_kernel<1><<<dim3(nb, R), kT, 0, s>>>(V, w, h1, part, nullptr, k1, R, n, nb, ldh);
  part_sum_kernel<<<dim3(k1, R), kT, 0, s>>>(part, h2, k1, nb, ldh);
  cgs_tile_kernel<2><<<dim3(nb, R), kT, 0, s>>>(V, w, h2, nullptr, npart, k1, R, n, nb, ldh);
  norm_final<<<R, kT, 0, s>>>(npart, nrm, nb);
  return 0;
}

int cgs2_partial_blocks(long long n) { return cgs_nb(n); }

void gmres_scale(const double2 *src, double2 *dst, const double *nrm, int R, long long n, cudaStream_t s) {
  count_launches(1);
  scale_kernel<<<dim3(blocks_for(n), R), kT, 0, s>>>(src, dst, nrm, n);
}

void vec_sub(const double2 *a, const double2 *b, double2 *out, long long n, cudaStream_t s) {
  count_launches(1);
  sub_kernel<<<blocks_for(n), kT, 0, s>>>(a, b, out, n);
}

void vec_add(const double2 *x, double2 *y, long long n, cudaStream_t s) {
  count_launches(1);
  add_kernel<<<blocks_for(n), kT, 0, s>>>(x, y, n);
}

}  // namespace ie
