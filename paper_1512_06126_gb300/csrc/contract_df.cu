// The wavenumber contraction (step 2 of the FFT product, Sect. 3.3) for c128 vectors in
// compensated double-float arithmetic on the FP32 pipe, for the residuals of the
// mixed-precision refinement.
//
// Every FP64 number x is carried as hi + lo, hi = fl32(x), lo = fl32(x - hi) (about 48
// significant bits).  Each row of Y = M X is a dot product accumulated as in the
// compensated dot product of Ogita, Rump and Oishi (Dot2): the rounding error of every
// product (TwoProduct, exact with an FMA) and of every addition (TwoSum) goes into a
// second FP32 accumulator, the cross terms hi lo are added to it and lo lo is dropped
// (~2^-48 of the product).  The result, s + c as an FP64 sum, is as accurate as a dot
// product computed in twice FP32 precision: an error of about (3 Nz eps32)^2 of the sum
// of the magnitudes of the terms, far below what a refinement residual at a tolerance
// of 1e-7 can notice.  The FP32 operations are explicitly rounded (__fmul_rn, __fadd_rn,
// ...) so that the compiler forms no FMAs that would break the error terms.
//
// One CTA per folded wavenumber; the mirror vectors (with the component signs of
// Lemma 2) are staged in shared memory as double-float, the packed block (Lemma 1)
// streams through a panel of double-float entries; thread (row, column group) owns
// one output row and CPT columns.
#include "contract.cuh"

namespace ie {
namespace {

constexpr int kCpt = 4;  // columns per thread

// value s + c
struct Acc {
  float s, c;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
}

// acc += (ah + al) (bh + bl)
__device__ __forceinline__ void acc_fma(Acc &acc, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float pe = __fmaf_rn(ah, bh, -p);
  pe = __fmaf_rn(ah, bl, pe);
  pe = __fmaf_rn(al, bh, pe);
  float s, e;
  two_sum(acc.s, p, s, e);
  acc.s = s;
  acc.c = __fadd_rn(acc.c, __fadd_rn(e, pe));
}

__device__ __forceinline__ float4 split_df(double2 v) {
  const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
  return make_float4(rh, __double2float_rn(v.x - (double)rh), ih, __double2float_rn(v.y - (double)ih));
}

__device__ __forceinline__ float4 neg4(float4 v) { return make_float4(-v.x, -v.y, -v.z, -v.w); }

// Element (row, col) of the 3 Nz x 3 Nz block from its packed double-float storage
// (Lemma 1: xx, yy, zz, xy symmetric, zx = -xz^T, zy = -yz^T).
__device__ __forceinline__ float4 entry_df(const float4 *__restrict__ q, int Nz, int P, int row, int col) {
  const int alpha = row / Nz, a = row - alpha * Nz;
  const int beta = col / Nz, b = col - beta * Nz;
  const bool full = (alpha == 2) != (beta == 2);
  if (!full) {
    const int kind = alpha == beta ? alpha : 3;
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return q[(size_t)kind * P + lo * Nz - lo * (lo - 1) / 2 + (hi - lo)];
  }
  if (beta == 2) return q[4 * (size_t)P + (size_t)alpha * Nz * Nz + a * Nz + b];
  return neg4(q[4 * (size_t)P + (size_t)beta * Nz * Nz + b * Nz + a]);
}

__global__ void split_df_kernel(const double2 *__restrict__ q, float4 *__restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = split_df(q[i]);
}

template <int MAXC>
__global__ void contract_df_kernel(double2 *__restrict__ spec, const float4 *__restrict__ qf, int Nx, int Ny, int Nz,
                                   int R, int PW, int ldz) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n3 = 3 * Nz;
  float4 *X = reinterpret_cast<float4 *>(smem_raw);  // [MAXC][3 Nz]
  float4 *pan = X + (size_t)MAXC * n3;                // [3 Nz][PW + 1]
  const int ldp = PW + 1;
  const int kxb = blockIdx.x, kyb = blockIdx.y;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int P = Nz * (Nz + 1) / 2;
  const long long BS = 2LL * Nz * (2 * Nz + 1);
  const float4 *q = qf + ((long long)kyb * (Nx + 1) + kxb) * BS;
  const int nmx = (kxb > 0 && kxb < Nx) ? 2 : 1, nmy = (kyb > 0 && kyb < Ny) ? 2 : 1;
  const int kx1 = 2 * Nx - kxb, ky1 = 2 * Ny - kyb;
  const int ncol = nmx * nmy * R;
  for (int e = tid; e < MAXC * n3; e += nthr) {
    const int col = e / n3, row = e - col * n3;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (col < ncol) {
      const int m = col / R, r = col - m * R;
      const int mx = m % nmx, my = m / nmx;
      const int comp = row / Nz;
      v = split_df(spec[((long long)(my ? ky1 : kyb) * 2 * Nx + (mx ? kx1 : kxb)) * ldz + r * n3 + row]);
      if ((comp == 0 && mx == 1) || (comp == 1 && my == 1)) v = neg4(v);
    }
    X[col * n3 + row] = v;
  }
  const int row = tid % n3, cg = tid / n3;  // blockDim = 3 Nz x (MAXC / kCpt)
  Acc ar[kCpt], ai[kCpt];
#pragma unroll
  for (int c = 0; c < kCpt; ++c) ar[c] = ai[c] = Acc{0.f, 0.f};
  for (int c0 = 0; c0 < n3; c0 += PW) {
    const int w = n3 - c0 < PW ? n3 - c0 : PW;
    __syncthreads();  // previous panel consumed (first pass: X staged)
    for (int e = tid; e < n3 * w; e += nthr) {
      const int rr = e / w, j = e - rr * w;
      pan[rr * ldp + j] = entry_df(q, Nz, P, rr, c0 + j);
    }
    __syncthreads();
    if (cg * kCpt < ncol) {
      const float4 *mrow = pan + (size_t)row * ldp;
      for (int j = 0; j < w; ++j) {
        const float4 m = mrow[j];  // (re hi, re lo, im hi, im lo)
        const float4 *xb = X + (size_t)(cg * kCpt) * n3 + c0 + j;
#pragma unroll
        for (int c = 0; c < kCpt; ++c) {
          const float4 x = xb[c * n3];
          // (mr + i mi)(xr + i xi): re = mr xr - mi xi, im = mr xi + mi xr
          acc_fma(ar[c], m.x, m.y, x.x, x.y);
          acc_fma(ar[c], -m.z, -m.w, x.z, x.w);
          acc_fma(ai[c], m.x, m.y, x.z, x.w);
          acc_fma(ai[c], m.z, m.w, x.x, x.y);
        }
      }
    }
  }
  const int alpha = row / Nz;
#pragma unroll
  for (int c = 0; c < kCpt; ++c) {
    const int col = cg * kCpt + c;
    if (col < ncol) {
      const int mm = col / R, r = col - mm * R;
      const int mx = mm % nmx, my = mm / nmx;
      double2 v = make_double2((double)ar[c].s + (double)ar[c].c, (double)ai[c].s + (double)ai[c].c);
      if ((alpha == 0 && mx == 1) || (alpha == 1 && my == 1)) { v.x = -v.x; v.y = -v.y; }
      spec[((long long)(my ? ky1 : kyb) * 2 * Nx + (mx ? kx1 : kxb)) * ldz + r * n3 + row] = v;
    }
  }
}

template <int MAXC>
int launch_df(double2 *spec, const float4 *qf, int Nx, int Ny, int Nz, int R, int ldz, cudaStream_t s) {
  const int n3 = 3 * Nz;
  const int threads = n3 * (MAXC / kCpt);
  if (threads > 1024) return -1;
  const size_t xb = sizeof(float4) * (size_t)MAXC * n3;
  constexpr size_t kMax = 227 * 1024;
  // widest panel that leaves room for three CTAs per SM, else the narrowest that fits
  int PW = 8;
  for (int cand : {64, 32, 16, 8}) {
    if (cand > n3) continue;
    if (xb + sizeof(float4) * (size_t)n3 * (cand + 1) <= kMax / 3) { PW = cand; break; }
  }
  const size_t sm = xb + sizeof(float4) * (size_t)n3 * (PW + 1);
  if (sm > kMax) return -1;
  auto k = contract_df_kernel<MAXC>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  count_launches(1);
  k<<<dim3(Nx + 1, Ny + 1), threads, sm, s>>>(spec, qf, Nx, Ny, Nz, R, PW, ldz);
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return 0;
}

}  // namespace

void launch_split_df(const double2 *q64, float4 *qdf, long long count, cudaStream_t s) {
  long long g = (count + 255) / 256;
  if (g > 152LL * 16) g = 152LL * 16;
  count_launches(1);
  split_df_kernel<<<(int)(g < 1 ? 1 : g), 256, 0, s>>>(q64, qdf, count);
}

int launch_contract_df(double2 *spec, const float4 *qdf, int Nx, int Ny, int Nz, int R, int ldz, cudaStream_t s) {
  if (R < 1 || ldz < R * 3 * Nz) return -1;
  if (R == 1) return launch_df<4>(spec, qdf, Nx, Ny, Nz, R, ldz, s);
  if (R == 2) return launch_df<8>(spec, qdf, Nx, Ny, Nz, R, ldz, s);
  if (R <= 4) return launch_df<16>(spec, qdf, Nx, Ny, Nz, R, ldz, s);
  return -1;
}

}  // namespace ie
