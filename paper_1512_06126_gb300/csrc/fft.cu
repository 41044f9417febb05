// Batched FFT kernels: the strided-axis pass and the two row passes that also
// transpose between the vector layout [cz][y][x] and the wavenumber-major
// layout [y][kx][cz] (cz = rhs * 3Nz + component * Nz + z).
#include "fft.cuh"
#include "fft_fast.cuh"

#include <stdexcept>

namespace ie {

FftPlan make_plan(int L) {
  FftPlan p{};
  p.L = L;
  p.n_stages = 0;
  int n = L;
  auto push = [&](int r) {
    if (p.n_stages >= kMaxStages) throw std::runtime_error("FFT plan too long");
    p.radix[p.n_stages++] = r;
  };
  while (n % 4 == 0) { push(4); n /= 4; }
  while (n % 2 == 0) { push(2); n /= 2; }
  for (int f = 3; n > 1; f += 2) {
    while (n % f == 0) {
      if (f != 3 && f != 5 && f != 7 && f != 11 && f != 13)
        throw std::runtime_error("FFT length has a prime factor other than 2, 3, 5, 7, 11, 13");
      push(f);
      n /= f;
    }
  }
  return p;
}

std::vector<FftPlan> candidate_plans(int L) {
  std::vector<FftPlan> out;
  FftPlan base;
  try {
    base = make_plan(L);
  } catch (...) {
    return out;
  }
  int n2 = 0, rest = L;
  while (rest % 2 == 0) { ++n2; rest /= 2; }
  std::vector<int> odd;
  for (int st = 0; st < base.n_stages; ++st)
    if (base.radix[st] % 2) odd.push_back(base.radix[st]);
  auto build = [&](const std::vector<int> &r) {
    FftPlan p{};
    p.L = L;
    if ((int)r.size() > kMaxStages) return;
    for (int v : r) p.radix[p.n_stages++] = v;
    for (const FftPlan &q : out) {
      if (q.n_stages != p.n_stages) continue;
      bool same = true;
      for (int k = 0; k < p.n_stages; ++k) same = same && q.radix[k] == p.radix[k];
      if (same) return;
    }
    out.push_back(p);
  };
  auto pow2_stages = [&](int first8, bool two_first) {
    std::vector<int> r;
    int m = n2;
    if (two_first && m % 2 == 1) { r.push_back(2); --m; }
    if (first8) while (m >= 3) { r.push_back(8); m -= 3; }
    while (m >= 2) { r.push_back(4); m -= 2; }
    if (m == 1) r.push_back(2);
    return r;
  };
  {
    std::vector<int> r(base.radix, base.radix + base.n_stages);
    build(r);
  }
  {
    std::vector<int> r = pow2_stages(1, false);
    r.insert(r.end(), odd.begin(), odd.end());
    build(r);
  }
  {
    std::vector<int> r = odd, t = pow2_stages(0, false);
    r.insert(r.end(), t.begin(), t.end());
    build(r);
  }
  {
    std::vector<int> r = odd, t = pow2_stages(1, false);
    r.insert(r.end(), t.begin(), t.end());
    build(r);
  }
  {
    std::vector<int> r = pow2_stages(0, true);
    r.insert(r.end(), odd.begin(), odd.end());
    build(r);
  }
  return out;
}

namespace {

constexpr int kThreads = 256;

template <typename T, bool INV>
__global__ void __launch_bounds__(kThreads) fft_axis_kernel(const C<T> *__restrict__ in, C<T> *__restrict__ out,
                                                            int Lin, int Lout, long long inner, FftPlan plan,
                                                            T scale) {
  extern __shared__ unsigned char smem_raw[];
  constexpr int TI = fft_ti<T>();
  const int L = plan.L;
  C<T> *tw = reinterpret_cast<C<T> *>(smem_raw);
  C<T> *A = tw + L;
  C<T> *B = A + (size_t)L * TI;
  const int tid = threadIdx.x;
  const long long i0 = (long long)blockIdx.x * TI;
  const long long o = blockIdx.y;
  fill_twiddles<T>(tw, L, tid, kThreads);
  for (int q = tid; q < L * TI; q += kThreads) {
    const int l = q / TI, t = q % TI;
    C<T> v = mk<T>(0, 0);
    if (l < Lin && i0 + t < inner) v = in[(o * Lin + l) * inner + i0 + t];
    A[l * TI + t] = v;
  }
  __syncthreads();
  C<T> *res = fft_smem<T, INV>(A, B, TI, TI, tw, plan, tid, kThreads);
  for (int q = tid; q < Lout * TI; q += kThreads) {
    const int l = q / TI, t = q % TI;
    if (i0 + t < inner) out[(o * Lout + l) * inner + i0 + t] = cscale(res[l * TI + t], scale);
  }
}

// a value of the vectors' type TX in the transform's arithmetic T (FP64 -> FP32 from the
// bits, see d2f_bits)
template <typename T, typename TX>
__device__ __forceinline__ C<T> to_t(C<TX> v) {
  if constexpr (sizeof(T) == 4 && sizeof(TX) == 8) return to_f32(v);
  else return mk<T>((T)v.x, (T)v.y);
}
template <typename TX, typename T>
__device__ __forceinline__ C<TX> from_t(C<T> v) {
  if constexpr (sizeof(T) == 4 && sizeof(TX) == 8) return to_prec<double>(v);
  else return mk<TX>((TX)v.x, (TX)v.y);
}

// T: arithmetic type of the transform; TX: element type of the vectors and scales.
template <typename T, typename TX>
__global__ void __launch_bounds__(kThreads) fft_rows_fwd_kernel(const C<TX> *__restrict__ x,
                                                                const C<T> *__restrict__ in_scale,
                                                                C<T> *__restrict__ t1, int CZ, int Nz, int Ny,
                                                                int Nx, FftPlan plan) {
  extern __shared__ unsigned char smem_raw[];
  constexpr int TI = fft_ti<T>();
  constexpr int LD = TI + 1;
  const int L = plan.L;  // 2 Nx
  C<T> *tw = reinterpret_cast<C<T> *>(smem_raw);
  C<T> *A = tw + L;
  C<T> *B = A + (size_t)L * LD;
  const int tid = threadIdx.x;
  const int cz0 = blockIdx.x * TI;
  const int y = blockIdx.y;
  fill_twiddles<T>(tw, L, tid, kThreads);
  for (int q = tid; q < Nx * TI; q += kThreads) {
    const int t = q / Nx, xx = q % Nx;
    const int cz = cz0 + t;
    C<T> v = mk<T>(0, 0);
    if (cz < CZ) {
      v = to_t<T, TX>(x[((long long)cz * Ny + y) * Nx + xx]);
      if (in_scale) v = cmul(v, in_scale[((long long)(cz % Nz) * Ny + y) * Nx + xx]);
    }
    A[xx * LD + t] = v;
  }
  for (int q = tid; q < (L - Nx) * TI; q += kThreads) {
    const int l = Nx + q / TI, t = q % TI;
    A[l * LD + t] = mk<T>(0, 0);
  }
  __syncthreads();
  C<T> *res = fft_smem<T, false>(A, B, LD, TI, tw, plan, tid, kThreads);
  for (int q = tid; q < L * TI; q += kThreads) {
    const int kx = q / TI, t = q % TI;
    if (cz0 + t < CZ) t1[((long long)y * L + kx) * CZ + cz0 + t] = res[kx * LD + t];
  }
}

template <typename T, typename TX>
__global__ void __launch_bounds__(kThreads) fft_rows_inv_kernel(const C<T> *__restrict__ t1,
                                                                const C<TX> *__restrict__ x,
                                                                const C<T> *__restrict__ diag,
                                                                const C<T> *__restrict__ out_scale,
                                                                C<TX> *__restrict__ y_out, int CZ, int Nz, int Ny,
                                                                int Nx, FftPlan plan) {
  extern __shared__ unsigned char smem_raw[];
  constexpr int TI = fft_ti<T>();
  constexpr int LD = TI + 1;
  const int L = plan.L;
  C<T> *tw = reinterpret_cast<C<T> *>(smem_raw);
  C<T> *A = tw + L;
  C<T> *B = A + (size_t)L * LD;
  const int tid = threadIdx.x;
  const int cz0 = blockIdx.x * TI;
  const int y = blockIdx.y;
  fill_twiddles<T>(tw, L, tid, kThreads);
  for (int q = tid; q < L * TI; q += kThreads) {
    const int kx = q / TI, t = q % TI;
    C<T> v = mk<T>(0, 0);
    if (cz0 + t < CZ) v = t1[((long long)y * L + kx) * CZ + cz0 + t];
    A[kx * LD + t] = v;
  }
  __syncthreads();
  C<T> *res = fft_smem<T, true>(A, B, LD, TI, tw, plan, tid, kThreads);
  for (int q = tid; q < Nx * TI; q += kThreads) {
    const int t = q / Nx, xx = q % Nx;
    const int cz = cz0 + t;
    if (cz < CZ) {
      const long long cell = ((long long)(cz % Nz) * Ny + y) * Nx + xx;
      const long long gi = ((long long)cz * Ny + y) * Nx + xx;
      C<T> v = cmul(res[xx * LD + t], out_scale[cell]);
      if (diag) cfma(v, diag[cell], to_t<T, TX>(x[gi]));
      y_out[gi] = from_t<TX, T>(v);
    }
  }
}

template <typename T> size_t axis_smem(int L) { return sizeof(C<T>) * ((size_t)L + 2 * (size_t)L * fft_ti<T>()); }
template <typename T> size_t rows_smem(int L) {
  return sizeof(C<T>) * ((size_t)L + 2 * (size_t)L * (fft_ti<T>() + 1));
}

template <typename K> void set_smem(K kern, size_t bytes) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Register-blocked FP32 kernels for L = 16 Q, Q in {8, 12, 16, 24, 32} (0: not applicable).
int fast_q(int L) { return (L == 128 || L == 192 || L == 256 || L == 384 || L == 512) ? L / 16 : 0; }

#define IE_FAST_Q_DISPATCH(q, CALL) \
  switch (q) {                      \
    case 8: CALL(8); break;         \
    case 12: CALL(12); break;       \
    case 16: CALL(16); break;       \
    case 24: CALL(24); break;       \
    default: CALL(32); break;       \
  }

template <int Q, bool INV>
void axis_fast(const float2 *in, float2 *out, int outer, int Lin, int Lout, long long inner, float scale,
               cudaStream_t s) {
  constexpr int L = 16 * Q;
  const bool half = INV ? (Lin == L && 2 * Lout == L) : (2 * Lin == L && Lout == L);
  auto k = half ? fftfast::axis_kernel<Q, INV, true> : fftfast::axis_kernel<Q, INV, false>;
  set_smem(k, fftfast::smem_bytes(Q));
  dim3 grid((unsigned)((inner + fftfast::kTI - 1) / fftfast::kTI), (unsigned)outer);
  k<<<grid, fftfast::threads(Q), fftfast::smem_bytes(Q), s>>>(in, out, Lin, Lout, inner, scale);
}

template <int Q, typename TX>
void rows_fwd_fast(const C<TX> *x, const float2 *in_scale, float2 *t1, int CZ, int Nz, int Ny, int Nx,
                   cudaStream_t s) {
  auto k = fftfast::rows_fwd_kernel<Q, TX>;
  set_smem(k, fftfast::smem_bytes(Q));
  dim3 grid((unsigned)((CZ + fftfast::kTI - 1) / fftfast::kTI), (unsigned)Ny);
  k<<<grid, fftfast::threads(Q), fftfast::smem_bytes(Q), s>>>(x, in_scale, t1, CZ, Nz, Ny, Nx);
}

template <int Q, typename TX>
void rows_inv_fast(const float2 *t1, const C<TX> *x, const float2 *diag, const float2 *out_scale, C<TX> *y, int CZ,
                   int Nz, int Ny, int Nx, cudaStream_t s) {
  auto k = fftfast::rows_inv_kernel<Q, TX>;
  set_smem(k, fftfast::smem_bytes(Q));
  dim3 grid((unsigned)((CZ + fftfast::kTI - 1) / fftfast::kTI), (unsigned)Ny);
  k<<<grid, fftfast::threads(Q), fftfast::smem_bytes(Q), s>>>(t1, x, diag, out_scale, y, CZ, Nz, Ny, Nx);
}

}  // namespace

template <typename T, bool INV>
void launch_fft_axis(const C<T> *in, C<T> *out, int outer, int Lin, int Lout, long long inner,
                     const FftPlan &plan, T scale, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    const int q = fast_q(plan.L);
    if (q) {
      count_launches(1);
#define IE_CALL(Q) axis_fast<Q, INV>(in, out, outer, Lin, Lout, inner, scale, s)
      IE_FAST_Q_DISPATCH(q, IE_CALL)
#undef IE_CALL
      return;
    }
  }
  constexpr int TI = fft_ti<T>();
  const size_t sm = axis_smem<T>(plan.L);
  auto k = fft_axis_kernel<T, INV>;
  set_smem(k, sm);
  dim3 grid((unsigned)((inner + TI - 1) / TI), (unsigned)outer);
  count_launches(1);
  k<<<grid, kThreads, sm, s>>>(in, out, Lin, Lout, inner, plan, scale);
}

template <typename T, typename TX>
void launch_fft_rows_fwd(const C<TX> *x, const C<T> *in_scale, C<T> *t1, int CZ, int Nz, int Ny, int Nx,
                         const FftPlan &plan, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    const int q = fast_q(plan.L);
    if (q && plan.L == 2 * Nx) {
      count_launches(1);
#define IE_CALL(Q) rows_fwd_fast<Q, TX>(x, in_scale, t1, CZ, Nz, Ny, Nx, s)
      IE_FAST_Q_DISPATCH(q, IE_CALL)
#undef IE_CALL
      return;
    }
  }
  constexpr int TI = fft_ti<T>();
  const size_t sm = rows_smem<T>(plan.L);
  auto k = fft_rows_fwd_kernel<T, TX>;
  set_smem(k, sm);
  dim3 grid((unsigned)((CZ + TI - 1) / TI), (unsigned)Ny);
  count_launches(1);
  k<<<grid, kThreads, sm, s>>>(x, in_scale, t1, CZ, Nz, Ny, Nx, plan);
}

template <typename T, typename TX>
void launch_fft_rows_inv(const C<T> *t1, const C<TX> *x, const C<T> *diag, const C<T> *out_scale, C<TX> *y,
                         int CZ, int Nz, int Ny, int Nx, const FftPlan &plan, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    const int q = fast_q(plan.L);
    if (q && plan.L == 2 * Nx) {
      count_launches(1);
#define IE_CALL(Q) rows_inv_fast<Q, TX>(t1, x, diag, out_scale, y, CZ, Nz, Ny, Nx, s)
      IE_FAST_Q_DISPATCH(q, IE_CALL)
#undef IE_CALL
      return;
    }
  }
  constexpr int TI = fft_ti<T>();
  const size_t sm = rows_smem<T>(plan.L);
  auto k = fft_rows_inv_kernel<T, TX>;
  set_smem(k, sm);
  dim3 grid((unsigned)((CZ + TI - 1) / TI), (unsigned)Ny);
  count_launches(1);
  k<<<grid, kThreads, sm, s>>>(t1, x, diag, out_scale, y, CZ, Nz, Ny, Nx, plan);
}

template void launch_fft_axis<float, false>(const float2 *, float2 *, int, int, int, long long, const FftPlan &,
                                            float, cudaStream_t);
template void launch_fft_axis<float, true>(const float2 *, float2 *, int, int, int, long long, const FftPlan &,
                                           float, cudaStream_t);
template void launch_fft_axis<double, false>(const double2 *, double2 *, int, int, int, long long,
                                             const FftPlan &, double, cudaStream_t);
template void launch_fft_axis<double, true>(const double2 *, double2 *, int, int, int, long long, const FftPlan &,
                                            double, cudaStream_t);
template void launch_fft_rows_fwd<float, float>(const float2 *, const float2 *, float2 *, int, int, int, int,
                                                const FftPlan &, cudaStream_t);
template void launch_fft_rows_fwd<double, double>(const double2 *, const double2 *, double2 *, int, int, int, int,
                                                  const FftPlan &, cudaStream_t);
template void launch_fft_rows_fwd<float, double>(const double2 *, const float2 *, float2 *, int, int, int, int,
                                                 const FftPlan &, cudaStream_t);
template void launch_fft_rows_inv<float, float>(const float2 *, const float2 *, const float2 *, const float2 *,
                                                float2 *, int, int, int, int, const FftPlan &, cudaStream_t);
template void launch_fft_rows_inv<double, double>(const double2 *, const double2 *, const double2 *,
                                                  const double2 *, double2 *, int, int, int, int, const FftPlan &,
                                                  cudaStream_t);
template void launch_fft_rows_inv<float, double>(const float2 *, const double2 *, const float2 *, const float2 *,
                                                 double2 *, int, int, int, int, const FftPlan &, cudaStream_t);

}  // namespace ie
