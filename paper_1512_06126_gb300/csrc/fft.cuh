// Batched mixed-radix Stockham FFTs staged in shared memory.
//
// Step 1 and step 3 of the FFT matrix-vector product (Sect. 3.3 of the paper):
// forward 2-D FFTs of the zero-padded (2Nx x 2Ny) layers and their inverses.  Every
// kernel transforms TI independent sequences at once, held in shared memory as
// [l][ti] (ti contiguous), so that global loads and stores move whole 128-byte
// rows and butterflies touch consecutive shared-memory words.
#pragma once
#include <vector>

#include "ie_common.cuh"

namespace ie {

// Host: factor L into radices 4, 2, 3, 5 and any remaining prime factors.
FftPlan make_plan(int L);
// Host: the distinct stage orders the plan autotuner times for length L: the default
// (4s, a 2, odd factors), radix-8 stages first, the odd factors first, a radix-2 stage
// first (empty if L has a prime factor above 13).
std::vector<FftPlan> candidate_plans(int L);

// Number of transforms per CTA for element type T (one 128-byte row of them).
template <typename T> __host__ __device__ constexpr int fft_ti() { return 128 / (int)sizeof(C<T>); }

// Twiddle table tw[l] = exp(-2 pi i l / L) for l < L (forward sign).
template <typename T>
__device__ __forceinline__ void fill_twiddles(C<T> *tw, int L, int tid, int nthr) {
  for (int l = tid; l < L; l += nthr) {
    T s, c;
    if constexpr (sizeof(T) == 4) {
      sincospif(2.0f * (float)l / (float)L, &s, &c);
    } else {
      sincospi(2.0 * (double)l / (double)L, &s, &c);
    }
    tw[l] = mk<T>(c, -s);
  }
}

template <typename T, bool INV>
__device__ __forceinline__ C<T> twid(const C<T> *tw, int idx) {
  C<T> w = tw[idx];
  if (INV) w.y = -w.y;
  return w;
}

template <typename T, bool INV>
__device__ __forceinline__ void dft4(C<T> &a0, C<T> &a1, C<T> &a2, C<T> &a3) {
  C<T> t0 = cadd(a0, a2), t1 = csub(a0, a2);
  C<T> t2 = cadd(a1, a3), d = csub(a1, a3);
  // forward: -i * d ; inverse: +i * d
  C<T> t3 = INV ? mk<T>(-d.y, d.x) : mk<T>(d.y, -d.x);
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

// In-register DFT of compile-time radix R (2, 4 and 8 closed form, others by the direct
// sum with the length-L twiddle table).
template <typename T, bool INV, int R>
__device__ __forceinline__ void dft_small(C<T> (&v)[R], const C<T> *tw, int L) {
  if constexpr (R == 8) {
    // even and odd halves by 4-point DFTs, then X[k] = E[k] + w_8^k O[k], X[k + 4] =
    // E[k] - w_8^k O[k] (w_8 = (1 -+ i) / sqrt 2, w_8^2 = -+ i)
    C<T> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C<T> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<T, INV>(e0, e1, e2, e3);
    dft4<T, INV>(o0, o1, o2, o3);
    const T h = (T)0.70710678118654752440;
    // w_8 o1, w_8^2 o2, w_8^3 o3 (forward; the inverse takes the conjugates)
    C<T> p1 = INV ? mk<T>(h * (o1.x - o1.y), h * (o1.x + o1.y)) : mk<T>(h * (o1.x + o1.y), h * (o1.y - o1.x));
    C<T> p2 = INV ? mk<T>(-o2.y, o2.x) : mk<T>(o2.y, -o2.x);
    C<T> p3 = INV ? mk<T>(-h * (o3.x + o3.y), h * (o3.x - o3.y)) : mk<T>(h * (o3.y - o3.x), -h * (o3.x + o3.y));
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, p1);
    v[5] = csub(e1, p1);
    v[2] = cadd(e2, p2);
    v[6] = csub(e2, p2);
    v[3] = cadd(e3, p3);
    v[7] = csub(e3, p3);
  } else if constexpr (R == 2) {
    C<T> a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if constexpr (R == 4) {
    C<T> t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    C<T> t2 = cadd(v[1], v[3]), d = csub(v[1], v[3]);
    // forward: -i * d ; inverse: +i * d
    C<T> t3 = INV ? mk<T>(-d.y, d.x) : mk<T>(d.y, -d.x);
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  } else {
    C<T> y[R];
    const int step = L / R;
#pragma unroll
    for (int s = 0; s < R; ++s) {
      C<T> acc = v[0];
#pragma unroll
      for (int r = 1; r < R; ++r) cfma(acc, v[r], twid<T, INV>(tw, ((r * s) % R) * step));
      y[s] = acc;
    }
#pragma unroll
    for (int s = 0; s < R; ++s) v[s] = y[s];
  }
}

// One Stockham stage of radix R: src -> dst for ntr sequences of length L.
template <typename T, bool INV, int R>
__device__ __forceinline__ void fft_stage(const C<T> *src, C<T> *dst, int ld, int ntr, const C<T> *tw, int L,
                                          int Ns, int tid, int nthr) {
  const int LR = L / R;
  const int tstep = L / (Ns * R);
  const int total = LR * ntr;
  for (int q = tid; q < total; q += nthr) {
    const int t = q % ntr;
    const int j = q / ntr;
    const int k = j % Ns;
    C<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      C<T> x = src[(j + r * LR) * ld + t];
      if (r > 0 && k > 0) x = cmul(x, twid<T, INV>(tw, k * r * tstep));
      v[r] = x;
    }
    dft_small<T, INV, R>(v, tw, L);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[(base + r * Ns) * ld + t] = v[r];
  }
}

// Run the plan on ntr sequences stored as buf[l * ld + t] (t < ntr).  A holds the
// input; B is scratch of the same shape.  Returns the buffer with the result.
// Supported radices: 2, 3, 4, 5, 7, 8, 11, 13 (make_plan rejects other prime factors).
template <typename T, bool INV>
__device__ C<T> *fft_smem(C<T> *A, C<T> *B, int ld, int ntr, const C<T> *tw, const FftPlan &p, int tid,
                          int nthr) {
  const int L = p.L;
  int Ns = 1;
  C<T> *src = A, *dst = B;
  for (int st = 0; st < p.n_stages; ++st) {
    const int R = p.radix[st];
    switch (R) {
      case 8: fft_stage<T, INV, 8>(src, dst, ld, ntr, tw, L, Ns, tid, nthr); break;
      case 4: fft_stage<T, INV, 4>(src, dst, ld, ntr, tw, L, Ns, tid, nthr); break;
      case 2: fft_stage<T, INV, 2>(src, dst, ld, ntr, tw, L, Ns, tid, nthr); break;
      case 3: fft_stage<T, INV, 3>(src, dst, ld, ntr, tw, L, Ns, tid, nthr); break;
      case 5: fft_stage<T, INV, 5>(src, dst, ld, ntr, tw, L, Ns, tid, nthr); break;
      case 7: fft_stage<T, INV, 7>(src, dst, ld, ntr, tw, L, Ns, tid, nthr); break;
      case 11: fft_stage<T, INV, 11>(src, dst, ld, ntr, tw, L, Ns, tid, nthr); break;
      case 13: fft_stage<T, INV, 13>(src, dst, ld, ntr, tw, L, Ns, tid, nthr); break;
      default: break;
    }
    __syncthreads();
    C<T> *tmp = src; src = dst; dst = tmp;
    Ns *= R;
  }
  return src;
}

// ---------------------------------------------------------------------------
// Launchers (defined in fft.cu)
// ---------------------------------------------------------------------------

// Transform along the middle axis of in[outer][Lin][inner] -> out[outer][Lout][inner]
// with transform length plan.L (rows >= Lin are zero; rows >= Lout are dropped),
// multiplying by `scale`.
template <typename T, bool INV>
void launch_fft_axis(const C<T> *in, C<T> *out, int outer, int Lin, int Lout, long long inner,
                     const FftPlan &plan, T scale, cudaStream_t s);

// Forward row pass: x[CZ][Ny][Nx] times in_scale[Nz][Ny][Nx] (cz -> z = cz % Nz), zero-padded
// to 2Nx and transformed along x -> T1[Ny][2Nx][CZ].
// T: arithmetic of the transform and of the scales; TX: element type of x (TX = double
// with T = float: FP64 vectors rounded to FP32 on load, then scaled in FP32).
template <typename T, typename TX = T>
void launch_fft_rows_fwd(const C<TX> *x, const C<T> *in_scale, C<T> *t1, int CZ, int Nz, int Ny, int Nx,
                         const FftPlan &plan, cudaStream_t s);

// Inverse row pass: T1[Ny][2Nx][CZ] -> inverse along kx, keep x < Nx, and write
// y[CZ][Ny][Nx] = diag[cell] * x[CZ][cell] + out_scale[cell] * value, in the arithmetic of
// T (TX = double with T = float: x rounded to FP32, the result stored as FP64).
template <typename T, typename TX = T>
void launch_fft_rows_inv(const C<T> *t1, const C<TX> *x, const C<T> *diag, const C<T> *out_scale, C<TX> *y,
                         int CZ, int Nz, int Ny, int Nx, const FftPlan &plan, cudaStream_t s);

}  // namespace ie
