// Register-blocked FP32 FFTs for transform lengths L = 16 Q, Q in {8, 12, 16, 24, 32}
// (L = 128, 192, 256, 384, 512: the zero-padded lengths 2N of 64-, 96-, 128-, 192- and
// 256-cell grids).
//
// A length-L DFT is split as L = 16 x Q: with l = q + Q p and k = k1 + 16 k2,
//   X[k1 + 16 k2] = sum_q w_Q^(q k2) w_L^(q k1) sum_p x[q + Q p] w_16^(p k1),
// so one thread per (sequence, q) does a 16-point DFT in registers, multiplies by the
// twiddles w_L^(q k1), and after one exchange through shared memory one thread per
// (sequence, k1) does a Q-point DFT in registers (radix 2, and one radix-3 step where
// Q = 3 M).  TI = 16 sequences share a CTA and
// sit in the lowest thread-index bits, so every global load or store of a half-warp
// moves 16 consecutive elements of the sequence index (128 bytes).  The in-register
// DFTs are radix-2 decimation in time, the input permutation resolved at compile time
// by loading the inputs permuted; their twiddles and the w_L^(q k1) come from one table w_L^m per CTA.
#pragma once
#include <utility>

#include "ie_common.cuh"

namespace ie {
namespace fftfast {

constexpr int kTI = 16;

// The exchange between the two steps holds entry (q, k1, t) (q < Q, k1 < 16, t < TI)
// at q kYQ + k1 kYK + t.  Both strides are odd multiples of one 8-byte word modulo 16,
// so 16 consecutive t, 16 consecutive k1 or 16 consecutive q (the three thread
// mappings below) touch 16 distinct 8-byte bank pairs.
constexpr int kYK = kTI + 1;
constexpr int kYQ = 16 * kYK + 1;
__device__ __forceinline__ int yix(int q, int k1, int t) { return q * kYQ + k1 * kYK + t; }

__device__ __forceinline__ float2 fmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <int N>
__host__ __device__ constexpr int bitrev(int i) {
  int r = 0;
  for (int b = 1; b < N; b <<= 1) {
    r = (r << 1) | (i & 1);
    i >>= 1;
  }
  return r;
}

// cos(2 pi j / 32) for j = 0 .. 8
__device__ __forceinline__ constexpr float cos32(int j) {
  return j == 0 ? 1.0f
       : j == 1 ? 0.98078528040323044913f
       : j == 2 ? 0.92387953251128675613f
       : j == 3 ? 0.83146961230254523708f
       : j == 4 ? 0.70710678118654752440f
       : j == 5 ? 0.55557023301960222474f
       : j == 6 ? 0.38268343236508977173f
       : j == 7 ? 0.19509032201612826785f
                : 0.0f;
}
// v times w_32^J (forward sign) or its conjugate, J a compile-time constant: the
// twiddles of the in-register DFTs (w_N^j = w_32^(32 j / N) for N <= 32), so that no
// table is read, the trivial factors (1, -+i) cost no multiplication and the others
// two multiplications and two fused multiply-adds with immediate operands
template <int J, bool INV>
__device__ __forceinline__ float2 twiddle32(float2 v) {
  static_assert(J >= 0 && J < 16, "half a turn at most");
  if constexpr (J == 0) {
    return v;
  } else if constexpr (J == 8) {  // -i (forward), +i (inverse)
    return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
  } else {
    // w = c - i s (forward): c = cos(2 pi J / 32), s = sin(2 pi J / 32)
    constexpr float c = J < 8 ? cos32(J) : -cos32(16 - J);
    constexpr float sn = J < 8 ? cos32(8 - J) : cos32(J - 8);
    constexpr float s = INV ? -sn : sn;
    return make_float2(fmaf(v.x, c, v.y * s), fmaf(v.y, c, -(v.x * s)));
  }
}

// In-register DFT of length N (power of two, N <= 32): the input in bit-reversed order
// (b[bitrev(i)] = x[i], so callers load it permuted at compile time), the output in
// natural order, in place.  The twiddles are compile-time constants (twiddle32).
// One butterfly stage of span LEN, then the next (one template instance per stage, so
// every register index is a compile-time constant).
template <int N, int LEN, bool INV>
struct BrStage {
  template <int J>
  static __device__ __forceinline__ void bfly(float2 (&b)[N], int i) {
    const float2 u = b[i + J];
    const float2 v = twiddle32<J * (32 / LEN), INV>(b[i + J + LEN / 2]);
    b[i + J] = make_float2(u.x + v.x, u.y + v.y);
    b[i + J + LEN / 2] = make_float2(u.x - v.x, u.y - v.y);
  }
  template <int... J>
  static __device__ __forceinline__ void group(float2 (&b)[N], int i, std::integer_sequence<int, J...>) {
    (bfly<J>(b, i), ...);
  }
  static __device__ __forceinline__ void run(float2 (&b)[N], const float2 *tw, int stride) {
    static_assert(N <= 32 && LEN <= N, "twiddles from w_32");
#pragma unroll
    for (int i = 0; i < N; i += LEN) group(b, i, std::make_integer_sequence<int, LEN / 2>{});
    BrStage<N, 2 * LEN, INV>::run(b, tw, stride);
  }
};
template <int N, bool INV>
struct BrStage<N, 2 * N, INV> {
  static __device__ __forceinline__ void run(float2 (&)[N], const float2 *, int) {}
};

template <int N, bool INV>
__device__ __forceinline__ void dft_br(float2 (&b)[N], const float2 *tw, int stride) {
  BrStage<N, 2, INV>::run(b, tw, stride);
}

// w_L^m = exp(-2 pi i m / L) for m < L
__device__ __forceinline__ void fill_table(float2 *tw, int L) {
  for (int m = threadIdx.x; m < L; m += blockDim.x) {
    float s, c;
    sincospif(2.0f * (float)m / (float)L, &s, &c);
    tw[m] = make_float2(c, -s);
  }
}

// Step 1 for one (sequence t, q): v[bitrev(p)] holds x[q + Q p]; writes entry
// (q, k1, t) of the exchange.
template <int Q, bool INV>
__device__ __forceinline__ void step1(float2 (&v)[16], const float2 *tw, float2 *Y, int q, int t) {
  constexpr int L = 16 * Q;
  dft_br<16, INV>(v, tw, L / 16);
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) {
    float2 r = v[k1];
    if (k1 != 0 && q != 0) {
      float2 w = tw[q * k1];
      if (INV) w.y = -w.y;
      r = fmul(r, w);
    }
    Y[yix(q, k1, t)] = r;
  }
}

// Step 2 for one (sequence t, k1): returns X[k1 + 16 k2] in w[k2].  Q a power of two:
// one radix-2 DFT in registers.  Q = 3 M (M a power of two): with q = r + 3 m and
// k2 = k + M s, X = sum_r w_3^(r s) w_Q^(r k) Z_r[k], Z_r the M-point DFT of the inputs
// r, r + 3, ...: three M-point DFTs, the twiddles w_Q^(r k), M 3-point DFTs.
template <int Q, bool INV>
__device__ __forceinline__ void step2(float2 (&w)[Q], const float2 *tw, const float2 *Y, int k1, int t) {
  constexpr int L = 16 * Q;
  if constexpr ((Q & (Q - 1)) == 0) {
#pragma unroll
    for (int q = 0; q < Q; ++q) w[bitrev<Q>(q)] = Y[yix(q, k1, t)];
    dft_br<Q, INV>(w, tw, L / Q);
  } else {
    constexpr int M = Q / 3;
    static_assert(3 * M == Q && (M & (M - 1)) == 0, "Q = 3 M with M a power of two");
    float2 z[3][M];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
      for (int m = 0; m < M; ++m) z[r][bitrev<M>(m)] = Y[yix(r + 3 * m, k1, t)];
      dft_br<M, INV>(z[r], tw, L / M);
    }
    // sin(2 pi / 3); w_3 = -1/2 -+ i s (forward / inverse)
    const float s3 = INV ? -0.86602540378443865f : 0.86602540378443865f;
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const float2 a = z[0][k];
      float2 b = z[1][k], c = z[2][k];
      if (k != 0) {
        float2 w1 = tw[k * (L / Q)], w2 = tw[2 * k * (L / Q)];
        if (INV) {
          w1.y = -w1.y;
          w2.y = -w2.y;
        }
        b = fmul(b, w1);
        c = fmul(c, w2);
      }
      const float2 sp = make_float2(b.x + c.x, b.y + c.y), sm = make_float2(b.x - c.x, b.y - c.y);
      const float2 h = make_float2(a.x - 0.5f * sp.x, a.y - 0.5f * sp.y);
      w[k] = make_float2(a.x + sp.x, a.y + sp.y);
      // w_3 b + w_3^2 c = -(b + c) / 2 - i s (b - c); the conjugate pair for s = 2
      w[k + M] = make_float2(h.x + s3 * sm.y, h.y - s3 * sm.x);
      w[k + 2 * M] = make_float2(h.x - s3 * sm.y, h.y + s3 * sm.x);
    }
  }
}

// Transform along the middle axis of in[outer][Lin][inner] (rows >= Lin are zero) ->
// out[outer][Lout][inner] (rows >= Lout dropped), times scale.  HALF: the zero-padded
// forward transform (Lin = L / 2, Lout = L) or the cropped inverse (Lin = L, Lout =
// L / 2), with the zero inputs and the dropped outputs known at compile time.  The
// loads are issued before the twiddle table is built, so the two overlap.
template <int Q, bool INV, bool HALF>
__global__ void __launch_bounds__(kTI *(Q > 16 ? Q : 16)) axis_kernel(const float2 *__restrict__ in,
                                                                     float2 *__restrict__ out, int Lin, int Lout,
                                                                     long long inner, float scale) {
  constexpr int L = 16 * Q;
  extern __shared__ float2 smf[];
  float2 *tw = smf, *Y = smf + L;
  const int t = threadIdx.x % kTI, j = threadIdx.x / kTI;
  const long long i0 = (long long)blockIdx.x * kTI;
  const long long o = blockIdx.y;
  const bool live = i0 + t < inner;
  float2 v[16];
  if (j < Q) {
#pragma unroll
    for (int p = 0; p < 16; ++p) {
      const int l = j + Q * p;
      const bool have = HALF ? (INV || p < 8) : l < Lin;
      v[bitrev<16>(p)] = (live && have) ? in[(o * Lin + l) * inner + i0 + t] : make_float2(0.f, 0.f);
    }
  }
  fill_table(tw, L);
  __syncthreads();
  if (j < Q) step1<Q, INV>(v, tw, Y, j, t);
  __syncthreads();
  if (j < 16) {
    float2 w[Q];
    step2<Q, INV>(w, tw, Y, j, t);
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) {
      const int l = j + 16 * k2;
      const bool keep = HALF ? (!INV || k2 < Q / 2) : l < Lout;
      if (live && keep) out[(o * Lout + l) * inner + i0 + t] = make_float2(w[k2].x * scale, w[k2].y * scale);
    }
  }
}

// Forward row pass: x[CZ][Ny][Nx] times in_scale[Nz][Ny][Nx], zero-padded to L = 2 Nx
// (Nx = 8 Q), transformed along x -> T1[Ny][L][CZ].  Step 1 runs with q in the low
// thread bits, so each thread loads its eight nonzero inputs straight from the rows
// (Q consecutive elements of a row per warp slice) while the table is being filled;
// step 2 runs with the sequence in the low bits, so the stores are 16 consecutive
// elements of the sequence index.
template <int Q, typename TX>
__global__ void __launch_bounds__(kTI *(Q > 16 ? Q : 16)) rows_fwd_kernel(
    const typename cplx<TX>::type *__restrict__ x, const float2 *__restrict__ in_scale,
    float2 *__restrict__ t1, int CZ, int Nz, int Ny, int Nx) {
  constexpr int L = 16 * Q, NXC = 8 * Q;
  extern __shared__ float2 smf[];
  float2 *tw = smf, *Y = smf + L;
  const int tid = threadIdx.x;
  const int cz0 = blockIdx.x * kTI;
  const int y = blockIdx.y;
  const int q = tid % Q, ts = tid / Q;
  const bool s1 = tid < Q * kTI;
  const bool live = s1 && cz0 + ts < CZ;
  float2 v[16], sc[8];
  {
    const int cz = live ? cz0 + ts : 0;
    const long long row = ((long long)cz * Ny + y) * NXC + q;
    const long long srow = ((long long)(cz % Nz) * Ny + y) * NXC + q;
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      v[bitrev<16>(p)] = live ? to_f32(x[row + Q * p]) : make_float2(0.f, 0.f);
      sc[p] = (live && in_scale) ? in_scale[srow + Q * p] : make_float2(1.f, 0.f);
    }
#pragma unroll
    for (int p = 8; p < 16; ++p) v[bitrev<16>(p)] = make_float2(0.f, 0.f);
  }
  fill_table(tw, L);
#pragma unroll
  for (int p = 0; p < 8; ++p) v[bitrev<16>(p)] = cmul(v[bitrev<16>(p)], sc[p]);
  __syncthreads();
  if (s1) step1<Q, false>(v, tw, Y, q, ts);
  __syncthreads();
  const int t = tid % kTI, j = tid / kTI;
  if (j < 16) {
    float2 w[Q];
    step2<Q, false>(w, tw, Y, j, t);
    if (cz0 + t < CZ) {
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) t1[((long long)y * L + j + 16 * k2) * CZ + cz0 + t] = w[k2];
    }
  }
}

// Inverse row pass: T1[Ny][L][CZ] -> inverse along kx, keep x < Nx (= 8 Q), and write
// y[CZ][Ny][Nx] = diag[cell] x[CZ][cell] + out_scale[cell] value.  Step 1 runs with the
// sequence in the low thread bits (loads of 16 consecutive sequence elements), step 2
// with k1 in the low bits, so each output x = k1 + 16 k2 goes straight to its row
// (16 consecutive elements per half-warp).
template <int Q, typename TX>
__global__ void __launch_bounds__(kTI *(Q > 16 ? Q : 16)) rows_inv_kernel(
    const float2 *__restrict__ t1, const typename cplx<TX>::type *__restrict__ x,
    const float2 *__restrict__ diag, const float2 *__restrict__ out_scale,
    typename cplx<TX>::type *__restrict__ y_out, int CZ, int Nz, int Ny, int Nx) {
  constexpr int L = 16 * Q, NXC = 8 * Q;
  extern __shared__ float2 smf[];
  float2 *tw = smf, *Y = smf + L;
  const int tid = threadIdx.x;
  const int cz0 = blockIdx.x * kTI;
  const int y = blockIdx.y;
  {
    const int t = tid % kTI, j = tid / kTI;
    const bool live = cz0 + t < CZ;
    float2 v[16];
    if (j < Q) {
#pragma unroll
      for (int p = 0; p < 16; ++p)
        v[bitrev<16>(p)] = live ? t1[((long long)y * L + j + Q * p) * CZ + cz0 + t] : make_float2(0.f, 0.f);
    }
    fill_table(tw, L);
    __syncthreads();
    if (j < Q) step1<Q, true>(v, tw, Y, j, t);
  }
  __syncthreads();
  const int k1 = tid % 16, ts = tid / 16;
  const int cz = cz0 + ts;
  if (ts < kTI && cz < CZ) {
    float2 w[Q];
    step2<Q, true>(w, tw, Y, k1, ts);
    const long long row = ((long long)cz * Ny + y) * NXC + k1;
    const long long srow = ((long long)(cz % Nz) * Ny + y) * NXC + k1;
#pragma unroll
    for (int k2 = 0; k2 < Q / 2; ++k2) {
      float2 val = cmul(w[k2], out_scale[srow + 16 * k2]);
      if (diag) cfma(val, diag[srow + 16 * k2], to_f32(x[row + 16 * k2]));
      y_out[row + 16 * k2] = to_prec<TX>(val);
    }
  }
}

// dynamic shared memory of every kernel above: the table and the exchange
constexpr size_t smem_bytes(int Q) { return sizeof(float2) * (size_t)Q * (16 + kYQ); }
constexpr int threads(int Q) { return kTI * (Q > 16 ? Q : 16); }

}  // namespace fftfast
}  // namespace ie
