// Persistent, TMA-pipelined wavenumber contraction (step 2 of the FFT product,
// Sect. 3.3) for compile-time Nz and right-hand-side count.
//
// Each CTA walks folded wavenumbers w = blockIdx.x, blockIdx.x + gridDim.x, ...
// The spectrum vector of a wavenumber is spec[(ky 2Nx + kx) ldz + 0 .. R 3Nz) (ldz >= R 3Nz:
// several instances may share one spectrum, each with its own slice and coefficients).
// The packed coefficient block of a wavenumber (2 Nz (2 Nz + 1) complex, contiguous)
// and its up to four mirror spectrum vectors (R * 3 Nz complex each, contiguous) are
// fetched by one thread with 1-D bulk TMA copies (cp.async.bulk) into a ring of
// NSTAGE shared-memory slots completed on an mbarrier, so that the copies of the
// next wavenumbers overlap the arithmetic of the current one.  The block is
// unpacked into six padded Nz x (Nz + 1) matrices (stride Nz + 1 makes both row and
// column reads of 8-byte elements free of bank conflicts) and applied as a small
// dense product Y = M X, M = [[xx, xy, xz], [xy, yy, yz], [-xz^T, -yz^T, zz]],
// X = the mirror vectors with the component signs of Lemma 2.  A thread owns RPT output
// rows (two for two right-hand sides, so that each broadcast load of X feeds twice the
// FMAs) and CPT = 4 columns; packed two-lane FP32 FMAs, FP32 accumulation.
//
// Every wait on an mbarrier is bounded; on timeout the kernel records an error
// code, waits (bounded) for its outstanding copies and returns.
#pragma once
#include "ie_common.cuh"

namespace ie {
namespace tma {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
// bounded wait: true when the phase completed, false after max_iter polls
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase, long long max_iter) {
  for (long long i = 0; i < max_iter; ++i)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

}  // namespace tma

// Packed two-lane FP32 FMA of sm_100+ (fma.rn.f32x2): one instruction, two FMAs.
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long pk(float lo, float hi) {
  return (unsigned long long)__float_as_uint(lo) | ((unsigned long long)__float_as_uint(hi) << 32);
}
__device__ __forceinline__ float2 upk(unsigned long long v) {
  return make_float2(__uint_as_float((unsigned)(v & 0xffffffffu)), __uint_as_float((unsigned)(v >> 32)));
}

// Polls before a wait is declared failed.  The main waits of a kernel take their limit
// as an argument (normally kWaitLimit; a test may lower it to make a wait run out);
// the drain after a timeout, which only waits for the CTA's own copies in flight,
// always uses kWaitLimit.
constexpr long long kWaitLimit = 1LL << 28;
enum ContractError { kContractOk = 0, kContractTimeout = 1 };

template <int NZ, int R, int NSTAGE, int RPT_ = (R == 2 ? 2 : 1)>
struct ContractCfg {
  static constexpr int N3 = 3 * NZ;
  static constexpr int CZ = R * N3;
  static constexpr int P = NZ * (NZ + 1) / 2;
  static constexpr int BS = 2 * NZ * (2 * NZ + 1);
  static constexpr int LD = NZ + 1;
  static constexpr int MAXC = 4 * R;              // 4 mirrors x R right-hand sides
  static constexpr int CPT = 4;                    // columns per thread
  static constexpr int CG = MAXC / CPT;            // column groups
  static constexpr int RPT = RPT_;                  // output rows per thread
  static constexpr int NR = N3 / RPT;              // row slots
  static constexpr int THREADS = NR * CG;
  // shared memory layout (bytes, 16-byte aligned pieces)
  static constexpr size_t OFF_BAR = 0;
  static constexpr size_t OFF_RAW = 128;
  static constexpr size_t RAW_BYTES = (size_t)BS * 8;
  static constexpr size_t XRAW_BYTES = (size_t)4 * CZ * 8;
  static constexpr size_t OFF_XRAW = OFF_RAW + NSTAGE * RAW_BYTES;
  static constexpr size_t OFF_BLK = OFF_XRAW + NSTAGE * XRAW_BYTES;
  static constexpr size_t BLK_BYTES = (size_t)6 * NZ * LD * 8;
  static constexpr size_t OFF_XS = OFF_BLK + BLK_BYTES;
  // X rows padded from MAXC to MAXC + 2 complex: the staging stores (consecutive
  // threads on consecutive rows) then spread over the banks, and rows stay 16-byte
  // aligned for the 128-bit broadcast loads of the product
  static constexpr int XLD = MAXC + 2;
  static constexpr size_t XS_BYTES = (size_t)N3 * XLD * 8;
  static constexpr size_t OFF_TRI = OFF_XS + XS_BYTES;
  static constexpr size_t SMEM = OFF_TRI + (size_t)P * 4;
};

// Folded wavenumber w = ky_bar (Nx + 1) + kx_bar and its mirrors 2 Nx - kx_bar,
// 2 Ny - ky_bar (present for 0 < k_bar < N).  Kept in scalars: indexing small
// per-thread arrays by a run-time mirror number would place them in local memory.
struct Mirrors {
  int kx0, kx1, ky0, ky1, nmx, nmy;
  __device__ __forceinline__ size_t pos(int mx, int my, int Nx) const {
    return (size_t)(my ? ky1 : ky0) * 2 * Nx + (mx ? kx1 : kx0);
  }
};
__device__ __forceinline__ Mirrors mirrors_of(int w, int Nx, int Ny) {
  Mirrors m;
  m.kx0 = w % (Nx + 1);
  m.ky0 = w / (Nx + 1);
  m.nmx = (m.kx0 > 0 && m.kx0 < Nx) ? 2 : 1;
  m.nmy = (m.ky0 > 0 && m.ky0 < Ny) ? 2 : 1;
  m.kx1 = 2 * Nx - m.kx0;
  m.ky1 = 2 * Ny - m.ky0;
  return m;
}

template <int NZ, int R, int NSTAGE, int RPT_>
__global__ void __launch_bounds__(ContractCfg<NZ, R, NSTAGE, RPT_>::THREADS)
    contract_tma_kernel(float2 *__restrict__ spec, const float2 *__restrict__ qf, int Nx, int Ny, int ldz, int *err,
                        long long lim) {
  using Cfg = ContractCfg<NZ, R, NSTAGE, RPT_>;
  constexpr int N3 = Cfg::N3, CZ = Cfg::CZ, P = Cfg::P, BS = Cfg::BS, LD = Cfg::LD, MAXC = Cfg::MAXC;
  constexpr int XLD = Cfg::XLD;
  constexpr int CPT = Cfg::CPT, RPT = Cfg::RPT;
  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + Cfg::OFF_BAR);
  float2 *raw = reinterpret_cast<float2 *>(sm + Cfg::OFF_RAW);
  float2 *xraw = reinterpret_cast<float2 *>(sm + Cfg::OFF_XRAW);
  float2 *blk = reinterpret_cast<float2 *>(sm + Cfg::OFF_BLK);
  float2 *xs = reinterpret_cast<float2 *>(sm + Cfg::OFF_XS);
  uint32_t *tri = reinterpret_cast<uint32_t *>(sm + Cfg::OFF_TRI);
  const int tid = threadIdx.x;
  const int nf = (Nx + 1) * (Ny + 1);

  // packed upper-triangle index -> (a, b)
  for (int a = tid; a < NZ; a += Cfg::THREADS) {
    const int base = a * NZ - a * (a - 1) / 2;
    for (int b = a; b < NZ; ++b) tri[base + b - a] = (uint32_t)(a << 16 | b);
  }
  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) tma::mbar_init(&bar[s], 1);
    tma::fence_mbar_init();
  }
  __syncthreads();

  // thread 0: issue the copies of wavenumber w into slot s
  auto issue = [&](int w, int s) {
    const Mirrors mi = mirrors_of(w, Nx, Ny);
    const int nm = mi.nmx * mi.nmy;
    const uint32_t bytes = (uint32_t)(Cfg::RAW_BYTES + (size_t)nm * CZ * 8);
    tma::fence_proxy_async();
    tma::mbar_expect_tx(&bar[s], bytes);
    tma::bulk_g2s(raw + (size_t)s * BS, qf + (size_t)w * BS, (uint32_t)Cfg::RAW_BYTES, &bar[s]);
    for (int m = 0; m < nm; ++m) {
      const int mx = m % mi.nmx, my = m / mi.nmx;
      tma::bulk_g2s(xraw + (size_t)s * 4 * CZ + (size_t)m * CZ, spec + mi.pos(mx, my, Nx) * ldz, (uint32_t)(CZ * 8),
                    &bar[s]);
    }
  };

  int w0 = blockIdx.x;
  if (tid == 0) {
    for (int k = 0; k < NSTAGE; ++k) {
      const int w = w0 + k * gridDim.x;
      if (w < nf) issue(w, k);
    }
  }
  // thread (rr, cg) owns rows rr + k NR (k < RPT) and columns cg CPT .. cg CPT + CPT - 1
  const int rr = tid % Cfg::NR;
  const int cg = tid / Cfg::NR;
  // per (row, beta): base pointer, stride and sign of M[row][beta*NZ + b]
  const float2 *Axx = blk, *Ayy = blk + NZ * LD, *Azz = blk + 2 * NZ * LD, *Axy = blk + 3 * NZ * LD;
  const float2 *Axz = blk + 4 * NZ * LD, *Ayz = blk + 5 * NZ * LD;
  const float2 *bp[RPT][3];
  int bs[RPT][3];
  float sg[RPT][3];
  int alph[RPT];
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int row = rr + k * Cfg::NR;
    const int alpha = row / NZ, a = row - alpha * NZ;
    alph[k] = alpha;
    if (alpha == 0) {
      bp[k][0] = Axx + a; bs[k][0] = LD; sg[k][0] = 1.f;
      bp[k][1] = Axy + a; bs[k][1] = LD; sg[k][1] = 1.f;
      bp[k][2] = Axz + a * LD; bs[k][2] = 1; sg[k][2] = 1.f;
    } else if (alpha == 1) {
      bp[k][0] = Axy + a; bs[k][0] = LD; sg[k][0] = 1.f;
      bp[k][1] = Ayy + a; bs[k][1] = LD; sg[k][1] = 1.f;
      bp[k][2] = Ayz + a * LD; bs[k][2] = 1; sg[k][2] = 1.f;
    } else {
      bp[k][0] = Axz + a; bs[k][0] = LD; sg[k][0] = -1.f;
      bp[k][1] = Ayz + a; bs[k][1] = LD; sg[k][1] = -1.f;
      bp[k][2] = Azz + a; bs[k][2] = LD; sg[k][2] = 1.f;
    }
  }

  int it = 0;
  for (int w = w0; w < nf; w += gridDim.x, ++it) {
    const int s = it % NSTAGE;
    const uint32_t phase = (uint32_t)((it / NSTAGE) & 1);
    if (!tma::mbar_wait_bounded(&bar[s], phase, lim)) {
      if (tid == 0) atomicExch(err, kContractTimeout);
      // drain: the slots hold the copies of iterations it .. it + NSTAGE - 1 (those that
      // were issued), each completing the phase of its own iteration
      for (int k = 0; k < NSTAGE; ++k)
        if (w + k * (int)gridDim.x < nf)
          tma::mbar_wait_bounded(&bar[(s + k) % NSTAGE], (uint32_t)(((it + k) / NSTAGE) & 1), kWaitLimit);
      return;
    }
    const Mirrors mw = mirrors_of(w, Nx, Ny);
    const int nmx = mw.nmx;
    const int ncol = mw.nmx * mw.nmy * R;
    // unpack the packed block of slot s
    const float2 *q = raw + (size_t)s * BS;
    for (int e = tid; e < 4 * P; e += Cfg::THREADS) {
      const int kind = e / P;
      const uint32_t ab = tri[e - kind * P];
      const int ia = ab >> 16, ib = ab & 0xffff;
      const float2 v = q[e];
      float2 *m = blk + kind * NZ * LD;
      m[ia * LD + ib] = v;
      m[ib * LD + ia] = v;
    }
    for (int e = tid; e < 2 * NZ * NZ; e += Cfg::THREADS) {
      const int kind = e / (NZ * NZ);
      const int r2 = e - kind * NZ * NZ;
      const int ia = r2 / NZ, ib = r2 - ia * NZ;
      blk[(4 + kind) * NZ * LD + ia * LD + ib] = q[4 * P + e];
    }
    // stage X[k][col] with the component signs of the mirrors
    const float2 *xr = xraw + (size_t)s * 4 * CZ;
    for (int e = tid; e < MAXC * N3; e += Cfg::THREADS) {
      const int col = e / N3, k = e - col * N3;
      float2 v = make_float2(0.f, 0.f);
      if (col < ncol) {
        const int m = col / R, r = col - m * R;
        const int mx = m % nmx, my = m / nmx;
        const int comp = k / NZ;
        v = xr[(size_t)m * CZ + r * N3 + k];
        if ((comp == 0 && mx == 1) || (comp == 1 && my == 1)) { v.x = -v.x; v.y = -v.y; }
      }
      xs[k * XLD + col] = v;
    }
    __syncthreads();
    // slot s is consumed: refill it with wavenumber w + NSTAGE * gridDim.x
    if (tid == 0) {
      const int wn = w + NSTAGE * gridDim.x;
      if (wn < nf) issue(wn, s);
    }
    if (cg * CPT < ncol) {
      // complex MAC as two packed FMAs into two accumulators: a1 += (xr, xi)(mr, mr) and,
      // in swapped order, a2 += (xr, xi)(mi, -mi); then re = a1.x + a2.y, im = a1.y + a2.x.
      unsigned long long a1[RPT][CPT], a2[RPT][CPT];
#pragma unroll
      for (int k = 0; k < RPT; ++k)
#pragma unroll
        for (int c = 0; c < CPT; ++c) a1[k][c] = a2[k][c] = 0ull;
#pragma unroll
      for (int beta = 0; beta < 3; ++beta) {
        unsigned long long t1[RPT][CPT], t2[RPT][CPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k)
#pragma unroll
          for (int c = 0; c < CPT; ++c) t1[k][c] = t2[k][c] = 0ull;
        const ulonglong2 *xp = reinterpret_cast<const ulonglong2 *>(xs + (size_t)beta * NZ * XLD + cg * CPT);
#pragma unroll 4
        for (int b = 0; b < NZ; ++b) {
          const ulonglong2 x01 = xp[b * (XLD / 2)], x23 = xp[b * (XLD / 2) + 1];
#pragma unroll
          for (int k = 0; k < RPT; ++k) {
            const float2 m = bp[k][beta][b * bs[k][beta]];
            const unsigned long long mr = pk(m.x, m.x), mi = pk(m.y, -m.y);
            t1[k][0] = ffma2(x01.x, mr, t1[k][0]);
            t2[k][0] = ffma2(x01.x, mi, t2[k][0]);
            t1[k][1] = ffma2(x01.y, mr, t1[k][1]);
            t2[k][1] = ffma2(x01.y, mi, t2[k][1]);
            t1[k][2] = ffma2(x23.x, mr, t1[k][2]);
            t2[k][2] = ffma2(x23.x, mi, t2[k][2]);
            t1[k][3] = ffma2(x23.y, mr, t1[k][3]);
            t2[k][3] = ffma2(x23.y, mi, t2[k][3]);
          }
        }
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
          const unsigned long long sgp = pk(sg[k][beta], sg[k][beta]);
#pragma unroll
          for (int c = 0; c < CPT; ++c) {
            a1[k][c] = ffma2(sgp, t1[k][c], a1[k][c]);
            a2[k][c] = ffma2(sgp, t2[k][c], a2[k][c]);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < RPT; ++k) {
        const int row = rr + k * Cfg::NR;
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          const int col = cg * CPT + c;
          if (col < ncol) {
            const int m = col / R, r = col - m * R;
            const int mx = m % nmx, my = m / nmx;
            const float2 u1 = upk(a1[k][c]), u2 = upk(a2[k][c]);
            float2 v = make_float2(u1.x + u2.y, u1.y + u2.x);
            if ((alph[k] == 0 && mx == 1) || (alph[k] == 1 && my == 1)) { v.x = -v.x; v.y = -v.y; }
            spec[mw.pos(mx, my, Nx) * ldz + r * N3 + row] = v;
          }
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace ie
