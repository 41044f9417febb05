// Persistent, TMA-pipelined wavenumber contraction (step 2 of the FFT product,
// Sect. 3.3) for compile-time Nz and right-hand-side count.
//
// Each CTA walks folded wavenumbers w = blockIdx.x, blockIdx.x + gridDim.x, ...
// The packed coefficient block of a wavenumber (2 Nz (2 Nz + 1) complex, contiguous)
// and its up to four mirror spectrum vectors (R * 3 Nz complex each, contiguous) are
// fetched by one thread with 1-D bulk TMA copies (cp.async.bulk) into a ring of
// NSTAGE shared-memory slots completed on an mbarrier, so that the copies of the
// next wavenumbers overlap the arithmetic of the current one.  The block is
// unpacked into six padded Nz x (Nz + 1) matrices (stride Nz + 1 makes both row and
// column reads of 8-byte elements free of bank conflicts) and applied as a small
// dense product Y = M X, M = [[xx, xy, xz], [xy, yy, yz], [-xz^T, -yz^T, zz]],
// X = the mirror vectors with the component signs of Lemma 2.  Thread t owns one
// output row and CPT columns (FP32 FMAs, FP32 accumulation).
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

constexpr long long kWaitLimit = 1LL << 28;  // polls before a wait is declared failed
enum ContractError { kContractOk = 0, kContractTimeout = 1 };

template <int NZ, int R, int NSTAGE>
struct ContractCfg {
  static constexpr int N3 = 3 * NZ;
  static constexpr int CZ = R * N3;
  static constexpr int P = NZ * (NZ + 1) / 2;
  static constexpr int BS = 2 * NZ * (2 * NZ + 1);
  static constexpr int LD = NZ + 1;
  static constexpr int MAXC = 4 * R;              // 4 mirrors x R right-hand sides
  static constexpr int CPT = 4;                    // columns per thread
  static constexpr int CG = MAXC / CPT;            // column groups
  static constexpr int THREADS = N3 * CG;
  // shared memory layout (bytes, 16-byte aligned pieces)
  static constexpr size_t OFF_BAR = 0;
  static constexpr size_t OFF_RAW = 128;
  static constexpr size_t RAW_BYTES = (size_t)BS * 8;
  static constexpr size_t XRAW_BYTES = (size_t)4 * CZ * 8;
  static constexpr size_t OFF_XRAW = OFF_RAW + NSTAGE * RAW_BYTES;
  static constexpr size_t OFF_BLK = OFF_XRAW + NSTAGE * XRAW_BYTES;
  static constexpr size_t BLK_BYTES = (size_t)6 * NZ * LD * 8;
  static constexpr size_t OFF_XS = OFF_BLK + BLK_BYTES;
  static constexpr size_t XS_BYTES = (size_t)N3 * MAXC * 8;
  static constexpr size_t OFF_TRI = OFF_XS + XS_BYTES;
  static constexpr size_t SMEM = OFF_TRI + (size_t)P * 4;
};

template <int NZ, int R, int NSTAGE>
__global__ void __launch_bounds__(ContractCfg<NZ, R, NSTAGE>::THREADS)
    contract_tma_kernel(float2 *__restrict__ spec, const float2 *__restrict__ qf, int Nx, int Ny, int *err) {
  using Cfg = ContractCfg<NZ, R, NSTAGE>;
  constexpr int N3 = Cfg::N3, CZ = Cfg::CZ, P = Cfg::P, BS = Cfg::BS, LD = Cfg::LD, MAXC = Cfg::MAXC;
  constexpr int CPT = Cfg::CPT;
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

  auto mirrors = [&](int w, int *kxs, int *kys, int &nmx, int &nmy) {
    const int kxb = w % (Nx + 1), kyb = w / (Nx + 1);
    kxs[0] = kxb; kys[0] = kyb; nmx = 1; nmy = 1;
    if (kxb > 0 && kxb < Nx) { kxs[1] = 2 * Nx - kxb; nmx = 2; }
    if (kyb > 0 && kyb < Ny) { kys[1] = 2 * Ny - kyb; nmy = 2; }
  };
  // thread 0: issue the copies of wavenumber w into slot s
  auto issue = [&](int w, int s) {
    int kxs[2], kys[2], nmx, nmy;
    mirrors(w, kxs, kys, nmx, nmy);
    const uint32_t bytes = (uint32_t)(Cfg::RAW_BYTES + (size_t)nmx * nmy * CZ * 8);
    tma::fence_proxy_async();
    tma::mbar_expect_tx(&bar[s], bytes);
    tma::bulk_g2s(raw + (size_t)s * BS, qf + (size_t)w * BS, (uint32_t)Cfg::RAW_BYTES, &bar[s]);
    for (int m = 0; m < nmx * nmy; ++m) {
      const int mx = m % nmx, my = m / nmx;
      const size_t g = ((size_t)kys[my] * 2 * Nx + kxs[mx]) * CZ;
      tma::bulk_g2s(xraw + (size_t)s * 4 * CZ + (size_t)m * CZ, spec + g, (uint32_t)(CZ * 8), &bar[s]);
    }
  };

  int w0 = blockIdx.x;
  if (tid == 0) {
    for (int k = 0; k < NSTAGE; ++k) {
      const int w = w0 + k * gridDim.x;
      if (w < nf) issue(w, k);
    }
  }
  const int row = tid % N3;
  const int cg = tid / N3;
  const int alpha = row / NZ, a = row - alpha * NZ;
  // per-beta base pointers, strides and signs of M[row][beta*NZ + b]
  const float2 *Axx = blk, *Ayy = blk + NZ * LD, *Azz = blk + 2 * NZ * LD, *Axy = blk + 3 * NZ * LD;
  const float2 *Axz = blk + 4 * NZ * LD, *Ayz = blk + 5 * NZ * LD;
  const float2 *bp[3];
  int bs[3];
  float sg[3];
  if (alpha == 0) {
    bp[0] = Axx + a; bs[0] = LD; sg[0] = 1.f;
    bp[1] = Axy + a; bs[1] = LD; sg[1] = 1.f;
    bp[2] = Axz + a * LD; bs[2] = 1; sg[2] = 1.f;
  } else if (alpha == 1) {
    bp[0] = Axy + a; bs[0] = LD; sg[0] = 1.f;
    bp[1] = Ayy + a; bs[1] = LD; sg[1] = 1.f;
    bp[2] = Ayz + a * LD; bs[2] = 1; sg[2] = 1.f;
  } else {
    bp[0] = Axz + a; bs[0] = LD; sg[0] = -1.f;
    bp[1] = Ayz + a; bs[1] = LD; sg[1] = -1.f;
    bp[2] = Azz + a; bs[2] = LD; sg[2] = 1.f;
  }

  int it = 0;
  for (int w = w0; w < nf; w += gridDim.x, ++it) {
    const int s = it % NSTAGE;
    const uint32_t phase = (uint32_t)((it / NSTAGE) & 1);
    if (!tma::mbar_wait_bounded(&bar[s], phase, kWaitLimit)) {
      if (tid == 0) atomicExch(err, kContractTimeout);
      // drain: wait (bounded) for every slot that may still have copies in flight
      for (int k = 0; k < NSTAGE; ++k) tma::mbar_wait_bounded(&bar[(s + k) % NSTAGE], phase, kWaitLimit);
      return;
    }
    int kxs[2], kys[2], nmx, nmy;
    mirrors(w, kxs, kys, nmx, nmy);
    const int ncol = nmx * nmy * R;
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
      xs[k * MAXC + col] = v;
    }
    __syncthreads();
    // slot s is consumed: refill it with wavenumber w + NSTAGE * gridDim.x
    if (tid == 0) {
      const int wn = w + NSTAGE * gridDim.x;
      if (wn < nf) issue(wn, s);
    }
    if (cg * CPT < ncol) {
      float2 acc[CPT];
#pragma unroll
      for (int c = 0; c < CPT; ++c) acc[c] = make_float2(0.f, 0.f);
#pragma unroll
      for (int beta = 0; beta < 3; ++beta) {
        float2 tmp[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) tmp[c] = make_float2(0.f, 0.f);
        const float2 *mp = bp[beta];
        const int st = bs[beta];
        const float4 *xp = reinterpret_cast<const float4 *>(xs + (size_t)beta * NZ * MAXC + cg * CPT);
#pragma unroll 8
        for (int b = 0; b < NZ; ++b) {
          const float2 m = mp[b * st];
          const float4 x01 = xp[b * (MAXC / 2)];
          const float4 x23 = xp[b * (MAXC / 2) + 1];
          const float2 xv[4] = {make_float2(x01.x, x01.y), make_float2(x01.z, x01.w), make_float2(x23.x, x23.y),
                                make_float2(x23.z, x23.w)};
#pragma unroll
          for (int c = 0; c < CPT; ++c) {
            tmp[c].x = fmaf(m.x, xv[c].x, tmp[c].x);
            tmp[c].x = fmaf(-m.y, xv[c].y, tmp[c].x);
            tmp[c].y = fmaf(m.x, xv[c].y, tmp[c].y);
            tmp[c].y = fmaf(m.y, xv[c].x, tmp[c].y);
          }
        }
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          acc[c].x = fmaf(sg[beta], tmp[c].x, acc[c].x);
          acc[c].y = fmaf(sg[beta], tmp[c].y, acc[c].y);
        }
      }
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        const int col = cg * CPT + c;
        if (col < ncol) {
          const int m = col / R, r = col - m * R;
          const int mx = m % nmx, my = m / nmx;
          float2 v = acc[c];
          if ((alpha == 0 && mx == 1) || (alpha == 1 && my == 1)) { v.x = -v.x; v.y = -v.y; }
          spec[((size_t)kys[my] * 2 * Nx + kxs[mx]) * CZ + r * N3 + row] = v;
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace ie
