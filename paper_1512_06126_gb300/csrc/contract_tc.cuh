// Wavenumber contraction (step 2 of the FFT product, Sect. 3.3) on the 5th-generation
// tensor cores: tcgen05.mma with the coefficient block in tensor memory (TMEM), the
// spectrum vectors in shared memory, FP32 accumulators in TMEM.  c64, compile-time Nz
// with 3 Nz <= 128 (one M = 128 tile of output rows), R <= 2 right-hand sides.
//
// Per folded wavenumber the 3Nz x 3Nz complex block M meets at most 8 columns X (4
// mirrors x R).  As a real product per input component beta (a K-chunk of 2 Nz):
//   D += [M_r | M_i](:, beta) . [[X_r, X_i], [-X_i, X_r]](beta)
// so D[:, c] = Y_r and D[:, 8 + c] = Y_i of column c (N = 16).  FP32 accuracy from the
// 3xTF32 split x = hi + lo (hi = x rounded to TF32, lo = x - hi exactly): one N = 32 MMA
// D1 += A_hi [B_hi | B_lo] (both parts of B are consecutive core-matrix groups) and one
// N = 16 MMA D2 += A_lo B_hi per k-step (the dropped A_lo B_lo is ~2^-22 of the
// product).  The tensor core takes a nearly fixed time per instruction at these small N,
// so fusing two of the three products into one N = 32 instruction saves a third of the
// issue time.
//
// Warp roles (one CTA per SM; persistent over folded wavenumbers w = blockIdx.x +
// k gridDim.x):
//  * warp 0, the producer: a 1-D bulk copy (cp.async.bulk) of the packed triangles of
//    xx, yy, zz, xy, tensor-map copies (cp.async.bulk.tensor, 128-byte swizzle) of the
//    full xz and yz blocks in boxes of 16 columns, and 1-D copies of the mirror spectrum
//    vectors into a ring of NS shared-memory stages: at most 1 + Nz/16 + 4 requests per
//    wavenumber (one request per row of xz and yz kept the copy engine busy for longer
//    than the data took to arrive);
//  * warp 1, the MMA issuer: one thread issues the 3 x (2 Nz / 8) x 3 tcgen05.mma of a
//    wavenumber and commits their completion to mbarriers;
//  * row warps (TMEM lane quadrant q = warp % 4 holds output rows 32q .. 32q + 31): each
//    thread unpacks its row of the block chunk by chunk (Lemma 1: zx = -xz^T, zy =
//    -yz^T), splits it and stores it to a ring of NA chunk buffers in TMEM
//    (tcgen05.st); after the MMAs of a wavenumber the same warps read the accumulators
//    (tcgen05.ld), apply the mirror component signs (Lemma 2) and store the outputs;
//  * B warps: split X (mirror signs applied) into the K-major no-swizzle layout of the
//    MMA's B operand (core matrices of 8 rows x 16 bytes), double-buffered.
// Every wait is bounded: on timeout the kernel records an error, each role stops, the
// producer drains its copies and the issuer its MMAs, and TMEM is released.
#pragma once
#include <cuda.h>  // CUtensorMap (the map is encoded on the host through the runtime's driver entry point)
#include <cuda_fp16.h>

#include "contract_tma.cuh"

namespace ie {
namespace tc {

__device__ __forceinline__ void alloc(uint32_t *dst, int ncols) {  // one full warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tma::smem_u32(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void dealloc(uint32_t taddr, int ncols) {  // one full warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 8 consecutive TMEM columns of this warp's lanes from 8 registers per thread
__device__ __forceinline__ void st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
               "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void st4(uint32_t taddr, const uint32_t (&r)[4]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr), "r"(r[0]), "r"(r[1]),
               "r"(r[2]), "r"(r[3])
               : "memory");
}
__device__ __forceinline__ void st2(uint32_t taddr, const uint32_t (&r)[2]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1,%2};" ::"r"(taddr), "r"(r[0]), "r"(r[1]) : "memory");
}
__device__ __forceinline__ void ld2(uint32_t taddr, uint32_t &a, uint32_t &b) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(a), "=r"(b) : "r"(taddr) : "memory");
}

// Shared-memory matrix descriptor: K-major, no swizzle; lbo = byte distance between
// core matrices adjacent in K, sbo = between core matrices adjacent in M/N.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// Instruction descriptor of kind::f16 with FP16 A and B (format 0), FP32 accumulator.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// D (+)= A B, A in TMEM, B from a shared-memory descriptor; kind::tf32 or kind::f16
template <bool F16>
__device__ __forceinline__ void mma_k(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  if constexpr (F16)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(
            d),
        "r"(a), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(
            d),
        "r"(a), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
// D (+)= A B, A in TMEM, B from a shared-memory descriptor
__device__ __forceinline__ void mma(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(
          d),
      "r"(a), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   tma::smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tma::smem_u32(bar)) : "memory");
}
// 1-D bulk copy global -> shared with an L2 cache policy (createpolicy)
__device__ __forceinline__ void bulk_g2s_hint(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                              uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          tma::smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(tma::smem_u32(bar)), "l"(policy)
      : "memory");
}
// 3-D tensor-map copy global -> shared (box at coordinates x, y, z) with an L2 policy
__device__ __forceinline__ void tensor3_g2s_hint(void *dst, const void *tmap, int x, int y, int z, uint64_t *bar,
                                                 uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%2, %3, "
      "%4}], [%5], %6;" ::"r"(tma::smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(tma::smem_u32(bar)), "l"(policy)
      : "memory");
}
// L2 policy for data read once: evicted first, so that the coefficient stream does not
// push the spectrum (re-read by the FFT passes around the contraction) out of L2
__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Bounded wait with a suspend-time hint: a polling thread sleeps until the phase
// completes or kSuspendNs elapse, instead of spinning (the warps of this kernel wait most
// of the time and would otherwise take the issue slots of the working ones).  The poll
// limit of a launch is scaled down accordingly (a poll lasts up to kSuspendNs).
constexpr uint32_t kSuspendNs = 10000;
// the same, counting the polls into *polls when COUNT (measurement builds)
template <bool COUNT>
__device__ __forceinline__ bool wait_c(uint64_t *bar, uint32_t phase, long long lim, unsigned long long *polls) {
  for (long long i = 0; i < lim; ++i) {
    if constexpr (COUNT) ++*polls;
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(tma::smem_u32(bar)), "r"(phase), "r"(kSuspendNs)
        : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ bool wait(uint64_t *bar, uint32_t phase, long long lim) {
  for (long long i = 0; i < lim; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(tma::smem_u32(bar)), "r"(phase), "r"(kSuspendNs)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// A bounded wait whose outcome is the same in every lane of the warp (all lanes poll;
// the warp proceeds only if every lane saw the phase complete), so that the warp's
// .sync.aligned TMEM instructions never run divergently after a timeout.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t phase, long long lim) {
  return __all_sync(0xffffffffu, wait(bar, phase, lim)) != 0;
}
// FP16 split of a pair: hi = fp16(x) (11 significant bits), lo = fp16(x - hi); the
// pairs packed as the two halves of a 32-bit word (first element in the low half)
__device__ __forceinline__ void split_h2(float x0, float x1, uint32_t &hi, uint32_t &lo) {
  const __half2 h = __floats2half2_rn(x0, x1);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(__fsub_rn(x0, hf.x), __fsub_rn(x1, hf.y));
  hi = *reinterpret_cast<const uint32_t *>(&h);
  lo = *reinterpret_cast<const uint32_t *>(&l);
}
// 2^e as a float, e in [-126, 127]
__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((uint32_t)(127 + e) << 23); }
// exponent that scales a maximum m into [2^13, 2^14) (0 for m = 0), clamped to [-100, 100]
__device__ __forceinline__ int scale_exp(float m) {
  if (!(m > 0.f)) return 0;
  const int e = (int)((__float_as_uint(m) >> 23) & 0xFFu) - 127;
  const int x = 13 - e;
  return x < -100 ? -100 : (x > 100 ? 100 : x);
}

// x = hi + lo exactly: hi = x rounded to TF32 (10 fraction bits), lo = x - hi
__device__ __forceinline__ void split(float x, uint32_t &hi, uint32_t &lo) {
  const uint32_t h = (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
  hi = h;
  lo = __float_as_uint(__fsub_rn(x, __uint_as_float(h)));
}

}  // namespace tc

template <int NZ, int R, bool F16 = false>
struct TcCfg {
  static_assert(NZ % 8 == 0 && 3 * NZ <= 128, "one M = 128 tile of 3 Nz output rows; chunks of whole k-steps");
  static_assert(R >= 1 && R <= 2, "N = 16: 8 complex columns = 4 mirrors x R");
  static constexpr int N3 = 3 * NZ;
  static constexpr int CZ = R * N3;
  static constexpr int P = NZ * (NZ + 1) / 2;
  static constexpr int BS = 2 * NZ * (2 * NZ + 1);
  static constexpr int NBOX = NZ / 16;  // tensor-map boxes of 16 complex columns per full-block row
  static constexpr int NQ = (N3 + 31) / 32;        // TMEM lane quadrants holding rows
  static constexpr int RW = 4;                     // row warps per quadrant
  static constexpr int EPW = NZ / RW;              // complex entries of a chunk per row warp
  static constexpr int NROW = 4 * RW;              // warps 4 .. 4 + NROW - 1 (quadrant = warp % 4)
  static constexpr int NROWA = NQ * RW;            // of them, those with rows
  // B warps: 2, 3, the row warps without rows and (FP16) extra warps up to 8, one per
  // column, so that no B warp stages two columns of X while others stage one
  static constexpr int NB0 = 2 + NROW - NROWA;
  static constexpr int NXB = F16 && NB0 < 8 ? 8 - NB0 : 0;  // extra warps 4 + NROW ..
  static constexpr int NB = NB0 + NXB;
  // with two extra warps, the one that would share the MMA-issuing warp's scheduler
  // (warp index = 1 mod 4) stays idle: warps 4 + NROW and 4 + NROW + 2 stage B
  static constexpr int SKIP = NXB == 2 && (4 + NROW + 1) % 4 == 1 ? 1 : 0;
  static constexpr int WARPS = 4 + NROW + NXB + SKIP;
  static constexpr int THREADS = 32 * WARPS;
  static constexpr int NS = 3;                     // shared-memory stages
  static constexpr int KC = 2 * NZ;                // K of a chunk (real)
  // kind::tf32: one element per TMEM column and K = 8 per instruction; kind::f16: two per
  // column and K = 16, so a chunk takes half the columns and the ring can be twice as deep
  static constexpr int EPC = F16 ? 2 : 1;
  static constexpr int KSTEP = F16 ? 16 : 8;
  static constexpr int NKS = KC / KSTEP;           // k-steps of a chunk
  static constexpr int AHALF = KC / EPC;           // TMEM columns of the hi (or lo) part of a chunk
  static constexpr int ACOLS = 2 * AHALF;          // TMEM columns of a chunk buffer (hi, lo)
  static constexpr int NA = F16 ? 6 : 3;           // TMEM chunk buffers
  static constexpr int DCOL = NA * ACOLS;          // first accumulator column
  static constexpr int DBUF = 64;                  // per buffer: D1 (32 columns) and D2 (16), padded
  static constexpr int TCOLS = DCOL + 2 * DBUF <= 256 ? 256 : 512;
  static_assert(DCOL + 2 * DBUF <= 512, "TMEM");
  // stage layout (bytes): the packed triangles, then the full xz, yz rows as NBOX boxes
  // of [2 Nz rows][128 bytes] in the 128-byte swizzle (each 1024-byte aligned), then the
  // mirror vectors.  Element (row r, column b) of the full blocks (rows 0..Nz-1 xz,
  // Nz..2Nz-1 yz) sits at complex index FULLC + (b / 16) BOXC + 16 r +
  // 2 (((b % 16) / 2) ^ (r % 8)) + b % 2.
  static constexpr size_t TRI = (size_t)4 * P * 8;
  static constexpr size_t OFF_FULL = ((TRI + 1023) / 1024) * 1024;
  static constexpr size_t BOX = (size_t)2 * NZ * 128;
  static constexpr size_t FULL = NBOX * BOX;
  static constexpr size_t OFF_XR = OFF_FULL + FULL;
  static constexpr size_t XR = (size_t)4 * CZ * 8;
  static constexpr size_t STAGE = ((OFF_XR + XR + 1023) / 1024) * 1024;
  static constexpr int FULLC = (int)(OFF_FULL / 8), BOXC = (int)(BOX / 8);
  // B operand: per chunk and hi / lo, N = 16 rows of K = KC (core matrices 8 rows x 16
  // bytes of KPC elements): byte (n % 8) 16 + (n / 8) SBO + (k / KPC) 128 + (k % KPC) esz
  // FP16 at Nz = 32: a chunk's K row is 64 halves = 128 bytes, one atom of the 128-byte
  // swizzle (row n of an 8-row group at (n % 8) 128, its 16-byte chunk j at position
  // j ^ (n % 8); groups 1024 bytes apart; a k-step moves the start address by 32 bytes),
  // in which the column-at-a-time stores of the B warps hit distinct banks
  static constexpr int KPC = F16 ? 8 : 4;
  static constexpr bool SWZ = F16 && KC * 2 == 128;
  static constexpr uint32_t LBO = SWZ ? 16 : 128;
  static constexpr uint32_t SBO = SWZ ? 1024 : (uint32_t)(KC / KPC) * 128;
  static constexpr uint32_t KADV = SWZ ? 2 : 16;  // descriptor units (16 bytes) per k-step
  static constexpr uint64_t DESC_LAYOUT = SWZ ? (2ull << 61) : 0ull;
  static constexpr size_t BPART = (size_t)2 * SBO;            // one chunk, hi or lo
  static constexpr size_t BBUF = (size_t)3 * 2 * BPART;       // one wavenumber
  static constexpr size_t OFF_BAR = 0;                        // 32 mbarriers + the TMEM address
  static constexpr size_t OFF_STAGE = 1024;  // stages and boxes 1024-byte aligned (the swizzle atom)
  static constexpr size_t OFF_B = OFF_STAGE + NS * STAGE;
  static constexpr size_t SMEM = OFF_B + 2 * BBUF;
  static_assert(NZ % 16 == 0, "full-block rows in boxes of 16 complex (128 bytes)");
  static_assert(STAGE / 8 < 32768, "16-bit stage offsets");
  static constexpr uint32_t IDESC = F16 ? tc::idesc_f16(128, 16) : tc::idesc_tf32(128, 16);
  static constexpr uint32_t IDESC32 = F16 ? tc::idesc_f16(128, 32) : tc::idesc_tf32(128, 32);
};

// Written by the B warps for every column c of X of a wavenumber (before they release the
// B buffer), read by the row warps' epilogue (before they release the accumulators):
// output element (row) of column c at spec[off + row] (off < 0: no such column), its mirror
// sign flips (bit 0: the x component, bit 1: the y component) and, FP16, its exponent.
struct ColInfo {
  long long off;
  int flags, xe;
};

// Timing instrumentation (PROF = true only in measurement builds): per warp, clock64()
// cycles accumulated in the slots of TcProf, written to prof[(block * WARPS + warp) * 16],
// and the number of barrier polls of lane 0 in slot 8.
enum TcProf { kPWaitA = 0, kPWaitB = 1, kPWaitC = 2, kPWork = 3, kPWaitSt = 4, kPEpi = 5, kPTotal = 6, kPIters = 7 };

// F16: the kind::f16 instructions on a scaled two-way FP16 split (11 + 11 significant bits,
// as in the TF32 split): the block of wavenumber w is scaled by 2^qexp[w] and column c of
// X by 2^xe[c] (powers of two that bring the largest magnitudes into [2^13, 2^14), so
// that FP16 keeps every entry whose size matters to the product), and the outputs are
// scaled back exactly.  With F16, qf holds the blocks already scaled and split
// (launch_split_f16, 8 bytes per complex like the c64 blocks); the B warps split X.
template <int NZ, int R, bool F16 = false, bool PROF = false>
__global__ void __launch_bounds__(TcCfg<NZ, R, F16>::THREADS, 1)
    contract_tc_kernel(float2 *__restrict__ spec, const float2 *__restrict__ qf, int Nx, int Ny, int ldz, int *err,
                       long long lim_polls, const __grid_constant__ CUtensorMap tfull,
                       const int *__restrict__ qexp, unsigned long long *prof) {
  unsigned long long pt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  long long t_mark = 0;
  auto tic = [&]() {
    if constexpr (PROF) t_mark = clock64();
  };
  auto toc = [&](int slot) {
    if constexpr (PROF) {
      const long long t = clock64();
      pt[slot] += (unsigned long long)(t - t_mark);
      t_mark = t;
    }
  };
  const long long t_begin = PROF ? clock64() : 0;
  unsigned long long polls = 0;
  auto wt = [&](uint64_t *bar, uint32_t ph, long long l) -> bool { return tc::wait_c<PROF>(bar, ph, l, &polls); };
  auto wwt = [&](uint64_t *bar, uint32_t ph, long long l) -> bool {
    return __all_sync(0xffffffffu, tc::wait_c<PROF>(bar, ph, l, &polls)) != 0;
  };
  using Cfg = TcCfg<NZ, R, F16>;
  constexpr int N3 = Cfg::N3, CZ = Cfg::CZ, P = Cfg::P, BS = Cfg::BS, NS = Cfg::NS, NA = Cfg::NA;
  constexpr int KC = Cfg::KC, EPW = Cfg::EPW;
  extern __shared__ __align__(128) unsigned char sm_raw[];
  // the swizzled boxes need 1024-byte aligned destinations: the launch adds 1024 bytes
  unsigned char *sm = sm_raw + ((1024u - (tma::smem_u32(sm_raw) & 1023u)) & 1023u);
  uint64_t *bars = reinterpret_cast<uint64_t *>(sm + Cfg::OFF_BAR);
  // barrier block: full[4] empty[4] afull[8] aempty[8] bfull[2] bempty[2] dfull[2] dempty[2]
  // fin (33 x 8 bytes), the TMEM address at 384 and the column records at 512..1023 of
  // the 1024-byte block
  static_assert(NS <= 4 && NA <= 8, "barrier block");
  uint64_t *full = bars, *empty = bars + 4, *afull = bars + 8, *aempty = bars + 16;
  uint64_t *bfull = bars + 24, *bempty = bars + 26, *dfull = bars + 28, *dempty = bars + 30, *fin = bars + 32;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + Cfg::OFF_BAR + 384);
  // per wavenumber (ring of 4) and column of X: where its output goes and its scale
  ColInfo *cinfo = reinterpret_cast<ColInfo *>(sm + Cfg::OFF_BAR + 512);      // [4][8]
  unsigned char *stages = sm + Cfg::OFF_STAGE;
  unsigned char *bbuf = sm + Cfg::OFF_B;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nf = (Nx + 1) * (Ny + 1);
  const int w0 = blockIdx.x, gs = gridDim.x;
  const int n_it = w0 < nf ? (nf - 1 - w0) / gs + 1 : 0;
  // a poll lasts up to kSuspendNs: the poll limits are scaled so that the default wait
  // limit still ends a stuck wait within seconds (0 stays 0: give up at once)
  const long long lim = lim_polls > 0 ? (lim_polls >> 8 > 0 ? lim_polls >> 8 : 1) : 0;
  constexpr long long kDrain = kWaitLimit >> 8;

  if (warp == 0) {
    if (lane == 0) {
      for (int s = 0; s < NS; ++s) {
        tma::mbar_init(&full[s], 1);
        tma::mbar_init(&empty[s], Cfg::NROWA + Cfg::NB);
      }
      for (int c = 0; c < NA; ++c) {
        tma::mbar_init(&afull[c], Cfg::NROWA);
        tma::mbar_init(&aempty[c], 1);
      }
      for (int b = 0; b < 2; ++b) {
        tma::mbar_init(&bfull[b], Cfg::NB);
        tma::mbar_init(&bempty[b], 1);
        tma::mbar_init(&dfull[b], 1);
        tma::mbar_init(&dempty[b], Cfg::NROWA);
      }
      tma::mbar_init(fin, 1);
      tma::fence_mbar_init();
    }
    __syncwarp();
    tc::alloc(tslot, Cfg::TCOLS);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *tslot;
  // rows beyond 3 Nz must read as zero from every chunk buffer: the row warps zero the
  // A columns of all their lanes once (the unpacking later overwrites rows < 3 Nz)
  if (warp >= 4 && warp < 8) {
    const uint32_t zero[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const uint32_t tq = tbase + ((uint32_t)(32 * (warp & 3)) << 16);
    for (int c = 0; c < NA * Cfg::ACOLS; c += 8) tc::st8(tq + c, zero);
    tc::wait_st();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();

  bool ok = true;
  if (warp == 0) {
    // ---- producer ----
    const uint64_t once = tc::evict_first_policy();
    int issued = 0;
    for (int it = 0; it < n_it; ++it) {
      const int s = it % NS;
      tic();
      if (it >= NS && !wwt(&empty[s], (uint32_t)((it / NS - 1) & 1), lim)) {
        ok = false;
        break;
      }
      toc(kPWaitA);
      const int w = w0 + it * gs;
      const Mirrors mi = mirrors_of(w, Nx, Ny);
      const int nm = mi.nmx * mi.nmy;
      unsigned char *st = stages + (size_t)s * Cfg::STAGE;
      const float2 *q = qf + (size_t)w * BS;
      // (no proxy fence: nothing writes the stages through the generic proxy; their readers
      // hand them back through the empty barrier)
      if (lane == 0) tma::mbar_expect_tx(&full[s], (uint32_t)((size_t)BS * 8 + (size_t)nm * CZ * 8));
      __syncwarp();
      const int ncopy = 1 + Cfg::NBOX + nm;
      for (int j = lane; j < ncopy; j += 32) {
        if (j == 0) {
          tc::bulk_g2s_hint(st, q, (uint32_t)Cfg::TRI, &full[s], once);
        } else if (j <= Cfg::NBOX) {
          const int h = j - 1;
          tc::tensor3_g2s_hint(st + Cfg::OFF_FULL + (size_t)h * Cfg::BOX, &tfull, 16 * h, 0, w, &full[s], once);
        } else {
          const int m = j - 1 - Cfg::NBOX;
          const int mx = m % mi.nmx, my = m / mi.nmx;
          tma::bulk_g2s(st + Cfg::OFF_XR + (size_t)m * CZ * 8, spec + mi.pos(mx, my, Nx) * ldz, (uint32_t)(CZ * 8),
                        &full[s]);
        }
      }
      ++issued;
      toc(kPWork);
    }
    // drain: the last NS issues must land before the CTA exits
    for (int k = issued - NS > 0 ? issued - NS : 0; k < issued; ++k)
      wt(&full[k % NS], (uint32_t)((k / NS) & 1), kDrain);
  } else if (warp == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      // the descriptor's start-address field holds the byte address / 16 (shared memory
      // addresses stay below 2^18, so adding an offset / 16 never carries out of it): a
      // k-step (256 bytes further) adds 16
      const uint64_t bdesc = tc::sdesc(tma::smem_u32(bbuf), Cfg::LBO, Cfg::SBO) | Cfg::DESC_LAYOUT;
      for (int it = 0; it < n_it && ok; ++it) {
        const int bb = it & 1;
        tic();
        if (!wt(&bfull[bb], (uint32_t)((it >> 1) & 1), lim)) {
          ok = false;
          break;
        }
        toc(kPWaitA);
        if (it >= 2 && !wt(&dempty[bb], (uint32_t)(((it >> 1) - 1) & 1), lim)) {
          ok = false;
          break;
        }
        toc(kPWaitB);
        tc::fence_after();
        const uint32_t d1 = tbase + Cfg::DCOL + Cfg::DBUF * bb, d2 = d1 + 32;
        for (int beta = 0; beta < 3 && ok; ++beta) {
          const int g = 3 * it + beta, c = g % NA;
          tic();
          if (!wt(&afull[c], (uint32_t)((g / NA) & 1), lim)) {
            ok = false;
            break;
          }
          toc(kPWaitC);
          tc::fence_after();
          const uint32_t ahi = tbase + c * Cfg::ACOLS, alo = ahi + Cfg::AHALF;
          const uint64_t dh0 = bdesc + (((size_t)bb * Cfg::BBUF + (size_t)(2 * beta) * Cfg::BPART) >> 4);
#pragma unroll
          for (int ks = 0; ks < Cfg::NKS; ++ks) {
            const uint32_t acc = (beta | ks) != 0;
            tc::mma_k<F16>(d1, ahi + 8 * ks, dh0 + Cfg::KADV * ks, Cfg::IDESC32, acc);  // A_hi [B_hi | B_lo]
            tc::mma_k<F16>(d2, alo + 8 * ks, dh0 + Cfg::KADV * ks, Cfg::IDESC, acc);    // A_lo B_hi
          }
          tc::commit(&aempty[c]);
          toc(kPWork);
        }
        if (!ok) break;
        tc::commit(&bempty[bb]);
        tc::commit(&dfull[bb]);
      }
      // drain: every MMA issued above completes before TMEM is released
      tc::commit(fin);
      wt(fin, 0u, kDrain);
    }
  } else if (warp >= 4 && warp < 4 + Cfg::NROW && (warp & 3) < Cfg::NQ) {
    // ---- row warps: unpack, then the epilogue of the previous wavenumber ----
    const int q = warp & 3, jw = (warp - 4) >> 2;  // quadrant, column share
    const int row = 32 * q + lane;
    const bool live = row < N3;
    const int alpha = live ? row / NZ : 0, a = live ? row - alpha * NZ : 0;
    const uint32_t tq = tbase + ((uint32_t)(32 * q) << 16);
    // where this thread's entries of a block sit in a stage (complex index; the same for
    // every wavenumber), two 16-bit offsets per register; entries of zx = -xz^T and
    // zy = -yz^T are negated (chunks beta < 2 of the rows of z)
    uint32_t offp[3][EPW / 2];
#pragma unroll
    for (int beta = 0; beta < 3; ++beta) {
#pragma unroll
      for (int e = 0; e < EPW; ++e) {
        const int b = jw * EPW + e;
        int off;
        if ((alpha == 2) == (beta == 2)) {
          const int kind = alpha == beta ? alpha : 3;  // xx, yy, zz on the diagonal; xy off it
          const int lo = a < b ? a : b, hi = a < b ? b : a;
          off = kind * P + ((lo * (2 * NZ - 1) - lo * lo) >> 1) + hi;
        } else {
          // xz / yz direct (rows of x, y; columns of z) or transposed (rows of z)
          const int r = beta == 2 ? alpha * NZ + a : beta * NZ + b;
          const int cc = beta == 2 ? b : a;
          off = Cfg::FULLC + (cc >> 4) * Cfg::BOXC + 16 * r + ((((cc & 15) >> 1) ^ (r & 7)) << 1) + (cc & 1);
        }
        if (e & 1) offp[beta][e >> 1] |= (uint32_t)off << 16;
        else offp[beta][e >> 1] = (uint32_t)off;
      }
    }
    int ea_cur = 0, ea_prev = 0;  // F16: block exponents of the current and the previous wavenumber
    auto epilogue = [&](int e, int ea) -> bool {
      const int bb = e & 1;
      tic();
      if (!wwt(&dfull[bb], (uint32_t)((e >> 1) & 1), lim)) return false;
      toc(kPWaitC);
      tc::fence_after();
      const uint32_t dc = tq + Cfg::DCOL + Cfg::DBUF * bb;
      uint32_t v[12];
      tc::ld2(dc + 2 * jw, v[0], v[1]);            // A_hi B_hi: Y_r of columns 2 jw, 2 jw + 1
      tc::ld2(dc + 8 + 2 * jw, v[2], v[3]);        //            Y_i
      tc::ld2(dc + 16 + 2 * jw, v[4], v[5]);       // A_hi B_lo: Y_r
      tc::ld2(dc + 24 + 2 * jw, v[6], v[7]);       //            Y_i
      tc::ld2(dc + 32 + 2 * jw, v[8], v[9]);       // A_lo B_hi: Y_r
      tc::ld2(dc + 40 + 2 * jw, v[10], v[11]);     //            Y_i
      tc::wait_ld();
      toc(kPWaitSt);
      // read before dempty is released (the B warps reuse the ring later)
      const ColInfo ci[2] = {cinfo[(e & 3) * 8 + 2 * jw], cinfo[(e & 3) * 8 + 2 * jw + 1]};
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::arrive(&dempty[bb]);
      if (live) {
        const int fbit = alpha == 0 ? 1 : (alpha == 1 ? 2 : 0);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (ci[h].off >= 0) {
            float2 y = make_float2(__uint_as_float(v[h]) + (__uint_as_float(v[4 + h]) + __uint_as_float(v[8 + h])),
                                   __uint_as_float(v[2 + h]) + (__uint_as_float(v[6 + h]) + __uint_as_float(v[10 + h])));
            if (ci[h].flags & fbit) { y.x = -y.x; y.y = -y.y; }
            if constexpr (F16) {  // undo the scalings (exact powers of two)
              const float sc = tc::pow2f(-ea) * tc::pow2f(-ci[h].xe);
              y.x *= sc;
              y.y *= sc;
            }
            spec[ci[h].off + row] = y;
          }
        }
      }
      toc(kPEpi);
      return true;
    };
    for (int it = 0; it < n_it && ok; ++it) {
      const int s = it % NS;
      tic();
      if (!wwt(&full[s], (uint32_t)((it / NS) & 1), lim)) { ok = false; break; }
      toc(kPWaitA);
      const float2 *st = reinterpret_cast<const float2 *>(stages + (size_t)s * Cfg::STAGE);
      ea_prev = ea_cur;
      if constexpr (F16) ea_cur = __ldg(qexp + w0 + it * gs);
#pragma unroll
      for (int beta = 0; beta < 3; ++beta) {
        const int g = 3 * it + beta, c = g % NA;
        tic();
        if (g >= NA && !wwt(&aempty[c], (uint32_t)((g / NA - 1) & 1), lim)) {
          ok = false;
          break;
        }
        toc(kPWaitB);
        tc::fence_after();
        const bool neg = alpha == 2 && beta < 2;
        if constexpr (F16) {
          // entries (b, b + 1) as one word: re parts at K = b (columns AHALF-relative b / 2),
          // im parts at K = Nz + b.  The stage holds the blocks already scaled and split
          // (launch_split_f16: per complex (hi | lo << 16) of re, then of im), so a word is
          // two halves picked from two entries; the minus of zx, zy flips the sign bits.
          constexpr int HW = EPW / 2;
          uint32_t rh[HW], ih[HW], rl[HW], il[HW];
          const uint2 *st2 = reinterpret_cast<const uint2 *>(st);
          const uint32_t sgn = neg ? 0x80008000u : 0u;
#pragma unroll
          for (int e2 = 0; e2 < HW; ++e2) {
            const uint32_t o = offp[beta][e2];
            const uint2 m0 = live ? st2[o & 0xFFFFu] : make_uint2(0u, 0u);
            const uint2 m1 = live ? st2[o >> 16] : make_uint2(0u, 0u);
            rh[e2] = __byte_perm(m0.x, m1.x, 0x5410) ^ sgn;
            rl[e2] = __byte_perm(m0.x, m1.x, 0x7632) ^ sgn;
            ih[e2] = __byte_perm(m0.y, m1.y, 0x5410) ^ sgn;
            il[e2] = __byte_perm(m0.y, m1.y, 0x7632) ^ sgn;
          }
          const uint32_t ab = tq + c * Cfg::ACOLS + jw * HW;
          if constexpr (HW == 4) {
            tc::st4(ab, rh);
            tc::st4(ab + NZ / 2, ih);
            tc::st4(ab + Cfg::AHALF, rl);
            tc::st4(ab + Cfg::AHALF + NZ / 2, il);
          } else {
            tc::st2(ab, rh);
            tc::st2(ab + NZ / 2, ih);
            tc::st2(ab + Cfg::AHALF, rl);
            tc::st2(ab + Cfg::AHALF + NZ / 2, il);
          }
        } else {
          uint32_t rh[EPW], ih[EPW], rl[EPW], il[EPW];
#pragma unroll
          for (int e = 0; e < EPW; ++e) {
            const uint32_t off = (offp[beta][e >> 1] >> (16 * (e & 1))) & 0xFFFFu;
            float2 m = live ? st[off] : make_float2(0.f, 0.f);
            if (neg) { m.x = -m.x; m.y = -m.y; }
            tc::split(m.x, rh[e], rl[e]);
            tc::split(m.y, ih[e], il[e]);
          }
          const uint32_t ab = tq + c * Cfg::ACOLS + jw * EPW;
          if constexpr (EPW == 8) {
            tc::st8(ab, rh);
            tc::st8(ab + NZ, ih);
            tc::st8(ab + KC, rl);
            tc::st8(ab + KC + NZ, il);
          } else {
            tc::st4(ab, rh);
            tc::st4(ab + NZ, ih);
            tc::st4(ab + KC, rl);
            tc::st4(ab + KC + NZ, il);
          }
        }
        toc(kPWork);
      }
      if (!ok) break;
      // one wait for the stores of the three chunks, then the MMAs may read them
      tc::wait_st();
      toc(kPWork);
      tc::fence_before();
      __syncwarp();
      if (lane == 0) {
#pragma unroll
        for (int beta = 0; beta < 3; ++beta) tc::arrive(&afull[(3 * it + beta) % NA]);
      }
      __syncwarp();
      if (lane == 0) tc::arrive(&empty[s]);
      if (it >= 1 && !epilogue(it - 1, ea_prev)) { ok = false; break; }
    }
    if (ok && n_it >= 1) ok = epilogue(n_it - 1, ea_cur);
  } else if (Cfg::SKIP && warp == 4 + Cfg::NROW + 1) {
    // idle (keeps the MMA-issuing warp's scheduler free of a B warp)
  } else {
    // ---- B warps: warps 2, 3 and the row warps of quadrants without rows ----
    // One complex value x = X[col][beta Nz + b] (mirror signs applied) per thread and
    // step; it fills B rows b (which multiply M_r: (X_r | X_i)) and Nz + b (which
    // multiply M_i: (-X_i | X_r)) of columns col and 8 + col, hi and lo.  Threads of a
    // warp take (col, b % 4) of one core-matrix row group, so the stores of a warp fill
    // 128-byte core matrices without bank conflicts.
    const int bw = warp < 4 ? warp - 2
                 : warp >= 4 + Cfg::NROW ? Cfg::NB0 + (warp - 4 - Cfg::NROW) / (1 + Cfg::SKIP)
                                         : 2 + ((warp - 4) >> 2) * (4 - Cfg::NQ) + ((warp & 3) - Cfg::NQ);
    const int bt = bw * 32 + lane, nbt = Cfg::NB * 32;
    for (int it = 0; it < n_it && ok; ++it) {
      const int s = it % NS, bb = it & 1;
      tic();
      bool got = wwt(&full[s], (uint32_t)((it / NS) & 1), lim);
      toc(kPWaitA);
      if (got && it >= 2) got = wwt(&bempty[bb], (uint32_t)(((it >> 1) - 1) & 1), lim);
      toc(kPWaitB);
      if (!got) {
        ok = false;
        break;
      }
      const Mirrors mw = mirrors_of(w0 + it * gs, Nx, Ny);
      const int ncol = mw.nmx * mw.nmy * R;
      const float2 *xr = reinterpret_cast<const float2 *>(stages + (size_t)s * Cfg::STAGE + Cfg::OFF_XR);
      unsigned char *bp = bbuf + (size_t)bb * Cfg::BBUF;
      if constexpr (F16) {
        // Each B warp owns whole columns (col = bw, bw + NB, ...): lanes 2 g and 2 g + 1 take
        // the two halves (rows 8 g .. 8 g + 3 and 8 g + 4 .. 8 g + 7) of 8-row group g
        // (one component: Nz % 8 == 0), a warp reduction of the largest |re|, |im| gives
        // the column's scale exponent, and the scaled, split rows go out as 8-byte halves
        // of the 16-byte core-matrix rows of hi and lo.
        constexpr int OPC = N3 / 8;  // 8-row groups per column
        static_assert(2 * OPC <= 32, "two lanes per 8-row group");
        for (int col = bw; col < 8; col += Cfg::NB) {
          const bool have = lane < 2 * OPC;
          const int g8 = have ? lane >> 1 : 0, half = lane & 1;
          const int beta = (g8 * 8) / NZ, b0 = g8 * 8 - beta * NZ;
          float xs[4], ys[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) xs[j] = ys[j] = 0.f;
          uint32_t mx = 0u;
          if (have && col < ncol) {
            const int m = col / R, r = col - m * R;
            const int mxm = m % mw.nmx, mym = m / mw.nmx;
            const bool flip = (beta == 0 && mxm == 1) || (beta == 1 && mym == 1);
            const float4 *x4 = reinterpret_cast<const float4 *>(xr + (size_t)m * CZ + r * N3 + g8 * 8 + half * 4);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              const float4 u = x4[j];
              xs[2 * j] = flip ? -u.x : u.x;
              ys[2 * j] = flip ? -u.y : u.y;
              xs[2 * j + 1] = flip ? -u.z : u.z;
              ys[2 * j + 1] = flip ? -u.w : u.w;
              mx = max(mx, __float_as_uint(fmaxf(fmaxf(fabsf(u.x), fabsf(u.y)), fmaxf(fabsf(u.z), fabsf(u.w)))));
            }
          }
          const int ex = tc::scale_exp(__uint_as_float(__reduce_max_sync(0xffffffffu, mx)));
          if (lane == 0) {
            ColInfo ci = {-1, 0, ex};
            if (col < ncol) {
              const int m = col / R, r = col - m * R;
              const int mxm = m % mw.nmx, mym = m / mw.nmx;
              ci.off = (long long)mw.pos(mxm, mym, Nx) * ldz + r * N3;
              ci.flags = (mxm == 1 ? 1 : 0) | (mym == 1 ? 2 : 0);
            }
            cinfo[(it & 3) * 8 + col] = ci;
          }
          if (have) {
            const float sc = tc::pow2f(ex);
            uint2 rh, rl, ih, il;
            tc::split_h2(xs[0] * sc, xs[1] * sc, rh.x, rl.x);
            tc::split_h2(xs[2] * sc, xs[3] * sc, rh.y, rl.y);
            tc::split_h2(ys[0] * sc, ys[1] * sc, ih.x, il.x);
            tc::split_h2(ys[2] * sc, ys[3] * sc, ih.y, il.y);
            const uint2 nih = make_uint2(ih.x ^ 0x80008000u, ih.y ^ 0x80008000u);
            const uint2 nil = make_uint2(il.x ^ 0x80008000u, il.y ^ 0x80008000u);
            // rows k = b0 .. b0 + 7 (multiply M_r) and Nz + b0 .. (multiply M_i) of columns
            // col (Y_r) and 8 + col (Y_i, one SBO further); this lane's half at 8 half
            unsigned char *cb = bp + (size_t)(2 * beta) * Cfg::BPART + 8 * half;
            unsigned char *p0, *p1;
            if constexpr (Cfg::SWZ) {
              p0 = cb + (size_t)col * 128 + (size_t)(((b0 >> 3) ^ col) << 4);
              p1 = cb + (size_t)col * 128 + (size_t)((((NZ >> 3) + (b0 >> 3)) ^ col) << 4);
            } else {  // byte (n % 8) 16 + (n / 8) SBO + (k / 8) 128
              p0 = cb + (size_t)col * 16 + (size_t)(b0 >> 3) * 128;
              p1 = p0 + (size_t)(NZ >> 3) * 128;
            }
            constexpr size_t LO = Cfg::BPART;
            *reinterpret_cast<uint2 *>(p0) = rh;
            *reinterpret_cast<uint2 *>(p0 + LO) = rl;
            *reinterpret_cast<uint2 *>(p0 + Cfg::SBO) = ih;
            *reinterpret_cast<uint2 *>(p0 + Cfg::SBO + LO) = il;
            *reinterpret_cast<uint2 *>(p1) = nih;
            *reinterpret_cast<uint2 *>(p1 + LO) = nil;
            *reinterpret_cast<uint2 *>(p1 + Cfg::SBO) = rh;
            *reinterpret_cast<uint2 *>(p1 + Cfg::SBO + LO) = rl;
          }
        }
      } else {
        if (bt < 8) {
          const int col = bt;
          ColInfo ci = {-1, 0, 0};
          if (col < ncol) {
            const int m = col / R, r = col - m * R;
            const int mxm = m % mw.nmx, mym = m / mw.nmx;
            ci.off = (long long)mw.pos(mxm, mym, Nx) * ldz + r * N3;
            ci.flags = (mxm == 1 ? 1 : 0) | (mym == 1 ? 2 : 0);
          }
          cinfo[(it & 3) * 8 + col] = ci;
        }
      // entry e = ((beta * Nz + b) / 4) * 32 + (col * 4 + b % 4)
      for (int e = bt; e < 3 * NZ * 8; e += nbt) {
        const int col = (e >> 2) & 7, bq = e & 3, grp = e >> 5;
        const int zrow = grp * 4 + bq;  // beta * Nz + b
        const int beta = zrow / NZ, b = zrow - beta * NZ;
        float2 x = make_float2(0.f, 0.f);
        if (col < ncol) {
          const int m = col / R, r = col - m * R;
          const int mx = m % mw.nmx, my = m / mw.nmx;
          x = xr[(size_t)m * CZ + r * N3 + zrow];
          if ((beta == 0 && mx == 1) || (beta == 1 && my == 1)) { x.x = -x.x; x.y = -x.y; }
        }
        uint32_t rh, rl, ih, il;
        tc::split(x.x, rh, rl);
        tc::split(x.y, ih, il);
        // byte of (row k, column n) in a chunk part: (n % 8) 16 + (n / 8) SBO + (k / 4) 128 + (k % 4) 4
        unsigned char *p0 = bp + (size_t)(2 * beta) * Cfg::BPART + (size_t)col * 16 + (size_t)(b >> 2) * 128 + bq * 4;
        unsigned char *p1 = p0 + (size_t)(NZ >> 2) * 128;  // row Nz + b
        constexpr size_t LO = Cfg::BPART;
        *reinterpret_cast<uint32_t *>(p0) = rh;                            // (b, col): X_r
        *reinterpret_cast<uint32_t *>(p0 + LO) = rl;
        *reinterpret_cast<uint32_t *>(p0 + Cfg::SBO) = ih;                 // (b, 8 + col): X_i
        *reinterpret_cast<uint32_t *>(p0 + Cfg::SBO + LO) = il;
        *reinterpret_cast<uint32_t *>(p1) = ih ^ 0x80000000u;              // (Nz + b, col): -X_i
        *reinterpret_cast<uint32_t *>(p1 + LO) = il ^ 0x80000000u;
        *reinterpret_cast<uint32_t *>(p1 + Cfg::SBO) = rh;                 // (Nz + b, 8 + col): X_r
        *reinterpret_cast<uint32_t *>(p1 + Cfg::SBO + LO) = rl;
      }
      }
      toc(kPWork);
      tma::fence_proxy_async();  // the MMA reads B through the async proxy
      __syncwarp();
      if (lane == 0) {
        tc::arrive(&bfull[bb]);
        tc::arrive(&empty[s]);
      }
      toc(kPEpi);
    }
  }
  if (!ok && lane == 0) atomicExch(err, kContractTimeout);
  if constexpr (PROF) {
    if (prof && lane == 0) {
      pt[kPTotal] = (unsigned long long)(clock64() - t_begin);
      pt[kPIters] = (unsigned long long)n_it;
      for (int k = 0; k < 8; ++k) prof[((size_t)blockIdx.x * Cfg::WARPS + warp) * 16 + k] = pt[k];
      prof[((size_t)blockIdx.x * Cfg::WARPS + warp) * 16 + 8] = polls;
    }
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::dealloc(tbase, Cfg::TCOLS);
}

}  // namespace ie
