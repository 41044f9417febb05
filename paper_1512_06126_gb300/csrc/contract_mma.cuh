// Wavenumber contraction (step 2 of the FFT product, Sect. 3.3) on the tensor cores:
// bulk copies (cp.async.bulk) into shared memory feeding warp-level TF32 MMAs
// (mma.sync m16n8k8) with the 3xTF32 split, for compile-time Nz (a multiple of 16) and
// R <= 2 right-hand sides.
//
// Per wavenumber the 3Nz x 3Nz complex block M is applied to the X of up to four
// mirror wavenumbers x R right-hand sides (8 columns at most, one n-tile).  As real
// products: Y_r = M_r X_r - M_i X_i, Y_i = M_r X_i + M_i X_r, so every warp owns 16
// complex rows of M and issues, per k-step of 8, the four products M_{r,i} X_{r,i};
// each thread then holds Y_r and Y_i of the same (row, column) positions.  Every
// operand x is split into x_hi = tf32(x) and x_lo = tf32(x - x_hi) and a product is
// taken as A_hi B_hi + (A_hi B_lo + A_lo B_hi) (the dropped A_lo B_lo is ~2^-22 of
// it), so the result keeps FP32 accuracy; the two parts accumulate separately in
// FP32.  The split (Veltkamp) runs on the FP32 pipe.
//
// Two kernels:
//  * contract_mma_kernel (warp-specialised): one producer warp issues the copies of
//    the next wavenumbers into a ring of slots; the compute warps read the fragments
//    where the copies land, with no unpacking pass, and hand a slot back through an
//    mbarrier: the packed triangles of the symmetric xx, yy, zz, xy blocks in one copy
//    (element (a, b) at f(min) + max, f(i) = i (2 Nz - 1 - i) / 2, the row-major upper
//    triangle), the rows of the full xz, yz blocks one copy each at a stride of Nz + 4,
//    and every column of X (mirror x right-hand side) one copy each at a stride of
//    3 Nz + 4.  Both strides are 4 (mod 16) complex, so the fragment loads of a
//    half-warp (4 rows x 4 columns, direct or transposed) fall on distinct banks.
//  * contract_mma_unpack_kernel: the one-slot ring of contract_tma.cuh; all warps
//    unpack the block into six Nz x (Nz + 4) matrices (the triangles in diagonal
//    order, so that the stores spread over the banks) and stage X in fragment order.
// The component signs of the mirrors (Lemma 2) and of zx = -xz^T, zy = -yz^T (Lemma 1)
// are applied to X.
#pragma once
#include "contract_tma.cuh"

namespace ie {

template <int NZ, int R, int NSTAGE>
struct MmaCfg {
  static_assert(NZ % 16 == 0 && NZ <= 48, "row tiles of 16 must not straddle the Nz sub-blocks");
  static_assert(R >= 1 && R <= 2, "one n-tile of 8 columns: 4 mirrors x R <= 8");
  static constexpr int N3 = 3 * NZ;
  static constexpr int CZ = R * N3;
  static constexpr int P = NZ * (NZ + 1) / 2;
  static constexpr int BS = 2 * NZ * (2 * NZ + 1);
  static constexpr int MAXC = 4 * R;
  static constexpr int LDF = NZ + 4;              // full-block row stride (= 4 mod 16)
  static constexpr int LDX = N3 + 4;              // X column stride (= 4 mod 16)
  static constexpr int WARPS = N3 / 16;           // compute warps: one 16-row tile each
  static constexpr int THREADS = (WARPS + 1) * 32;  // + the producer warp
  // one slot (complex offsets): packed triangles, padded full rows, padded X columns
  static constexpr int OFF_F = 4 * P;
  static constexpr int OFF_X = OFF_F + 2 * NZ * LDF;
  static constexpr int SLOT = OFF_X + MAXC * LDX;
  static constexpr size_t OFF_BAR = 0;
  static constexpr size_t OFF_SLOT = 128;
  static constexpr size_t SMEM = OFF_SLOT + (size_t)NSTAGE * SLOT * 8;
  static_assert((OFF_F * 8) % 16 == 0 && (OFF_X * 8) % 16 == 0 && (SLOT * 8) % 16 == 0, "bulk copy alignment");
  static_assert(NSTAGE <= 8, "full and empty barriers of every slot in 128 bytes");
  // resident CTAs per SM that shared memory allows (at most 3): the register budget
  static constexpr int FIT = (int)((227 * 1024) / (SMEM + 1024));
  static constexpr int MINB = FIT > 3 ? 3 : (FIT < 1 ? 1 : FIT);
};

namespace mma {

// x = hi + lo exactly, hi with at most 11 significant bits (a TF32 value, so the MMA
// reads it unchanged): Veltkamp's splitting with the factor 2^13 + 1 of the 24-bit
// significand, in explicitly rounded FP32 operations (no contraction into FMAs, which
// would break the exactness).  lo keeps at most 13 bits; the MMA reads its leading 11,
// an error below 2^-22 |x|.
__device__ __forceinline__ void split(float x, uint32_t &hi, uint32_t &lo) {
  const float t = __fmul_rn(8193.0f, x);
  const float h = __fsub_rn(t, __fsub_rn(t, x));
  hi = __float_as_uint(h);
  lo = __float_as_uint(__fsub_rn(x, h));
}

// d += a b  (m16n8k8, A row-major 16 x 8, B column-major 8 x 8, FP32 accumulate)
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// The 12 MMAs of one k-step from split operands (r/i: real and imaginary part, h/l:
// hi and lo).
__device__ __forceinline__ void mma12(float (&acc)[2][2][2][4], const uint32_t (&arh)[4], const uint32_t (&arl)[4],
                                      const uint32_t (&aih)[4], const uint32_t (&ail)[4], const uint32_t (&brh)[2],
                                      const uint32_t (&brl)[2], const uint32_t (&bih)[2], const uint32_t (&bil)[2]) {
  mma_tf32(acc[0][0][0], arh, brh);
  mma_tf32(acc[0][1][0], arh, bih);
  mma_tf32(acc[1][0][0], aih, brh);
  mma_tf32(acc[1][1][0], aih, bih);
  mma_tf32(acc[0][0][1], arh, brl);
  mma_tf32(acc[0][1][1], arh, bil);
  mma_tf32(acc[1][0][1], aih, brl);
  mma_tf32(acc[1][1][1], aih, bil);
  mma_tf32(acc[0][0][1], arl, brh);
  mma_tf32(acc[0][1][1], arl, bih);
  mma_tf32(acc[1][0][1], ail, brh);
  mma_tf32(acc[1][1][1], ail, bih);
}

// A of a k-step: M rows (16 x 8 complex: m[0] (g, t), m[1] (g + 8, t), m[2] (g, t + 4),
// m[3] (g + 8, t + 4)), split
__device__ __forceinline__ void split_a(const float2 (&m)[4], uint32_t (&arh)[4], uint32_t (&arl)[4],
                                        uint32_t (&aih)[4], uint32_t (&ail)[4]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    split(m[c].x, arh[c], arl[c]);
    split(m[c].y, aih[c], ail[c]);
  }
}

// One k-step with B = X (8 x 8 complex: x[0] (t, g), x[1] (t + 4, g)) split here.
__device__ __forceinline__ void kstep(float (&acc)[2][2][2][4], const float2 (&m)[4], const float2 (&x)[2]) {
  uint32_t arh[4], arl[4], aih[4], ail[4], brh[2], brl[2], bih[2], bil[2];
  split_a(m, arh, arl, aih, ail);
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    split(x[c].x, brh[c], brl[c]);
    split(x[c].y, bih[c], bil[c]);
  }
  mma12(acc, arh, arl, aih, ail, brh, brl, bih, bil);
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tma::smem_u32(bar)) : "memory");
}

}  // namespace mma

template <int NZ, int R, int NSTAGE>
__global__ void __launch_bounds__(MmaCfg<NZ, R, NSTAGE>::THREADS, MmaCfg<NZ, R, NSTAGE>::MINB)
    contract_mma_kernel(float2 *__restrict__ spec, const float2 *__restrict__ qf, int Nx, int Ny, int ldz, int *err,
                        long long lim) {
  using Cfg = MmaCfg<NZ, R, NSTAGE>;
  constexpr int N3 = Cfg::N3, CZ = Cfg::CZ, P = Cfg::P, BS = Cfg::BS, LDF = Cfg::LDF, LDX = Cfg::LDX;
  constexpr int SLOT = Cfg::SLOT, OFF_F = Cfg::OFF_F, OFF_X = Cfg::OFF_X;
  constexpr int WARPS = Cfg::WARPS;
  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t *full = reinterpret_cast<uint64_t *>(sm + Cfg::OFF_BAR);  // copies landed
  uint64_t *empty = full + NSTAGE;                                    // compute warps done
  float2 *slots = reinterpret_cast<float2 *>(sm + Cfg::OFF_SLOT);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nf = (Nx + 1) * (Ny + 1);
  uint64_t *bar = full;

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      tma::mbar_init(&full[s], 1);
      tma::mbar_init(&empty[s], WARPS);
    }
    tma::fence_mbar_init();
  }
  __syncthreads();

  // producer warp: the copies of wavenumber w into slot s (lane 0 registers the bytes
  // first, then the lanes share the 1 + 2 Nz + (mirrors x R) copies)
  auto issue = [&](int w, int s) {
    const Mirrors mi = mirrors_of(w, Nx, Ny);
    const int nm = mi.nmx * mi.nmy;
    float2 *dst = slots + (size_t)s * SLOT;
    const float2 *q = qf + (size_t)w * BS;
    tma::fence_proxy_async();
    if (lane == 0) tma::mbar_expect_tx(&bar[s], (uint32_t)((size_t)BS * 8 + (size_t)nm * CZ * 8));
    __syncwarp();
    const int ncopy = 1 + 2 * NZ + nm * R;
    for (int j = lane; j < ncopy; j += 32) {
      if (j == 0) {
        tma::bulk_g2s(dst, q, (uint32_t)(4 * P * 8), &bar[s]);
      } else if (j <= 2 * NZ) {
        const int i = j - 1;
        tma::bulk_g2s(dst + OFF_F + i * LDF, q + 4 * P + i * NZ, (uint32_t)(NZ * 8), &bar[s]);
      } else {
        const int c = j - 1 - 2 * NZ;  // column m R + r
        const int m = c / R, r = c - m * R;
        const int mx = m % mi.nmx, my = m / mi.nmx;
        tma::bulk_g2s(dst + OFF_X + c * LDX, spec + mi.pos(mx, my, Nx) * ldz + r * N3, (uint32_t)(N3 * 8), &bar[s]);
      }
    }
  };

  const int w0 = blockIdx.x;
  if (warp == WARPS) {
    // producer: slot s of use u waits until the compute warps released use u - 1
    int it = 0;
    for (int w = w0; w < nf; w += gridDim.x, ++it) {
      const int s = it % NSTAGE;
      if (it >= NSTAGE && !tma::mbar_wait_bounded(&empty[s], (uint32_t)((it / NSTAGE - 1) & 1), lim)) {
        if (lane == 0) atomicExch(err, kContractTimeout);
        break;
      }
      issue(w, s);
    }
    // drain: the copies of the last NSTAGE issues must land before the CTA exits, even
    // where the compute warps gave up on them
    const int n_issued = it;
    for (int k = n_issued - NSTAGE > 0 ? n_issued - NSTAGE : 0; k < n_issued; ++k)
      tma::mbar_wait_bounded(&full[k % NSTAGE], (uint32_t)((k / NSTAGE) & 1), kWaitLimit);
    return;
  }

  // this warp's rows: row0 .. row0 + 15 of M, inside sub-block alpha at a0
  const int g = lane >> 2, t = lane & 3;
  const int row0 = warp * 16;
  const int alpha = row0 / NZ, a0 = row0 - alpha * NZ;
  const int A0 = a0 + g, A1 = a0 + g + 8;
  // column g of B: mirror m = g / R, right-hand side g % R
  const int mcol = g / R;

  int it = 0;
  for (int w = w0; w < nf; w += gridDim.x, ++it) {
    const int s = it % NSTAGE;
    const uint32_t phase = (uint32_t)((it / NSTAGE) & 1);
    if (!tma::mbar_wait_bounded(&full[s], phase, lim)) {
      // the producer warp drains the copies it issued before the CTA exits
      if (lane == 0) atomicExch(err, kContractTimeout);
      return;
    }
    const Mirrors mw = mirrors_of(w, Nx, Ny);
    const int nmx = mw.nmx;
    const int ncol = mw.nmx * mw.nmy * R;
    const float2 *slot = slots + (size_t)s * SLOT;
    const bool valid = g < ncol;
    const int cmx = valid ? mcol % nmx : 0, cmy = valid ? mcol / nmx : 0;
    // (lanes past the staged columns read column 0, inside the slot, and use zero)
    const float2 *xcol = slot + OFF_X + (valid ? g : 0) * LDX + t;

    float acc[2][2][2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[i][j][h][c] = 0.f;

#pragma unroll
    for (int beta = 0; beta < 3; ++beta) {
      // sub-block M[alpha][beta]: symmetric (xx, yy, zz, xy) or full (xz, yz; read
      // transposed and negated in the rows of z)
      const bool full = (alpha == 2) != (beta == 2);
      const bool trn = alpha == 2 && beta < 2;
      // X signs: the mirror component flip and the minus of zx, zy
      float sg = ((beta == 0 && cmx == 1) || (beta == 1 && cmy == 1)) ? -1.f : 1.f;
      if (trn) sg = -sg;
      if (full) {
        const int kind = beta == 2 ? alpha : beta;  // xz: 0, yz: 1
        const float2 *fb = slot + OFF_F + kind * NZ * LDF;
        // element (a, b): direct at a LDF + b, transposed at b LDF + a
        const int rs = trn ? 1 : LDF, cs = trn ? LDF : 1;
        const float2 *p0 = fb + A0 * rs + t * cs;
#pragma unroll 2
        for (int bb = 0; bb < NZ; bb += 8) {
          const float2 *p = p0 + bb * cs;
          float2 m[4], x[2];
          m[0] = p[0];
          m[1] = p[8 * rs];
          m[2] = p[4 * cs];
          m[3] = p[8 * rs + 4 * cs];
          const float2 x0 = xcol[beta * NZ + bb], x1 = xcol[beta * NZ + bb + 4];
          x[0] = valid ? make_float2(sg * x0.x, sg * x0.y) : make_float2(0.f, 0.f);
          x[1] = valid ? make_float2(sg * x1.x, sg * x1.y) : make_float2(0.f, 0.f);
          mma::kstep(acc, m, x);
        }
      } else {
        const int kind = alpha == beta ? alpha : 3;  // xx, yy, zz, xy
        const float2 *sb = slot + kind * P;
#pragma unroll 2
        for (int bb = 0; bb < NZ; bb += 8) {
          const int B0 = bb + t, B1 = bb + t + 4;
          auto at = [&](int a, int b) {
            const int lo = a < b ? a : b, hi = a < b ? b : a;
            return sb[((lo * (2 * NZ - 1) - lo * lo) >> 1) + hi];
          };
          float2 m[4], x[2];
          m[0] = at(A0, B0);
          m[1] = at(A1, B0);
          m[2] = at(A0, B1);
          m[3] = at(A1, B1);
          const float2 x0 = xcol[beta * NZ + bb], x1 = xcol[beta * NZ + bb + 4];
          x[0] = valid ? make_float2(sg * x0.x, sg * x0.y) : make_float2(0.f, 0.f);
          x[1] = valid ? make_float2(sg * x1.x, sg * x1.y) : make_float2(0.f, 0.f);
          mma::kstep(acc, m, x);
        }
      }
    }
    // D fragment: c -> row g + 8 (c >> 1), column 2 t + (c & 1)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int col = 2 * t + (c & 1);
      if (col < ncol) {
        const int row = row0 + g + 8 * (c >> 1);
        const int m = col / R, r = col - m * R;
        const int mx = m % nmx, my = m / nmx;
        const float rr = acc[0][0][0][c] + acc[0][0][1][c], ii = acc[1][1][0][c] + acc[1][1][1][c];
        const float ri = acc[0][1][0][c] + acc[0][1][1][c], ir = acc[1][0][0][c] + acc[1][0][1][c];
        float2 v = make_float2(rr - ii, ri + ir);
        if ((alpha == 0 && mx == 1) || (alpha == 1 && my == 1)) { v.x = -v.x; v.y = -v.y; }
        spec[mw.pos(mx, my, Nx) * ldz + r * N3 + row] = v;
      }
    }
    // this warp is done with slot s
    __syncwarp();
    if (lane == 0) mma::mbar_arrive(&empty[s]);
  }
}

template <int NZ, int R>
struct MmaUnpackCfg {
  static_assert(NZ % 16 == 0 && NZ <= 48, "row tiles of 16 must not straddle the Nz sub-blocks");
  static_assert(R >= 1 && R <= 2, "one n-tile of 8 columns: 4 mirrors x R <= 8");
  static constexpr int N3 = 3 * NZ;
  static constexpr int CZ = R * N3;
  static constexpr int P = NZ * (NZ + 1) / 2;
  static constexpr int BS = 2 * NZ * (2 * NZ + 1);
  static constexpr int LD = NZ + 4;               // = 4 (mod 16)
  static constexpr int WARPS = N3 / 16;
  static constexpr int THREADS = WARPS * 32;
  static constexpr int KS = N3 / 8;
  static constexpr size_t OFF_BAR = 0;
  static constexpr size_t OFF_RAW = 128;
  static constexpr size_t RAW_BYTES = (size_t)BS * 8;
  // the mirror vectors at a stride of CZ + 4 complex (= 4 mod 16 for the staging reads)
  static constexpr int LDXR = CZ + 4;
  static constexpr size_t XRAW_BYTES = (size_t)4 * LDXR * 8;
  static constexpr size_t OFF_XRAW = OFF_RAW + RAW_BYTES;
  static constexpr size_t OFF_BLK = OFF_XRAW + XRAW_BYTES;
  static constexpr size_t BLK_BYTES = (size_t)6 * NZ * LD * 8;
  static constexpr size_t OFF_XS = OFF_BLK + BLK_BYTES;
  // X split, in two planes (hi, lo), each [k-step][lane] of 16 bytes
  static constexpr size_t XS_PLANE = (size_t)KS * 32 * 16;
  static constexpr size_t XS_BYTES = 2 * XS_PLANE;
  static constexpr size_t OFF_TRI = OFF_XS + XS_BYTES;
  static constexpr size_t SMEM = OFF_TRI + (size_t)P * 4;
};

template <int NZ, int R>
__global__ void __launch_bounds__(MmaUnpackCfg<NZ, R>::THREADS)
    contract_mma_unpack_kernel(float2 *__restrict__ spec, const float2 *__restrict__ qf, int Nx, int Ny, int ldz,
                               int *err, long long lim) {
  using Cfg = MmaUnpackCfg<NZ, R>;
  constexpr int N3 = Cfg::N3, CZ = Cfg::CZ, P = Cfg::P, BS = Cfg::BS, LD = Cfg::LD;
  constexpr int THREADS = Cfg::THREADS;
  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + Cfg::OFF_BAR);
  float2 *raw = reinterpret_cast<float2 *>(sm + Cfg::OFF_RAW);
  float2 *xraw = reinterpret_cast<float2 *>(sm + Cfg::OFF_XRAW);
  float2 *blk = reinterpret_cast<float2 *>(sm + Cfg::OFF_BLK);
  uint4 *xs = reinterpret_cast<uint4 *>(sm + Cfg::OFF_XS);
  uint32_t *tri = reinterpret_cast<uint32_t *>(sm + Cfg::OFF_TRI);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nf = (Nx + 1) * (Ny + 1);

  // triangle entries in diagonal order: entry S(d) + a is (a, a + d), S(d) = sum_{d' < d}
  // (NZ - d'); packed (row-major upper triangle) index a NZ - a (a - 1) / 2 + d
  for (int d = tid; d < NZ; d += THREADS) {
    const int s0 = d * NZ - d * (d - 1) / 2;
    for (int a = 0; a + d < NZ; ++a)
      tri[s0 + a] = (uint32_t)((a * NZ - a * (a - 1) / 2 + d) << 12 | a << 6 | (a + d));
  }
  if (tid == 0) {
    tma::mbar_init(&bar[0], 1);
    tma::fence_mbar_init();
  }
  __syncthreads();

  auto issue = [&](int w) {
    const Mirrors mi = mirrors_of(w, Nx, Ny);
    const int nm = mi.nmx * mi.nmy;
    tma::fence_proxy_async();
    tma::mbar_expect_tx(&bar[0], (uint32_t)(Cfg::RAW_BYTES + (size_t)nm * CZ * 8));
    tma::bulk_g2s(raw, qf + (size_t)w * BS, (uint32_t)Cfg::RAW_BYTES, &bar[0]);
    for (int m = 0; m < nm; ++m) {
      const int mx = m % mi.nmx, my = m / mi.nmx;
      tma::bulk_g2s(xraw + (size_t)m * Cfg::LDXR, spec + mi.pos(mx, my, Nx) * ldz, (uint32_t)(CZ * 8), &bar[0]);
    }
  };

  const int w0 = blockIdx.x;
  if (tid == 0 && w0 < nf) issue(w0);

  // this warp's rows: row0 .. row0 + 15 of M, inside sub-block alpha at a0
  const int g = lane >> 2, t = lane & 3;
  const int row0 = warp * 16;
  const int alpha = row0 / NZ, a0 = row0 - alpha * NZ;
  // per beta: the matrix holding M[alpha][beta], read directly (element (a, b) at
  // a LD + b) or transposed (at b LD + a, negated): rows alpha < 2 read xx, xy, xz /
  // xy, yy, yz; alpha = 2 reads -xz^T, -yz^T, zz
  const float2 *Axx = blk, *Ayy = blk + NZ * LD, *Azz = blk + 2 * NZ * LD, *Axy = blk + 3 * NZ * LD;
  const float2 *Axz = blk + 4 * NZ * LD, *Ayz = blk + 5 * NZ * LD;
  const float2 *mb[3];
  if (alpha == 0) { mb[0] = Axx; mb[1] = Axy; mb[2] = Axz; }
  else if (alpha == 1) { mb[0] = Axy; mb[1] = Ayy; mb[2] = Ayz; }
  else { mb[0] = Axz; mb[1] = Ayz; mb[2] = Azz; }
  const bool tr = alpha == 2;  // betas 0, 1 transposed and negated

  int it = 0;
  for (int w = w0; w < nf; w += gridDim.x, ++it) {
    if (!tma::mbar_wait_bounded(&bar[0], (uint32_t)(it & 1), lim)) {
      if (tid == 0) atomicExch(err, kContractTimeout);
      // drain the one copy in flight
      tma::mbar_wait_bounded(&bar[0], (uint32_t)(it & 1), kWaitLimit);
      return;
    }
    const Mirrors mw = mirrors_of(w, Nx, Ny);
    const int nmx = mw.nmx;
    const int ncol = mw.nmx * mw.nmy * R;
    // symmetric kinds xx, yy, zz, xy: both triangles
    for (int e = tid; e < 4 * P; e += THREADS) {
      const int kind = e / P;
      const uint32_t ent = tri[e - kind * P];
      const int p = ent >> 12, a = (ent >> 6) & 63, b = ent & 63;
      const float2 v = raw[kind * P + p];
      float2 *m = blk + kind * NZ * LD;
      m[a * LD + b] = v;
      m[b * LD + a] = v;
    }
    // full kinds xz, yz (row-major)
    for (int e = tid; e < 2 * NZ * NZ; e += THREADS) {
      const int kind = e / (NZ * NZ);
      const int r2 = e - kind * NZ * NZ;
      const int a = r2 / NZ, b = r2 - a * NZ;
      blk[(4 + kind) * NZ * LD + a * LD + b] = raw[4 * P + e];
    }
    // X split and in fragment order: entry (k-step ks, lane 4 col + t) of the hi plane
    // holds re, im of row 8 ks + t and re, im of row 8 ks + t + 4 of column col (the lo
    // plane the same for the lo parts), with the mirror component signs; zero beyond
    // ncol.  One thread per entry, 16-byte stores.
    for (int e = tid; e < Cfg::KS * 32; e += THREADS) {
      const int ks = e >> 5, col = (e >> 2) & 7, t = e & 3;
      const int k0 = ks * 8 + t;  // rows k0 and k0 + 4 lie in the same component (NZ % 8 == 0)
      float2 v0 = make_float2(0.f, 0.f), v1 = v0;
      if (col < ncol) {
        const int m = col / R, r = col - m * R;
        const int mx = m % nmx, my = m / nmx;
        const int comp = k0 / NZ;
        const float2 *xp = xraw + (size_t)m * Cfg::LDXR + r * N3 + k0;
        v0 = xp[0];
        v1 = xp[4];
        if ((comp == 0 && mx == 1) || (comp == 1 && my == 1)) {
          v0 = make_float2(-v0.x, -v0.y);
          v1 = make_float2(-v1.x, -v1.y);
        }
      }
      uint4 h, l;
      mma::split(v0.x, h.x, l.x);
      mma::split(v0.y, h.y, l.y);
      mma::split(v1.x, h.z, l.z);
      mma::split(v1.y, h.w, l.w);
      xs[e] = h;
      xs[Cfg::KS * 32 + e] = l;
    }
    __syncthreads();
    // the raw slot is consumed: refill it with wavenumber w + gridDim.x
    if (tid == 0 && w + (int)gridDim.x < nf) issue(w + gridDim.x);
    float acc[2][2][2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[i][j][h][c] = 0.f;
    const uint4 *xfh = xs, *xfl = xs + Cfg::KS * 32;
#pragma unroll
    for (int beta = 0; beta < 3; ++beta) {
      const bool trb = tr && beta < 2;
      const uint32_t neg = trb ? 0x80000000u : 0u;  // the minus of zx, zy: flip the signs of X
      // element (a0 + g + 8 i, b + t + 4 j) of this sub-block at p + 8 i rs + 4 j cs
      const int rs = trb ? 1 : LD, cs = trb ? LD : 1;
      const float2 *p0 = mb[beta] + (a0 + g) * rs + t * cs;
#pragma unroll
      for (int bb = 0; bb < NZ; bb += 8) {
        const float2 *p = p0 + bb * cs;
        float2 m[4];
        m[0] = p[0];
        m[1] = p[8 * rs];
        m[2] = p[4 * cs];
        m[3] = p[8 * rs + 4 * cs];
        const int ks = beta * (NZ / 8) + bb / 8;
        const uint4 xh = xfh[ks * 32 + lane], xl = xfl[ks * 32 + lane];
        const uint32_t brh[2] = {xh.x ^ neg, xh.z ^ neg}, bih[2] = {xh.y ^ neg, xh.w ^ neg};
        const uint32_t brl[2] = {xl.x ^ neg, xl.z ^ neg}, bil[2] = {xl.y ^ neg, xl.w ^ neg};
        uint32_t arh[4], arl[4], aih[4], ail[4];
        mma::split_a(m, arh, arl, aih, ail);
        mma::mma12(acc, arh, arl, aih, ail, brh, brl, bih, bil);
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int col = 2 * t + (c & 1);
      if (col < ncol) {
        const int row = row0 + g + 8 * (c >> 1);
        const int m = col / R, r = col - m * R;
        const int mx = m % nmx, my = m / nmx;
        const float rr = acc[0][0][0][c] + acc[0][0][1][c], ii = acc[1][1][0][c] + acc[1][1][1][c];
        const float ri = acc[0][1][0][c] + acc[0][1][1][c], ir = acc[1][0][0][c] + acc[1][0][1][c];
        float2 v = make_float2(rr - ii, ri + ir);
        if ((alpha == 0 && mx == 1) || (alpha == 1 && my == 1)) { v.x = -v.x; v.y = -v.y; }
        spec[mw.pos(mx, my, Nx) * ldz + r * N3 + row] = v;
      }
    }
    __syncthreads();
  }
}

// contract_mma_mat_kernel: the block of a wavenumber one Nz x Nz matrix M[alpha][beta]
// at a time (nine sub-steps; the symmetric xy and the full xz, yz serve two of them
// each and are copied twice, the second time mostly from L2), so that a CTA stages
// one packed matrix and one unpacked one: at Nz = 64 the whole unpacked block (6 x 64 x
// 68 complex) does not fit in shared memory with its staging, one matrix does, twice
// per SM.  Per sub-step one thread copies the packed matrix (a bulk copy, the next
// sub-step's issued as soon as the current one is unpacked), all warps unpack it, and
// warp (row tile, K half) applies it to its half of X's component beta with the
// 3xTF32 MMAs, accumulating over beta in registers; after beta = 2 the two K halves
// meet in shared memory and component alpha of Y is stored.  X is staged once per
// wavenumber.
template <int NZ, int R>
struct MmaMatCfg {
  static_assert(NZ % 16 == 0 && NZ <= 64, "row tiles of 16; at most 64 layers");
  static_assert(R >= 1 && R <= 2, "one n-tile of 8 columns: 4 mirrors x R <= 8");
  static constexpr int N3 = 3 * NZ;
  static constexpr int CZ = R * N3;
  static constexpr int P = NZ * (NZ + 1) / 2;
  static constexpr int BS = 2 * NZ * (2 * NZ + 1);
  static constexpr int LD = NZ + 4;     // = 4 (mod 16)
  static constexpr int RT = NZ / 16;    // row tiles per component
  static constexpr int WARPS = 2 * RT;  // (row tile, K half)
  static constexpr int THREADS = WARPS * 32;
  static constexpr int KS = N3 / 8;     // k-steps of the staged X
  static constexpr int LDXR = CZ + 4;
  static constexpr size_t OFF_BAR = 0;  // [0]: the matrix copies, [1]: X's copies
  static constexpr size_t OFF_RAW = 128;
  static constexpr size_t RAW_BYTES = (size_t)NZ * NZ * 8;
  static constexpr size_t OFF_XRAW = OFF_RAW + RAW_BYTES;
  static constexpr size_t XRAW_BYTES = (size_t)4 * LDXR * 8;
  static constexpr size_t OFF_BLK = OFF_XRAW + XRAW_BYTES;
  static constexpr size_t BLK_BYTES = (size_t)NZ * LD * 8;
  static constexpr size_t OFF_XS = OFF_BLK + BLK_BYTES;
  static constexpr size_t XS_PLANE = (size_t)KS * 32 * 16;
  static constexpr size_t OFF_TRI = OFF_XS + 2 * XS_PLANE;
  static constexpr size_t SMEM = OFF_TRI + (((size_t)P * 2 + 15) / 16) * 16;
  // the K-half partial sums (8 floats per thread of the second-half warps) reuse the
  // unpacked matrix's space once the MMAs are done
  static_assert((size_t)RT * 32 * 8 * 4 <= BLK_BYTES, "partial sums fit the matrix space");
  static_assert(((size_t)P * 8) % 16 == 0 && OFF_XRAW % 16 == 0 && (LDXR * 8) % 16 == 0 && OFF_XS % 16 == 0,
                "bulk copy and vector alignment");
};

template <int NZ, int R>
__global__ void __launch_bounds__(MmaMatCfg<NZ, R>::THREADS)
    contract_mma_mat_kernel(float2 *__restrict__ spec, const float2 *__restrict__ qf, int Nx, int Ny, int ldz,
                            int *err, long long lim) {
  using Cfg = MmaMatCfg<NZ, R>;
  constexpr int N3 = Cfg::N3, CZ = Cfg::CZ, P = Cfg::P, BS = Cfg::BS, LD = Cfg::LD, RT = Cfg::RT;
  constexpr int THREADS = Cfg::THREADS, NN = NZ * NZ;
  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + Cfg::OFF_BAR);
  float2 *raw = reinterpret_cast<float2 *>(sm + Cfg::OFF_RAW);
  float2 *xraw = reinterpret_cast<float2 *>(sm + Cfg::OFF_XRAW);
  float2 *blk = reinterpret_cast<float2 *>(sm + Cfg::OFF_BLK);
  float *red = reinterpret_cast<float *>(sm + Cfg::OFF_BLK);
  uint4 *xs = reinterpret_cast<uint4 *>(sm + Cfg::OFF_XS);
  uint16_t *tri = reinterpret_cast<uint16_t *>(sm + Cfg::OFF_TRI);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nf = (Nx + 1) * (Ny + 1);

  // triangle entries (a, a + d) in diagonal order, so that the two stores of each spread
  // over the banks
  for (int d = tid; d < NZ; d += THREADS) {
    const int s0 = d * NZ - d * (d - 1) / 2;
    for (int a = 0; a + d < NZ; ++a) tri[s0 + a] = (uint16_t)(a << 8 | (a + d));
  }
  if (tid == 0) {
    tma::mbar_init(&bar[0], 1);
    tma::mbar_init(&bar[1], 1);
    tma::fence_mbar_init();
  }
  __syncthreads();

  // packed kind of M[alpha][beta]: xx, yy, zz, xy (triangles 0-3), xz, yz (full 4, 5);
  // M[1][0] = xy, M[2][0] = -xz^T, M[2][1] = -yz^T
  auto kind_of = [](int alpha, int beta) -> int {
    return alpha == beta ? alpha : (alpha + beta == 1 ? 3 : (alpha + beta == 2 ? 4 : 5));
  };
  auto issue_mat = [&](int w, int step) {
    const int kind = kind_of(step / 3, step % 3);
    const float2 *q = qf + (size_t)w * BS + (kind < 4 ? (size_t)kind * P : 4 * (size_t)P + (size_t)(kind - 4) * NN);
    const uint32_t bytes = (uint32_t)((kind < 4 ? P : NN) * 8);
    tma::fence_proxy_async();
    tma::mbar_expect_tx(&bar[0], bytes);
    tma::bulk_g2s(raw, q, bytes, &bar[0]);
  };
  auto issue_x = [&](int w) {
    const Mirrors mi = mirrors_of(w, Nx, Ny);
    const int nm = mi.nmx * mi.nmy;
    tma::fence_proxy_async();
    tma::mbar_expect_tx(&bar[1], (uint32_t)(nm * CZ * 8));
    for (int m = 0; m < nm; ++m) {
      const int mx = m % mi.nmx, my = m / mi.nmx;
      tma::bulk_g2s(xraw + (size_t)m * Cfg::LDXR, spec + mi.pos(mx, my, Nx) * ldz, (uint32_t)(CZ * 8), &bar[1]);
    }
  };

  // copies issued and waited for, per barrier (thread 0 issues; every thread waits)
  int nb_issued = 0, nx_issued = 0, nb_done = 0, nx_done = 0;
  const int w0 = blockIdx.x;
  if (tid == 0 && w0 < nf) {
    issue_x(w0);
    issue_mat(w0, 0);
    nx_issued = nb_issued = 1;
  }
  // on a wait that ran out: record it, let thread 0 wait for its copies still in
  // flight, and stop (the decision is collective, so no thread is left at a barrier)
  auto give_up = [&]() {
    if (tid == 0) {
      atomicExch(err, kContractTimeout);
      for (; nb_done < nb_issued; ++nb_done) tma::mbar_wait_bounded(&bar[0], (uint32_t)(nb_done & 1), kWaitLimit);
      for (; nx_done < nx_issued; ++nx_done) tma::mbar_wait_bounded(&bar[1], (uint32_t)(nx_done & 1), kWaitLimit);
    }
  };

  const int g = lane >> 2, t = lane & 3;
  const int rt = warp % RT, kh = warp / RT;
  const int a0 = rt * 16;
  for (int w = w0; w < nf; w += gridDim.x) {
    const Mirrors mw = mirrors_of(w, Nx, Ny);
    const int nmx = mw.nmx;
    const int ncol = mw.nmx * mw.nmy * R;
    // X of this wavenumber, split and in fragment order (as in contract_mma_unpack_kernel)
    if (!__syncthreads_and(tma::mbar_wait_bounded(&bar[1], (uint32_t)(nx_done & 1), lim))) {
      give_up();
      return;
    }
    ++nx_done;
    for (int e = tid; e < Cfg::KS * 32; e += THREADS) {
      const int ks = e >> 5, col = (e >> 2) & 7, tt = e & 3;
      const int k0 = ks * 8 + tt;
      float2 v0 = make_float2(0.f, 0.f), v1 = v0;
      if (col < ncol) {
        const int m = col / R, r = col - m * R;
        const int mx = m % nmx, my = m / nmx;
        const int comp = k0 / NZ;
        const float2 *xp = xraw + (size_t)m * Cfg::LDXR + r * N3 + k0;
        v0 = xp[0];
        v1 = xp[4];
        if ((comp == 0 && mx == 1) || (comp == 1 && my == 1)) {
          v0 = make_float2(-v0.x, -v0.y);
          v1 = make_float2(-v1.x, -v1.y);
        }
      }
      uint4 h, l;
      mma::split(v0.x, h.x, l.x);
      mma::split(v0.y, h.y, l.y);
      mma::split(v1.x, h.z, l.z);
      mma::split(v1.y, h.w, l.w);
      xs[e] = h;
      xs[Cfg::KS * 32 + e] = l;
    }
    float acc[2][2][2][4];
    for (int step = 0; step < 9; ++step) {
      const int alpha = step / 3, beta = step - 3 * alpha;
      const int kind = kind_of(alpha, beta);
      if (!__syncthreads_and(tma::mbar_wait_bounded(&bar[0], (uint32_t)(nb_done & 1), lim))) {
        give_up();
        return;
      }
      ++nb_done;
      // unpack: rows a, columns b at a LD + b
      if (kind < 4) {
        for (int e = tid; e < P; e += THREADS) {
          const int ab = tri[e], a = ab >> 8, b = ab & 255;
          const float2 v = raw[a * NZ - a * (a - 1) / 2 + (b - a)];
          blk[a * LD + b] = v;
          blk[b * LD + a] = v;
        }
      } else {
        for (int e = tid; e < NN; e += THREADS) {
          const int a = e / NZ, b = e - a * NZ;
          blk[a * LD + b] = raw[e];
        }
      }
      __syncthreads();  // blk (and in the first step xs) ready; raw (and xraw) consumed
      if (tid == 0) {
        if (step < 8) {
          issue_mat(w, step + 1);
          ++nb_issued;
        } else if (w + (int)gridDim.x < nf) {
          issue_mat(w + gridDim.x, 0);
          ++nb_issued;
        }
        if (step == 0 && w + (int)gridDim.x < nf) {
          issue_x(w + gridDim.x);
          ++nx_issued;
        }
      }
      if (beta == 0) {
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
              for (int c = 0; c < 4; ++c) acc[i][j][h][c] = 0.f;
      }
      {
        // M[2][0] = -xz^T, M[2][1] = -yz^T: read transposed, the minus on X
        const bool trb = alpha == 2 && beta < 2;
        const uint32_t neg = trb ? 0x80000000u : 0u;
        const int rs = trb ? 1 : LD, cs = trb ? LD : 1;
        const int b0 = kh * (NZ / 2);
        const float2 *p0 = blk + (a0 + g) * rs + (b0 + t) * cs;
        const uint4 *xfh = xs, *xfl = xs + Cfg::KS * 32;
#pragma unroll
        for (int bb = 0; bb < NZ / 2; bb += 8) {
          const float2 *p = p0 + bb * cs;
          float2 m[4];
          m[0] = p[0];
          m[1] = p[8 * rs];
          m[2] = p[4 * cs];
          m[3] = p[8 * rs + 4 * cs];
          const int ks = (beta * NZ + b0 + bb) / 8;
          const uint4 xh = xfh[ks * 32 + lane], xl = xfl[ks * 32 + lane];
          const uint32_t brh[2] = {xh.x ^ neg, xh.z ^ neg}, bih[2] = {xh.y ^ neg, xh.w ^ neg};
          const uint32_t brl[2] = {xl.x ^ neg, xl.z ^ neg}, bil[2] = {xl.y ^ neg, xl.w ^ neg};
          uint32_t arh[4], arl[4], aih[4], ail[4];
          mma::split_a(m, arh, arl, aih, ail);
          mma::mma12(acc, arh, arl, aih, ail, brh, brl, bih, bil);
        }
      }
      __syncthreads();  // every warp is done with blk
      if (beta < 2) continue;
      // component alpha of Y: the two K halves meet in blk's space
      float part[4][2];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float rr = acc[0][0][0][c] + acc[0][0][1][c], ii = acc[1][1][0][c] + acc[1][1][1][c];
        const float ri = acc[0][1][0][c] + acc[0][1][1][c], ir = acc[1][0][0][c] + acc[1][0][1][c];
        part[c][0] = rr - ii;
        part[c][1] = ri + ir;
      }
      if (kh == 1) {
        float4 *rp = reinterpret_cast<float4 *>(red + (rt * 32 + lane) * 8);
        rp[0] = make_float4(part[0][0], part[0][1], part[1][0], part[1][1]);
        rp[1] = make_float4(part[2][0], part[2][1], part[3][0], part[3][1]);
      }
      __syncthreads();
      if (kh == 0) {
        const float4 *rp = reinterpret_cast<const float4 *>(red + (rt * 32 + lane) * 8);
        const float4 u0 = rp[0], u1 = rp[1];
        part[0][0] += u0.x;
        part[0][1] += u0.y;
        part[1][0] += u0.z;
        part[1][1] += u0.w;
        part[2][0] += u1.x;
        part[2][1] += u1.y;
        part[3][0] += u1.z;
        part[3][1] += u1.w;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int col = 2 * t + (c & 1);
          if (col < ncol) {
            const int row = alpha * NZ + a0 + g + 8 * (c >> 1);
            const int m = col / R, r = col - m * R;
            const int mx = m % nmx, my = m / nmx;
            float2 v = make_float2(part[c][0], part[c][1]);
            if ((alpha == 0 && mx == 1) || (alpha == 1 && my == 1)) { v.x = -v.x; v.y = -v.y; }
            spec[mw.pos(mx, my, Nx) * ldz + r * N3 + row] = v;
          }
        }
      }
      __syncthreads();  // the partial sums are read before the next unpacking
    }
  }
}

}  // namespace ie
