// Per-wavenumber block contraction (step 2 of the FFT matrix-vector product,
// Sect. 3.3): for every horizontal wavenumber k the spectrum vector v(k), of
// 3 Nz components per right-hand side, is replaced by Qt(k) v(k), where Qt(k) is
// the 3x3 block of Nz x Nz matrices of the DFT'd coefficients.
//
// Coefficients are stored once per folded wavenumber (kx_bar in [0, Nx], ky_bar in
// [0, Ny]) in the symmetry-compressed layout of eq. (matrix_symm): packed upper
// triangles of the symmetric xx, yy, zz, xy blocks and the full xz, yz blocks,
// 2 Nz (2 Nz + 1) complex numbers.  The other blocks follow from Lemma 1
// (zx = -xz^T, zy = -yz^T, yx = xy).  A mirror wavenumber 2N - k reflects the
// corresponding lateral axis, which flips the sign of that field component:
// Qt(-kx, ky) = T Qt(kx, ky) T with T = diag(-1, 1, 1) on the components
// (Lemma 2), so one CTA loads a block once and applies it to all its mirrors and
// all right-hand sides.
#include "contract.cuh"
#include "contract_mma.cuh"
#include "contract_tc.cuh"
#include "contract_tma.cuh"

namespace ie {
namespace {

// Element (row, col) of the 3 Nz x 3 Nz block from its packed storage, row = alpha Nz + a,
// col = beta Nz + b: symmetric xx, yy, zz, xy from their upper triangles, xz and yz in
// full, zx = -xz^T and zy = -yz^T (Lemma 1).
template <typename T>
__device__ __forceinline__ C<T> block_entry(const C<T> *__restrict__ q, int Nz, int P, int row, int col) {
  const int alpha = row / Nz, a = row - alpha * Nz;
  const int beta = col / Nz, b = col - beta * Nz;
  const bool full = (alpha == 2) != (beta == 2);  // xz / yz / zx / zy
  if (!full) {
    const int kind = alpha == beta ? alpha : 3;  // xx, yy, zz on the diagonal; xy off it
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return q[(size_t)kind * P + lo * Nz - lo * (lo - 1) / 2 + (hi - lo)];
  }
  if (beta == 2) return q[4 * (size_t)P + (size_t)alpha * Nz * Nz + a * Nz + b];
  return cneg(q[4 * (size_t)P + (size_t)beta * Nz * Nz + b * Nz + a]);
}

// One CTA per folded wavenumber.  The mirror vectors (with their component signs) sit
// in shared memory as X[MAXC][3 Nz]; the block streams through a panel of PW columns
// [3 Nz][PW + 1] (PW = 3 Nz when the whole block fits three CTAs per SM; the odd row stride keeps the
// per-thread row reads free of bank conflicts); thread t accumulates output row t over
// all panels in registers.
template <typename T, int MAXC>
__global__ void contract_kernel(C<T> *__restrict__ spec, const C<T> *__restrict__ qf, int Nx, int Ny, int Nz,
                                int R, int PW, int ldz) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n3 = 3 * Nz;
  C<T> *X = reinterpret_cast<C<T> *>(smem_raw);  // [MAXC][3 Nz]
  C<T> *pan = X + (size_t)MAXC * n3;              // [3 Nz][PW + 1]
  const int ldp = PW + 1;
  const int kxb = blockIdx.x, kyb = blockIdx.y;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int CZ = ldz;
  const int P = Nz * (Nz + 1) / 2;
  const long long BS = 2LL * Nz * (2 * Nz + 1);
  const C<T> *q = qf + ((long long)kyb * (Nx + 1) + kxb) * BS;

  // mirror wavenumbers and their component signs (scalars: see the pipelined kernel)
  const int nmx = (kxb > 0 && kxb < Nx) ? 2 : 1, nmy = (kyb > 0 && kyb < Ny) ? 2 : 1;
  const int kx1 = 2 * Nx - kxb, ky1 = 2 * Ny - kyb;
  const int ncol = nmx * nmy * R;
  for (int e = tid; e < ncol * n3; e += nthr) {
    const int col = e / n3, row = e - col * n3;
    const int m = col / R, r = col - m * R;
    const int mx = m % nmx, my = m / nmx;
    const int comp = row / Nz;
    const long long g = ((long long)(my ? ky1 : kyb) * 2 * Nx + (mx ? kx1 : kxb)) * CZ + r * n3 + row;
    C<T> v = spec[g];
    if ((comp == 0 && mx == 1) || (comp == 1 && my == 1)) v = cneg(v);
    X[col * n3 + row] = v;
  }
  const int row = tid;
  C<T> acc[MAXC];
#pragma unroll
  for (int c = 0; c < MAXC; ++c) acc[c] = mk<T>(0, 0);
  for (int c0 = 0; c0 < n3; c0 += PW) {
    const int w = n3 - c0 < PW ? n3 - c0 : PW;
    __syncthreads();  // previous panel consumed (first pass: X staged)
    for (int e = tid; e < n3 * w; e += nthr) {
      const int rr = e / w, j = e - rr * w;
      pan[rr * ldp + j] = block_entry<T>(q, Nz, P, rr, c0 + j);
    }
    __syncthreads();
    if (row < n3) {
      const C<T> *mrow = pan + (size_t)row * ldp;
      for (int j = 0; j < w; ++j) {
        const C<T> m = mrow[j];
        const C<T> *xb = X + c0 + j;
#pragma unroll
        for (int c = 0; c < MAXC; ++c)
          if (c < ncol) cfma(acc[c], m, xb[c * n3]);
      }
    }
  }
  if (row < n3) {
    const int alpha = row / Nz;
#pragma unroll
    for (int c = 0; c < MAXC; ++c) {
      if (c < ncol) {
        const int mm = c / R, r = c - mm * R;
        const int mx = mm % nmx, my = mm / nmx;
        C<T> v = acc[c];
        if ((alpha == 0 && mx == 1) || (alpha == 1 && my == 1)) v = cneg(v);
        spec[((long long)(my ? ky1 : kyb) * 2 * Nx + (mx ? kx1 : kxb)) * CZ + r * n3 + row] = v;
      }
    }
  }
}

constexpr size_t kMaxSmem = 227 * 1024;

template <typename T, int MAXC>
int launch_t(C<T> *spec, const C<T> *qf, int Nx, int Ny, int Nz, int R, int ldz, cudaStream_t s) {
  const int n3 = 3 * Nz;
  if (n3 > 1024) return -1;
  const size_t e = sizeof(C<T>);
  const size_t xb = e * (size_t)MAXC * n3;
  // widest panel that leaves room for three CTAs per SM (one stages while the others
  // compute); else the narrowest that fits at all
  int PW = 16;
  for (int cand : {n3, 64, 32, 16}) {
    if (cand > n3) continue;
    if (xb + e * (size_t)n3 * (cand + 1) <= kMaxSmem / 3) { PW = cand; break; }
  }
  const size_t sm = xb + e * (size_t)n3 * (PW + 1);
  if (sm > kMaxSmem) return -1;
  auto k = contract_kernel<T, MAXC>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) return -1;
  const int threads = ((n3 + 31) / 32) * 32;
  dim3 grid(Nx + 1, Ny + 1);
  count_launches(1);
  k<<<grid, threads, sm, s>>>(spec, qf, Nx, Ny, Nz, R, PW, ldz);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

// Error word of the launches that are given none (ie_matvec_noalloc, the autotuner).
__device__ int g_contract_err = 0;
long long g_wait_limit = kWaitLimit;

int *default_err() {
  int *err = nullptr;
  if (cudaGetSymbolAddress((void **)&err, g_contract_err) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return err;
}

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

template <int NZ, int R, int NS, int RPT>
bool try_tma(float2 *spec, const float2 *qf, int Nx, int Ny, int ldz, int per_sm, int *err, cudaStream_t s) {
  using Cfg = ContractCfg<NZ, R, NS, RPT>;
  if (Cfg::SMEM > 227 * 1024) return false;
  auto k = contract_tma_kernel<NZ, R, NS, RPT>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int nf = (Nx + 1) * (Ny + 1);
  const int want = per_sm * num_sms();
  const int grid = nf < want ? nf : want;
  count_launches(1);
  k<<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(spec, qf, Nx, Ny, ldz, err, g_wait_limit);
  if (cudaPeekAtLastError() != cudaSuccess) {  // not launched: the caller falls back to the panel kernel
    cudaGetLastError();
    return false;
  }
  return true;
}

// Ring variants: one slot per CTA and two CTAs per SM where they fit (the copy of the next
// wavenumber overlaps the arithmetic of the current one, and the other CTA on the SM
// covers the unpacking phase), or three slots and one CTA per SM.
template <int NZ, int R>
bool try_tma_variant(float2 *spec, const float2 *qf, int Nx, int Ny, int ldz, int variant, int *err,
                     cudaStream_t s) {
  constexpr int RPT2 = R == 2 ? 2 : 1;
  if (variant == kContractTma1) {
    if (2 * ContractCfg<NZ, R, 1, RPT2>::SMEM <= 227 * 1024)
      return try_tma<NZ, R, 1, RPT2>(spec, qf, Nx, Ny, ldz, 2, err, s);
    return try_tma<NZ, R, 1, RPT2>(spec, qf, Nx, Ny, ldz, 1, err, s);
  }
  if (variant == kContractTma1Row) {
    if (2 * ContractCfg<NZ, R, 1, 1>::SMEM <= 227 * 1024)
      return try_tma<NZ, R, 1, 1>(spec, qf, Nx, Ny, ldz, 2, err, s);
    return try_tma<NZ, R, 1, 1>(spec, qf, Nx, Ny, ldz, 1, err, s);
  }
  if (variant == kContractTma3) return try_tma<NZ, R, 3, RPT2>(spec, qf, Nx, Ny, ldz, 1, err, s);
  return false;
}

// The tensor-core kernels (persistent: as many resident CTAs per SM as registers and
// shared memory allow).
template <typename K>
bool launch_persistent(K k, int threads, size_t smem, int *per_sm, float2 *spec, const float2 *qf, int Nx, int Ny,
                       int ldz, int *err, cudaStream_t s) {
  if (smem > 227 * 1024) return false;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (*per_sm == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, threads, smem) != cudaSuccess || *per_sm < 1) {
      cudaGetLastError();
      *per_sm = 1;
    }
  }
  const int nf = (Nx + 1) * (Ny + 1);
  const int want = *per_sm * num_sms();
  const int grid = nf < want ? nf : want;
  count_launches(1);
  k<<<grid, threads, smem, s>>>(spec, qf, Nx, Ny, ldz, err, g_wait_limit);
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

template <int NZ, int R>
bool try_mma(float2 *spec, const float2 *qf, int Nx, int Ny, int ldz, bool unpack, int *err, cudaStream_t s) {
  if (unpack) {
    static int per_sm = 0;
    using Cfg = MmaUnpackCfg<NZ, R>;
    return launch_persistent(contract_mma_unpack_kernel<NZ, R>, Cfg::THREADS, Cfg::SMEM, &per_sm, spec, qf, Nx, Ny,
                             ldz, err, s);
  }
  static int per_sm = 0;
  using Cfg = MmaCfg<NZ, R, 2>;
  return launch_persistent(contract_mma_kernel<NZ, R, 2>, Cfg::THREADS, Cfg::SMEM, &per_sm, spec, qf, Nx, Ny, ldz,
                           err, s);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda)
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// The full xz, yz blocks of every folded wavenumber as a 3-D tensor of 8-byte
// elements: [nf blocks][2 Nz rows][Nz columns] starting 4P complex into each packed
// block (strides Nz * 8 and 2 Nz (2 Nz + 1) * 8 bytes); boxes of 16 columns x 2 Nz rows
// x 1 block, 128-byte swizzle.
bool encode_full_map(CUtensorMap *map, const float2 *qf, int Nz, long long nf) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const long long P = (long long)Nz * (Nz + 1) / 2, BS = 2LL * Nz * (2 * Nz + 1);
  const cuuint64_t dims[3] = {(cuuint64_t)Nz, (cuuint64_t)(2 * Nz), (cuuint64_t)nf};
  const cuuint64_t strides[2] = {(cuuint64_t)Nz * 8, (cuuint64_t)BS * 8};
  const cuuint32_t box[3] = {16, (cuuint32_t)(2 * Nz), 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<float2 *>(qf + 4 * P), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The tcgen05 kernel: persistent, as many CTAs per SM as occupancy and tensor memory
// allow (each holds TcCfg::TCOLS of the SM's 512 columns for its lifetime).
template <int NZ, int R, bool F16>
bool try_tc(float2 *spec, const float2 *qf, const int *qexp, int Nx, int Ny, int ldz, int *err, cudaStream_t s) {
  using Cfg = TcCfg<NZ, R, F16>;
  static int per_sm = 0;
  auto k = contract_tc_kernel<NZ, R, F16, false>;
  if (F16 && !qexp) return false;
  constexpr size_t smem = Cfg::SMEM + 1024;  // the kernel aligns its base to 1024 bytes
  if (smem > 227 * 1024) return false;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (per_sm == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, Cfg::THREADS, smem) != cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
    if (per_sm > 512 / Cfg::TCOLS) per_sm = 512 / Cfg::TCOLS;
  }
  const int nf = (Nx + 1) * (Ny + 1);
  CUtensorMap tmap;
  if (!encode_full_map(&tmap, qf, NZ, nf)) return false;
  const int want = per_sm * num_sms();
  const int grid = nf < want ? nf : want;
  count_launches(1);
  k<<<grid, Cfg::THREADS, smem, s>>>(spec, qf, Nx, Ny, ldz, err, g_wait_limit, tmap, qexp, nullptr);
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

template <int R, bool F16>
bool dispatch_tc(float2 *spec, const float2 *qf, const int *qexp, int Nx, int Ny, int Nz, int ldz, int *err,
                 cudaStream_t s) {
  switch (Nz) {
    case 16: return try_tc<16, R, F16>(spec, qf, qexp, Nx, Ny, ldz, err, s);
    case 32: return try_tc<32, R, F16>(spec, qf, qexp, Nx, Ny, ldz, err, s);
    default: return false;
  }
}

// exponent e_w of every folded wavenumber's packed block: max |re|, |im| times 2^e_w in
// [2^13, 2^14) (0 for a zero block), clamped to [-100, 100]
__global__ void block_exponent_kernel(const float2 *__restrict__ qf, int *__restrict__ qexp, int BS) {
  __shared__ float sh[8];
  const float2 *q = qf + (size_t)blockIdx.x * BS;
  float m = 0.f;
  for (int i = threadIdx.x; i < BS; i += blockDim.x) {
    const float2 v = q[i];
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, sh[w]);
    qexp[blockIdx.x] = tc::scale_exp(m);
  }
}

template <int NZ, int R>
bool try_mma_comp(float2 *spec, const float2 *qf, int Nx, int Ny, int ldz, int *err, cudaStream_t s) {
  static int per_sm = 0;
  using Cfg = MmaMatCfg<NZ, R>;
  return launch_persistent(contract_mma_mat_kernel<NZ, R>, Cfg::THREADS, Cfg::SMEM, &per_sm, spec, qf, Nx, Ny, ldz,
                           err, s);
}

template <int R>
bool dispatch_mma_comp(float2 *spec, const float2 *qf, int Nx, int Ny, int Nz, int ldz, int *err, cudaStream_t s) {
  switch (Nz) {
    case 16: return try_mma_comp<16, R>(spec, qf, Nx, Ny, ldz, err, s);
    case 32: return try_mma_comp<32, R>(spec, qf, Nx, Ny, ldz, err, s);
    case 48: return try_mma_comp<48, R>(spec, qf, Nx, Ny, ldz, err, s);
    case 64: return try_mma_comp<64, R>(spec, qf, Nx, Ny, ldz, err, s);
    default: return false;
  }
}

// the FP16 pairs of variant 7's A operand: hi = fp16(x 2^e), lo = fp16(x 2^e - hi), for
// the real and the imaginary part, hi in the low half
__global__ void split_f16_kernel(const float2 *__restrict__ qf, const int *__restrict__ qexp, uint2 *__restrict__ qh,
                                 long long n, int BS) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float sc = tc::pow2f(qexp[i / BS]);
    const float2 v = qf[i];
    const float xr = v.x * sc, xi = v.y * sc;
    const __half hr = __float2half_rn(xr), hi = __float2half_rn(xi);
    const __half lr = __float2half_rn(__fsub_rn(xr, __half2float(hr)));
    const __half li = __float2half_rn(__fsub_rn(xi, __half2float(hi)));
    qh[i] = make_uint2((uint32_t)__half_as_ushort(hr) | (uint32_t)__half_as_ushort(lr) << 16,
                       (uint32_t)__half_as_ushort(hi) | (uint32_t)__half_as_ushort(li) << 16);
  }
}

template <int R>
bool dispatch_mma(float2 *spec, const float2 *qf, int Nx, int Ny, int Nz, int ldz, bool unpack, int *err,
                  cudaStream_t s) {
  switch (Nz) {
    case 16: return try_mma<16, R>(spec, qf, Nx, Ny, ldz, unpack, err, s);
    case 32: return try_mma<32, R>(spec, qf, Nx, Ny, ldz, unpack, err, s);
    case 48: return try_mma<48, R>(spec, qf, Nx, Ny, ldz, unpack, err, s);
    default: return false;
  }
}

template <int R>
bool dispatch_tma(float2 *spec, const float2 *qf, int Nx, int Ny, int Nz, int ldz, int variant, int *err,
                  cudaStream_t s) {
  switch (Nz) {
    case 16: return try_tma_variant<16, R>(spec, qf, Nx, Ny, ldz, variant, err, s);
    case 24: return try_tma_variant<24, R>(spec, qf, Nx, Ny, ldz, variant, err, s);
    case 32: return try_tma_variant<32, R>(spec, qf, Nx, Ny, ldz, variant, err, s);
    case 48: return try_tma_variant<48, R>(spec, qf, Nx, Ny, ldz, variant, err, s);
    default: return false;
  }
}

template <int NZ, int R>
bool tma3_fits() { return ContractCfg<NZ, R, 3, (R == 2 ? 2 : 1)>::SMEM <= 227 * 1024; }

}  // namespace

bool contract_tma_enabled = true;

int contract_take_error(int *err, cudaStream_t s) {
  if (!err) err = default_err();
  if (!err) return -1;
  int h = 0;
  if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return -1;
  if (h && (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess))
    return -1;
  return h;
}

void set_wait_limit(long long polls) { g_wait_limit = polls >= 0 ? polls : kWaitLimit; }

bool contract_fits(int Nz, int R, bool c64) {
  if (Nz < 1 || R < 1 || R > 4 || 3 * Nz > 1024) return false;
  const size_t e = c64 ? sizeof(float2) : sizeof(double2);
  const size_t maxc = R <= 1 ? 4 : (R <= 2 ? 8 : 16);
  // launch_t with its narrowest panel (16 columns)
  return e * (size_t)3 * Nz * (maxc + 17) <= kMaxSmem;
}

bool contract_variant_available(int variant, int Nz, int R, bool c64) {
  if (variant == kContractPanel) return R >= 1 && R <= 4 && 3 * Nz <= 1024;
  if (!c64 || R < 1 || R > 2 || !contract_tma_enabled) return false;
  if (variant == kContractMmaComp) return Nz == 16 || Nz == 32 || Nz == 48 || Nz == 64;
  if (Nz != 16 && Nz != 24 && Nz != 32 && Nz != 48) return false;
  if (variant == kContractTc || variant == kContractTc16) return Nz == 16 || Nz == 32;
  if (variant == kContractMma || variant == kContractMmaUnpack) return Nz % 16 == 0;
  if (variant == kContractTma1) return true;
  if (variant == kContractTma1Row) return R == 2;
  if (variant == kContractTma3) {
    switch (Nz) {
      case 16: return R == 1 ? tma3_fits<16, 1>() : tma3_fits<16, 2>();
      case 24: return R == 1 ? tma3_fits<24, 1>() : tma3_fits<24, 2>();
      case 32: return R == 1 ? tma3_fits<32, 1>() : tma3_fits<32, 2>();
      default: return R == 1 ? tma3_fits<48, 1>() : tma3_fits<48, 2>();
    }
  }
  return false;
}

template <typename T>
int launch_contract(C<T> *spec, const C<T> *qf, int Nx, int Ny, int Nz, int R, int ldz, int variant, int *err,
                    cudaStream_t s, const int *qexp, const void *qh) {
  if (ldz < R * 3 * Nz) return -1;
  if constexpr (sizeof(T) == 4) {
    if (!err) err = default_err();
    if (!err) return -1;
    if (variant == kContractAuto) variant = contract_variant_available(kContractTma1, Nz, R, true) ? kContractTma1
                                                                                                    : kContractPanel;
    if ((variant == kContractMma || variant == kContractMmaUnpack) &&
        contract_variant_available(variant, Nz, R, true)) {
      const bool unpack = variant == kContractMmaUnpack;
      if (R == 1 && dispatch_mma<1>(spec, qf, Nx, Ny, Nz, ldz, unpack, err, s)) return 0;
      if (R == 2 && dispatch_mma<2>(spec, qf, Nx, Ny, Nz, ldz, unpack, err, s)) return 0;
    }
    if (variant == kContractMmaComp && contract_variant_available(variant, Nz, R, true)) {
      if (R == 1 && dispatch_mma_comp<1>(spec, qf, Nx, Ny, Nz, ldz, err, s)) return 0;
      if (R == 2 && dispatch_mma_comp<2>(spec, qf, Nx, Ny, Nz, ldz, err, s)) return 0;
    }
    if (variant == kContractTc && contract_variant_available(variant, Nz, R, true)) {
      if (R == 1 && dispatch_tc<1, false>(spec, qf, nullptr, Nx, Ny, Nz, ldz, err, s)) return 0;
      if (R == 2 && dispatch_tc<2, false>(spec, qf, nullptr, Nx, Ny, Nz, ldz, err, s)) return 0;
    }
    if (variant == kContractTc16 && qexp && qh && contract_variant_available(variant, Nz, R, true)) {
      const float2 *q16 = reinterpret_cast<const float2 *>(qh);  // 8 bytes per complex, as qf
      if (R == 1 && dispatch_tc<1, true>(spec, q16, qexp, Nx, Ny, Nz, ldz, err, s)) return 0;
      if (R == 2 && dispatch_tc<2, true>(spec, q16, qexp, Nx, Ny, Nz, ldz, err, s)) return 0;
    }
    if ((variant == kContractTma1 || variant == kContractTma3 || variant == kContractTma1Row) &&
        contract_variant_available(variant, Nz, R, true)) {
      if (R == 1 && dispatch_tma<1>(spec, qf, Nx, Ny, Nz, ldz, variant, err, s)) return 0;
      if (R == 2 && dispatch_tma<2>(spec, qf, Nx, Ny, Nz, ldz, variant, err, s)) return 0;
    }
  }
  if (R <= 1) return launch_t<T, 4>(spec, qf, Nx, Ny, Nz, R, ldz, s);
  if (R <= 2) return launch_t<T, 8>(spec, qf, Nx, Ny, Nz, R, ldz, s);
  if (R <= 4) return launch_t<T, 16>(spec, qf, Nx, Ny, Nz, R, ldz, s);
  return -1;
}

template int launch_contract<float>(float2 *, const float2 *, int, int, int, int, int, int, int *, cudaStream_t,
                                    const int *, const void *);
template int launch_contract<double>(double2 *, const double2 *, int, int, int, int, int, int, int *, cudaStream_t,
                                     const int *, const void *);

void launch_split_f16(const float2 *qf, const int *qexp, void *qh, long long nf, int Nz, cudaStream_t s) {
  const long long n = nf * 2LL * Nz * (2 * Nz + 1);
  const long long blocks = (n + 255) / 256;
  count_launches(1);
  split_f16_kernel<<<(unsigned)(blocks < 65535LL * 64 ? blocks : 65535LL * 64), 256, 0, s>>>(
      qf, qexp, reinterpret_cast<uint2 *>(qh), n, 2 * Nz * (2 * Nz + 1));
}

void launch_block_exponents(const float2 *qf, int *qexp, long long nf, int Nz, cudaStream_t s) {
  count_launches(1);
  block_exponent_kernel<<<(unsigned)nf, 256, 0, s>>>(qf, qexp, 2 * Nz * (2 * Nz + 1));
}

}  // namespace ie
