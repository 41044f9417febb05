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
#include "contract_tma.cuh"

namespace ie {
namespace {

template <typename T>
__device__ __forceinline__ void unpack_block(const C<T> *__restrict__ q, C<T> *sm, int Nz, int ld, int tid,
                                             int nthr) {
  // sm holds 6 matrices [Nz][ld]: xx, yy, zz, xy (both triangles), xz, yz
  const int P = Nz * (Nz + 1) / 2;
  for (int e = tid; e < 4 * P; e += nthr) {
    const int blk = e / P;
    int p = e - blk * P;
    // row a of the packed upper triangle starts at a*Nz - a(a-1)/2 and has Nz - a entries
    int a = 0;
    int rowlen = Nz;
    while (p >= rowlen) { p -= rowlen; ++a; --rowlen; }
    const int b = a + p;
    const C<T> v = q[e];
    C<T> *m = sm + (size_t)blk * Nz * ld;
    m[a * ld + b] = v;
    m[b * ld + a] = v;
  }
  const C<T> *qf = q + 4 * P;
  for (int e = tid; e < 2 * Nz * Nz; e += nthr) {
    const int blk = e / (Nz * Nz);
    const int r = e - blk * Nz * Nz;
    const int a = r / Nz, b = r - a * Nz;
    sm[(size_t)(4 + blk) * Nz * ld + a * ld + b] = qf[e];
  }
}

template <typename T, int MAXC>
__global__ void contract_kernel(C<T> *__restrict__ spec, const C<T> *__restrict__ qf, int Nx, int Ny, int Nz,
                                int R) {
  extern __shared__ unsigned char smem_raw[];
  const int ld = Nz + 1;
  C<T> *blk = reinterpret_cast<C<T> *>(smem_raw);
  C<T> *X = blk + (size_t)6 * Nz * ld;  // [MAXC][3 Nz]
  const int kxb = blockIdx.x, kyb = blockIdx.y;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int n3 = 3 * Nz;
  const int CZ = R * n3;
  const long long BS = 2LL * Nz * (2 * Nz + 1);
  const C<T> *q = qf + ((long long)kyb * (Nx + 1) + kxb) * BS;
  unpack_block<T>(q, blk, Nz, ld, tid, nthr);

  // mirror wavenumbers and their component signs
  int kxs[2], kys[2];
  int nmx = 1, nmy = 1;
  kxs[0] = kxb;
  kys[0] = kyb;
  if (kxb > 0 && kxb < Nx) { kxs[1] = 2 * Nx - kxb; nmx = 2; }
  if (kyb > 0 && kyb < Ny) { kys[1] = 2 * Ny - kyb; nmy = 2; }
  const int ncol = nmx * nmy * R;
  for (int e = tid; e < ncol * n3; e += nthr) {
    const int col = e / n3, row = e - col * n3;
    const int m = col / R, r = col - m * R;
    const int mx = m % nmx, my = m / nmx;
    const int comp = row / Nz;
    const long long g = ((long long)kys[my] * 2 * Nx + kxs[mx]) * CZ + r * n3 + row;
    C<T> v = spec[g];
    if ((comp == 0 && mx == 1) || (comp == 1 && my == 1)) v = cneg(v);
    X[col * n3 + row] = v;
  }
  __syncthreads();
  const C<T> *Axx = blk, *Ayy = blk + Nz * ld, *Azz = blk + 2 * Nz * ld, *Axy = blk + 3 * Nz * ld;
  const C<T> *Axz = blk + 4 * Nz * ld, *Ayz = blk + 5 * Nz * ld;
  for (int row = tid; row < n3; row += nthr) {
    const int alpha = row / Nz, a = row - alpha * Nz;
    C<T> acc[MAXC];
#pragma unroll
    for (int c = 0; c < MAXC; ++c) acc[c] = mk<T>(0, 0);
    for (int beta = 0; beta < 3; ++beta) {
      for (int b = 0; b < Nz; ++b) {
        C<T> m;
        if (alpha == 0) {
          m = beta == 0 ? Axx[b * ld + a] : (beta == 1 ? Axy[b * ld + a] : Axz[a * ld + b]);
        } else if (alpha == 1) {
          m = beta == 0 ? Axy[b * ld + a] : (beta == 1 ? Ayy[b * ld + a] : Ayz[a * ld + b]);
        } else {
          m = beta == 0 ? cneg(Axz[b * ld + a]) : (beta == 1 ? cneg(Ayz[b * ld + a]) : Azz[b * ld + a]);
        }
        const C<T> *xb = X + beta * Nz + b;
#pragma unroll
        for (int c = 0; c < MAXC; ++c)
          if (c < ncol) cfma(acc[c], m, xb[c * n3]);
      }
    }
#pragma unroll
    for (int c = 0; c < MAXC; ++c) {
      if (c < ncol) {
        const int mm = c / R, r = c - mm * R;
        const int mx = mm % nmx, my = mm / nmx;
        C<T> v = acc[c];
        if ((alpha == 0 && mx == 1) || (alpha == 1 && my == 1)) v = cneg(v);
        spec[((long long)kys[my] * 2 * Nx + kxs[mx]) * CZ + r * n3 + row] = v;
      }
    }
  }
}

template <typename T, int MAXC>
void launch_t(C<T> *spec, const C<T> *qf, int Nx, int Ny, int Nz, int R, cudaStream_t s) {
  const size_t sm = sizeof(C<T>) * ((size_t)6 * Nz * (Nz + 1) + (size_t)MAXC * 3 * Nz);
  auto k = contract_kernel<T, MAXC>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int threads = ((3 * Nz + 31) / 32) * 32;
  if (threads > 512) threads = 512;
  dim3 grid(Nx + 1, Ny + 1);
  count_launches(1);
  k<<<grid, threads, sm, s>>>(spec, qf, Nx, Ny, Nz, R);
}

__device__ int g_contract_err = 0;

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

template <int NZ, int R, int NS>
bool try_tma(float2 *spec, const float2 *qf, int Nx, int Ny, cudaStream_t s) {
  using Cfg = ContractCfg<NZ, R, NS>;
  if (Cfg::SMEM > 227 * 1024) return false;
  auto k = contract_tma_kernel<NZ, R, NS>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int *err = nullptr;
  cudaGetSymbolAddress((void **)&err, g_contract_err);
  const int nf = (Nx + 1) * (Ny + 1);
  const int grid = nf < num_sms() ? nf : num_sms();
  count_launches(1);
  k<<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(spec, qf, Nx, Ny, err);
  return true;
}

template <int NZ, int R>
bool try_tma_stages(float2 *spec, const float2 *qf, int Nx, int Ny, cudaStream_t s) {
  if (ContractCfg<NZ, R, 3>::SMEM <= 227 * 1024) return try_tma<NZ, R, 3>(spec, qf, Nx, Ny, s);
  if (ContractCfg<NZ, R, 2>::SMEM <= 227 * 1024) return try_tma<NZ, R, 2>(spec, qf, Nx, Ny, s);
  return try_tma<NZ, R, 1>(spec, qf, Nx, Ny, s);
}

template <int R>
bool dispatch_tma(float2 *spec, const float2 *qf, int Nx, int Ny, int Nz, cudaStream_t s) {
  switch (Nz) {
    case 16: return try_tma_stages<16, R>(spec, qf, Nx, Ny, s);
    case 24: return try_tma_stages<24, R>(spec, qf, Nx, Ny, s);
    case 32: return try_tma_stages<32, R>(spec, qf, Nx, Ny, s);
    case 48: return try_tma_stages<48, R>(spec, qf, Nx, Ny, s);
    default: return false;
  }
}

}  // namespace

bool contract_tma_enabled = true;

int contract_take_error() {
  int h = 0, z = 0;
  cudaMemcpyFromSymbol(&h, g_contract_err, sizeof(int));
  if (h) cudaMemcpyToSymbol(g_contract_err, &z, sizeof(int));
  return h;
}

size_t contract_smem_bytes(int Nz, int R, size_t elem) {
  return elem * ((size_t)6 * Nz * (Nz + 1) + (size_t)4 * R * 3 * Nz);
}

template <typename T>
int launch_contract(C<T> *spec, const C<T> *qf, int Nx, int Ny, int Nz, int R, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (contract_tma_enabled) {
      if (R == 1 && dispatch_tma<1>(spec, qf, Nx, Ny, Nz, s)) return 0;
      if (R == 2 && dispatch_tma<2>(spec, qf, Nx, Ny, Nz, s)) return 0;
    }
  }
  if (R <= 1) launch_t<T, 4>(spec, qf, Nx, Ny, Nz, R, s);
  else if (R <= 2) launch_t<T, 8>(spec, qf, Nx, Ny, Nz, R, s);
  else if (R <= 4) launch_t<T, 16>(spec, qf, Nx, Ny, Nz, R, s);
  else return -1;
  return 0;
}

template int launch_contract<float>(float2 *, const float2 *, int, int, int, int, cudaStream_t);
template int launch_contract<double>(double2 *, const double2 *, int, int, int, int, cudaStream_t);

}  // namespace ie
