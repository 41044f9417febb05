// Setup kernels: the DFT of the compressed coefficient tensor (stored as Qt,
// Sect. 3.3: "instead of matrices Q(i, j) the discrete Fourier transformations
// are stored") and small element-wise helpers.
//
// The real-space tensor Q(i, j), i in [0, Ny), j in [0, Nx), is embedded in a
// 2Ny x 2Nx periodic array using the lateral parities of Lemma 2 (negative
// offsets from the stored ones, zero at i = Ny or j = Nx), transformed, and the
// folded wavenumbers kx in [0, Nx], ky in [0, Ny] are packed in the layout of the
// contraction kernel.  The DFT keeps each block's parity, so the folded half
// determines the rest.
#include "setup.cuh"

namespace ie {
namespace {

// parity signs (x, y) of blocks xx, yy, zz, xy, xz, yz
__device__ __forceinline__ void block_parity(int b, int &px, int &py) {
  px = (b == 3 || b == 4) ? -1 : 1;
  py = (b == 3 || b == 5) ? -1 : 1;
}

// emb[iy][jx][e - e0] for e in [e0, e0 + E), e = (b * Nz + a) * Nz + c
__global__ void embed_kernel(const double2 *__restrict__ qreal, double2 *__restrict__ emb, int Nx, int Ny, int Nz,
                             long long e0, long long E) {
  const long long tot = 4LL * Nx * Ny * E;
  const long long NE = 6LL * Nz * Nz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const long long el = t % E;
    const long long pos = t / E;
    const int jx = (int)(pos % (2 * Nx));
    const int iy = (int)(pos / (2 * Nx));
    const long long e = e0 + el;
    double2 v = make_double2(0.0, 0.0);
    if (iy != Ny && jx != Nx) {
      const int i = iy < Ny ? iy : iy - 2 * Ny;
      const int j = jx < Nx ? jx : jx - 2 * Nx;
      const int b = (int)(e / (Nz * Nz));
      int px, py;
      block_parity(b, px, py);
      const int ai = i < 0 ? -i : i, aj = j < 0 ? -j : j;
      double sgn = 1.0;
      if (i < 0) sgn *= py;
      if (j < 0) sgn *= px;
      const double2 q = qreal[((long long)ai * Nx + aj) * NE + e];
      v = make_double2(sgn * q.x, sgn * q.y);
    }
    emb[t] = v;
  }
}

// spectrum[ky][kx][e - e0] -> packed folded blocks (c128 and c64)
__global__ void pack_kernel(const double2 *__restrict__ spec, double2 *__restrict__ q64, float2 *__restrict__ q32,
                            int Nx, int Ny, int Nz, long long e0, long long E) {
  const long long nf = (long long)(Nx + 1) * (Ny + 1);
  const long long tot = nf * E;
  const long long P = (long long)Nz * (Nz + 1) / 2;
  const long long BS = 2LL * Nz * (2 * Nz + 1);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const long long el = t % E;
    const long long f = t / E;
    const int kxb = (int)(f % (Nx + 1));
    const int kyb = (int)(f / (Nx + 1));
    const long long e = e0 + el;
    const int b = (int)(e / (Nz * Nz));
    const int r = (int)(e % (Nz * Nz));
    const int a = r / Nz, c = r % Nz;
    long long dst;
    if (b < 4) {
      if (c < a) continue;
      dst = b * P + (long long)a * Nz - (long long)a * (a - 1) / 2 + (c - a);
    } else {
      dst = 4 * P + (long long)(b - 4) * Nz * Nz + r;
    }
    const double2 v = spec[((long long)kyb * 2 * Nx + kxb) * E + el];
    const long long o = f * BS + dst;
    q64[o] = v;
    q32[o] = make_float2((float)v.x, (float)v.y);
  }
}

__global__ void cast64to32(const double2 *__restrict__ a, float2 *__restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = make_float2((float)a[i].x, (float)a[i].y);
}
__global__ void cast32to64(const float2 *__restrict__ a, double2 *__restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = make_double2((double)a[i].x, (double)a[i].y);
}

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  if (g > 152LL * 64) g = 152LL * 64;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

void launch_embed(const double2 *qreal, double2 *emb, int Nx, int Ny, int Nz, long long e0, long long E,
                  cudaStream_t s) {
  count_launches(1);
  embed_kernel<<<grid_for(4LL * Nx * Ny * E), 256, 0, s>>>(qreal, emb, Nx, Ny, Nz, e0, E);
}

void launch_pack(const double2 *spec, double2 *q64, float2 *q32, int Nx, int Ny, int Nz, long long e0, long long E,
                 cudaStream_t s) {
  count_launches(1);
  pack_kernel<<<grid_for((long long)(Nx + 1) * (Ny + 1) * E), 256, 0, s>>>(spec, q64, q32, Nx, Ny, Nz, e0, E);
}

void launch_cast64to32(const double2 *a, float2 *b, long long n, cudaStream_t s) {
  count_launches(1);
  cast64to32<<<grid_for(n), 256, 0, s>>>(a, b, n);
}
void launch_cast32to64(const float2 *a, double2 *b, long long n, cudaStream_t s) {
  count_launches(1);
  cast32to64<<<grid_for(n), 256, 0, s>>>(a, b, n);
}

}  // namespace ie
