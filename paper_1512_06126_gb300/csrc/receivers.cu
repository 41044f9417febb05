// Fields at MT receivers, the impedance misfit and its adjoint gradient.
//
// The field at a receiver outside the domain is the normal field plus the sum over
// cells of the receiver kernels times the cell current J = (sigma_a - sigma_b) E =
// 2 s gamma U (eq. (APR_lab)).  Only anomalous cells carry current, so the sums skip
// cells whose factor 2 s gamma is zero.  The kernels are stored for offsets in the
// non-negative quadrant; a negative offset flips the sign of the kernels that are odd
// in it: those built from d/dx (E_xz, H_yz) are odd in x, from d/dy (E_yz, H_xz) odd
// in y, from d2/dxdy (E_xy, H_xx) odd in both; the rest are even.
#include "receivers.cuh"

namespace ie {
namespace {

constexpr int kRT = 256;
constexpr int kE = 10;

__device__ __forceinline__ double2 cm(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 ca(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cs(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ void cfma2(double2 &acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

// The 2 x 3 kernels GE (rows Ex, Ey) and GH (rows Hx, Hy) for receiver-minus-cell
// offset (di, dj) and source z-cell b.
struct Kern {
  double2 e[2][3], h[2][3];
};
__device__ __forceinline__ Kern load_kern(const double2 *tab, int di, int dj, int b, int nx, int nz) {
  const double sx = dj < 0 ? -1.0 : 1.0, sy = di < 0 ? -1.0 : 1.0;
  const int ai = di < 0 ? -di : di, aj = dj < 0 ? -dj : dj;
  const double2 *t = tab + (((size_t)ai * nx + aj) * nz + b) * kE;
  Kern K;
  const double2 exy = cs(__ldg(t + 2), sx * sy);
  K.e[0][0] = __ldg(t + 0);
  K.e[0][1] = exy;
  K.e[0][2] = cs(__ldg(t + 3), sx);
  K.e[1][0] = exy;
  K.e[1][1] = __ldg(t + 1);
  K.e[1][2] = cs(__ldg(t + 4), sy);
  const double2 hxx = cs(__ldg(t + 5), sx * sy);
  K.h[0][0] = hxx;
  K.h[0][1] = __ldg(t + 7);
  K.h[0][2] = cs(__ldg(t + 8), sy);
  K.h[1][0] = __ldg(t + 6);
  K.h[1][1] = cs(hxx, -1.0);
  K.h[1][2] = cs(__ldg(t + 9), sx);
  return K;
}

// Kernels of receiver r for the cell at (i, j, b): di = rec_iy[r] - i, dj = rec_ix[r] - j.
// grp == NULL: the quadrant table above.  Otherwise receivers at arbitrary sites: tab
// holds one table per group of sites that share a sub-cell position,
// [group][2 Ny][2 Nx][Nz][10] over di in [-Ny, Ny), dj in [-Nx, Nx), signs included.
__device__ __forceinline__ Kern load_kern_r(const double2 *tab, const int *grp, int r, int di, int dj, int b, int nx,
                                            int ny, int nz) {
  if (!grp) return load_kern(tab, di, dj, b, nx, nz);
  const double2 *t =
      tab + (((((size_t)__ldg(grp + r) * 2 * ny + (di + ny)) * 2 * nx + (dj + nx)) * nz + b) * kE);
  Kern K;
  K.e[0][0] = __ldg(t + 0);
  K.e[0][1] = K.e[1][0] = __ldg(t + 2);
  K.e[0][2] = __ldg(t + 3);
  K.e[1][1] = __ldg(t + 1);
  K.e[1][2] = __ldg(t + 4);
  K.h[0][0] = __ldg(t + 5);
  K.h[0][1] = __ldg(t + 7);
  K.h[0][2] = __ldg(t + 8);
  K.h[1][0] = __ldg(t + 6);
  K.h[1][1] = cs(K.h[0][0], -1.0);
  K.h[1][2] = __ldg(t + 9);
  return K;
}

// One CTA per receiver; 4 * nrhs complex sums reduced over the CTA.
__global__ void __launch_bounds__(kRT) receiver_fields_kernel(const double2 *__restrict__ tab,
                                                              const int *__restrict__ rec_ix,
                                                              const int *__restrict__ rec_iy,
                                                              const int *__restrict__ rec_grp,
                                                              const double2 *__restrict__ u,
                                                              const double2 *__restrict__ jfac, int nrhs, int nx,
                                                              int ny, int nz, int4 pols, double2 en, double2 hn,
                                                              double2 *__restrict__ f, int n_rec) {
  __shared__ double2 red[kRT / 32][16];
  const int r = blockIdx.x;
  const int rx = rec_ix[r], ry = rec_iy[r];
  const long long N = (long long)nx * ny * nz;
  double2 acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[p][k] = make_double2(0.0, 0.0);
  for (long long m = threadIdx.x; m < N; m += kRT) {
    const double2 jf = jfac[m];
    if (jf.x == 0.0 && jf.y == 0.0) continue;
    const int j = (int)(m % nx), i = (int)((m / nx) % ny), b = (int)(m / ((long long)nx * ny));
    const Kern K = load_kern_r(tab, rec_grp, r, ry - i, rx - j, b, nx, ny, nz);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      if (p >= nrhs) break;
      double2 J[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) J[c] = cm(jf, u[((long long)p * 3 + c) * N + m]);
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          cfma2(acc[p][a], K.e[a][c], J[c]);
          cfma2(acc[p][2 + a], K.h[a][c], J[c]);
        }
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double2 v = acc[p][k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
      }
      if (lane == 0) red[wid][p * 4 + k] = v;
    }
  __syncthreads();
  if (threadIdx.x < 4 * nrhs) {
    const int p = threadIdx.x / 4, k = threadIdx.x % 4;
    double2 v = make_double2(0.0, 0.0);
    for (int w = 0; w < kRT / 32; ++w) v = ca(v, red[w][p * 4 + k]);
    const int pol = p == 0 ? pols.x : (p == 1 ? pols.y : (p == 2 ? pols.z : pols.w));
    if (pol == 0) {
      if (k == 0) v = ca(v, en);
      if (k == 3) v = ca(v, hn);
    } else {
      if (k == 1) v = ca(v, en);
      if (k == 2) v = ca(v, cs(hn, -1.0));
    }
    f[((long long)p * n_rec + r) * 4 + k] = v;
  }
}

// One thread per cell: the transpose of the receiver operator, scaled by jfac.
__global__ void __launch_bounds__(kRT) receiver_adjoint_kernel(const double2 *__restrict__ tab,
                                                               const int *__restrict__ rec_ix,
                                                               const int *__restrict__ rec_iy,
                                                               const int *__restrict__ rec_grp, int n_rec,
                                                               const double2 *__restrict__ cvec,
                                                               const double2 *__restrict__ jfac, int nrhs, int nx,
                                                               int ny, int nz, double2 *__restrict__ rhs) {
  const long long N = (long long)nx * ny * nz;
  for (long long m = blockIdx.x * (long long)kRT + threadIdx.x; m < N; m += (long long)gridDim.x * kRT) {
    const double2 jf = jfac[m];
    double2 q[4][3];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int c = 0; c < 3; ++c) q[p][c] = make_double2(0.0, 0.0);
    if (!(jf.x == 0.0 && jf.y == 0.0)) {
      const int j = (int)(m % nx), i = (int)((m / nx) % ny), b = (int)(m / ((long long)nx * ny));
      for (int r = 0; r < n_rec; ++r) {
        const Kern K = load_kern_r(tab, rec_grp, r, __ldg(rec_iy + r) - i, __ldg(rec_ix + r) - j, b, nx, ny, nz);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          if (p >= nrhs) break;
          const double2 *cr = cvec + ((long long)p * n_rec + r) * 4;
          const double2 c0 = __ldg(cr), c1 = __ldg(cr + 1), c2 = __ldg(cr + 2), c3 = __ldg(cr + 3);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            cfma2(q[p][c], K.e[0][c], c0);
            cfma2(q[p][c], K.e[1][c], c1);
            cfma2(q[p][c], K.h[0][c], c2);
            cfma2(q[p][c], K.h[1][c], c3);
          }
        }
      }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      if (p >= nrhs) break;
#pragma unroll
      for (int c = 0; c < 3; ++c) rhs[((long long)p * 3 + c) * N + m] = cm(jf, q[p][c]);
    }
  }
}

// Apparent resistivity |Z|^2 / (w mu0) (ohm m) and phase arg Z (degrees) of n impedance
// entries (the MT maps)
__global__ void mt_apparent_kernel(const double2 *__restrict__ z, int n, double omega, double *__restrict__ rho,
                                   double *__restrict__ phase) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double2 v = z[k];
  const double mu0 = 4.0e-7 * 3.14159265358979323846;
  rho[k] = (v.x * v.x + v.y * v.y) / (omega * mu0);
  phase[k] = atan2(v.y, v.x) * (180.0 / 3.14159265358979323846);
}

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// 2 x 2 complex products, row-major m[0..3] = [[m0, m1], [m2, m3]]
__device__ __forceinline__ void mm2(const double2 *a, const double2 *b, double2 *c) {
  c[0] = ca(cm(a[0], b[0]), cm(a[1], b[2]));
  c[1] = ca(cm(a[0], b[1]), cm(a[1], b[3]));
  c[2] = ca(cm(a[2], b[0]), cm(a[3], b[2]));
  c[3] = ca(cm(a[2], b[1]), cm(a[3], b[3]));
}

__global__ void mt_misfit_kernel(const double2 *__restrict__ f, const double2 *__restrict__ zobs, int n_rec,
                                 double2 *__restrict__ z, double *__restrict__ phi_r, double2 *__restrict__ cvec) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rec) return;
  const double2 *f0 = f + (long long)r * 4, *f1 = f + ((long long)n_rec + r) * 4;
  // E = [[Ex1, Ex2], [Ey1, Ey2]], H = [[Hx1, Hx2], [Hy1, Hy2]] (columns: polarisations)
  const double2 E[4] = {f0[0], f1[0], f0[1], f1[1]};
  const double2 H[4] = {f0[2], f1[2], f0[3], f1[3]};
  const double2 det = csub(cm(H[0], H[3]), cm(H[1], H[2]));
  const double2 Hi[4] = {cdiv(H[3], det), cdiv(cs(H[1], -1.0), det), cdiv(cs(H[2], -1.0), det), cdiv(H[0], det)};
  double2 Z[4];
  mm2(E, Hi, Z);
  double2 DT[4];  // (conj(Z - Zobs))^T
  double phi = 0.0;
  for (int k = 0; k < 4; ++k) {
    const double2 d = csub(Z[k], zobs[(long long)r * 4 + k]);
    phi += d.x * d.x + d.y * d.y;
    z[(long long)r * 4 + k] = Z[k];
    DT[(k % 2) * 2 + k / 2] = cconj(d);
  }
  phi_r[r] = 0.5 * phi;
  double2 M[4], MZ[4];
  mm2(Hi, DT, M);
  mm2(M, Z, MZ);
  // polarisation j: c^E_i = M[j][i], c^H_i = -(M Z)[j][i]
  for (int j = 0; j < 2; ++j) {
    double2 *c = cvec + ((long long)j * n_rec + r) * 4;
    c[0] = M[j * 2 + 0];
    c[1] = M[j * 2 + 1];
    c[2] = cs(MZ[j * 2 + 0], -1.0);
    c[3] = cs(MZ[j * 2 + 1], -1.0);
  }
}

__global__ void gradient_kernel(const double2 *__restrict__ u, const double2 *__restrict__ w,
                                const double2 *__restrict__ gdiv, int nrhs, long long N, double *__restrict__ grad) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N; m += (long long)gridDim.x * blockDim.x) {
    const double2 g = gdiv[m];
    if (g.x == 0.0 && g.y == 0.0) continue;
    double2 acc = make_double2(0.0, 0.0);
    for (int p = 0; p < nrhs; ++p)
      for (int c = 0; c < 3; ++c) {
        const long long o = ((long long)p * 3 + c) * N + m;
        cfma2(acc, w[o], u[o]);
      }
    grad[m] += g.x * acc.x - g.y * acc.y;
  }
}

// e[p][c][m] = u[p][c][m] * fac[m]: the in-cell field E = U / a of every component
__global__ void cell_scale_kernel(const double2 *__restrict__ u, const double2 *__restrict__ fac, long long N,
                                  long long total, double2 *__restrict__ e) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    e[i] = cm(u[i], __ldg(fac + i % N));
}

int grid_for(long long n) {
  long long g = (n + kRT - 1) / kRT;
  return (int)(g < 1 ? 1 : (g > 152LL * 16 ? 152LL * 16 : g));
}

}  // namespace

void launch_receiver_fields(const double2 *tab, const int *rec_ix, const int *rec_iy, const int *rec_grp,
                            int n_rec, const double2 *u, const double2 *jfac, int nrhs, int nx, int ny, int nz,
                            int pol0, int pol1, int pol2, int pol3, double2 en, double2 hn, double2 *f,
                            cudaStream_t s) {
  count_launches(1);
  receiver_fields_kernel<<<n_rec, kRT, 0, s>>>(tab, rec_ix, rec_iy, rec_grp, u, jfac, nrhs, nx, ny, nz,
                                               make_int4(pol0, pol1, pol2, pol3), en, hn, f, n_rec);
}

void launch_receiver_adjoint(const double2 *tab, const int *rec_ix, const int *rec_iy, const int *rec_grp,
                             int n_rec, const double2 *c, const double2 *jfac, int nrhs, int nx, int ny, int nz,
                             double2 *rhs, cudaStream_t s) {
  count_launches(1);
  receiver_adjoint_kernel<<<grid_for((long long)nx * ny * nz), kRT, 0, s>>>(tab, rec_ix, rec_iy, rec_grp, n_rec, c,
                                                                           jfac, nrhs, nx, ny, nz, rhs);
}

void launch_mt_apparent(const double2 *z, int n, double omega, double *rho, double *phase, cudaStream_t s) {
  count_launches(1);
  mt_apparent_kernel<<<(n + 127) / 128, 128, 0, s>>>(z, n, omega, rho, phase);
}

void launch_mt_misfit(const double2 *f, const double2 *zobs, int n_rec, double2 *z, double *phi_r, double2 *c,
                      cudaStream_t s) {
  count_launches(1);
  mt_misfit_kernel<<<(n_rec + 127) / 128, 128, 0, s>>>(f, zobs, n_rec, z, phi_r, c);
}

void launch_gradient_accumulate(const double2 *u, const double2 *w, const double2 *gdiv, int nrhs, long long ncell,
                                double *grad, cudaStream_t s) {
  count_launches(1);
  gradient_kernel<<<grid_for(ncell), kRT, 0, s>>>(u, w, gdiv, nrhs, ncell, grad);
}

void launch_cell_scale(const double2 *u, const double2 *fac, int nvec, long long ncell, double2 *e, cudaStream_t s) {
  count_launches(1);
  const long long total = (long long)nvec * ncell;
  cell_scale_kernel<<<grid_for(total), kRT, 0, s>>>(u, fac, ncell, total, e);
}

}  // namespace ie
