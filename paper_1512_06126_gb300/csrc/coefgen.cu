// Device generator of the Galerkin coefficients B_n^m (Appendices A-C of the paper):
// the compressed real-space tensor Q(i, j) = B for lateral offsets i in [0, Ny),
// j in [0, Nx), block order xx, yy, zz, xy, xz, yz.
//
//   4 pi B_xx = I1 + Ixx, 4 pi B_yy = I1 + Iyy, 4 pi B_zz = I2 + Izz,
//   4 pi B_xy = Ixy, 4 pi B_xz = Ix, 4 pi B_yz = Iy                    (Appendix A)
//   I1 = int K_J V1 lam dlam,  I2 = int K_J V2 lam dlam,  Izz = int K_J V5 lam dlam,
//   Ix = int K_x V4 lam dlam,  Ixx = int K_xx (V1 + V3) dlam / lam,     eq. (Hor_Int)
//
// with the vertical integrals V1..V5 of eq. (Ver_Int) of the fundamental functions
// U_1, U_sigma (Appendix B: recursions (pq_req), amplitudes (A_rs), the
// overflow-free form (UU2), integrated analytically over the cells) and the lateral
// kernels K of two rectangular cells (the function K(R lam; p, q, phi) of eq. (transf)
// and its lateral derivatives), evaluated from the 2-D Fourier form of J0:
//   K_J = (2/pi) int_0^{pi/2} T_hx(lam cos t) T_hy(lam sin t) cos(lam cos t Dx) cos(lam sin t Dy) dt,
//   T_h(k) = h^2 sinc^2(k h / 2).
//
// Organisation (separable in lambda, like the digital filter of Appendix C whose
// knots and weights depend on the lateral geometry only):
//   1. F[t][pair] = V-kinds at a master grid of lambda, uniform in ln(lambda);
//   2. W[offset][t] = lateral weights: for each offset, Gauss-Legendre panels in lambda
//      (width min(lam/4, pi/R_max)), the lateral kernels at the knots, spread onto the
//      master grid with 8-point Lagrange interpolation in ln(lambda);
//   3. Q = W F by plain matrix products (cuBLAS DGEMM);
//   4. for footprints that touch (|i|, |j| <= 1) the quasi-static part of the
//      U_sigma kinds is subtracted from F and added back from closed-form box
//      integrals of 1/r; separated footprints are integrated under a smooth window
//      0.5 erfc((lam - C/R_min) / (W/R_min)) instead.
// V3 enters Ixx, Iyy, Ixy as the classical derivative (without the delta of
// d/dz d/dz* U at z = z*), the zx, zy blocks follow from Lemma 1.
#include "coefgen.cuh"

#include <cublas_v2.h>
#include <thrust/complex.h>

#include <algorithm>
#include <cmath>
#include <vector>

namespace ie {
namespace {

using zc = thrust::complex<double>;
constexpr double kPi = 3.14159265358979323846;
constexpr double kMu0 = 4e-7 * kPi;
constexpr int kMaxLay = 24;  // interfaces supported by the generator

struct LayDev {
  int L;                       // number of interfaces d_1..d_L
  double d[kMaxLay + 2];       // d_0 .. d_{L+1} with d_0 = d_1 and d_{L+1} = d_L
  double l[kMaxLay + 1];       // l_m = d_{m+1} - d_m for m = 1..L-1; l_0 = l_L = 0
  double sr[kMaxLay + 1], si[kMaxLay + 1];  // sigma_0 .. sigma_L
};

struct GridDev {
  int nz;
  double ze[257];
  int lay[256];
};

__device__ __forceinline__ zc sig(const LayDev &L, int m) { return zc(L.sr[m], L.si[m]); }

// ---------------------------------------------------------------------------
// 1. Spectra: eta, p, q, A_nn and the transfer factors of (pq_req), (A_rs)
//    out[(g * T + t) * (L+1) + m] * 5 fields: eta, p, q, Ann, tf
// ---------------------------------------------------------------------------
__global__ void spectra_kernel(int T, double t0, double dt, double omega, LayDev L, zc *out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  const double lam = exp(t0 + dt * t);
  const int nl = L.L + 1;
  for (int g = 0; g < 2; ++g) {
    zc *o = out + ((size_t)g * T + t) * nl * 5;
    zc eta[kMaxLay + 1], p[kMaxLay + 1], q[kMaxLay + 1];
    for (int m = 0; m < nl; ++m) eta[m] = thrust::sqrt(zc(lam * lam, 0.0) - zc(0.0, omega * kMu0) * sig(L, m));
    p[0] = 0.0;
    for (int m = 0; m < L.L; ++m) {
      const zc e = p[m] * thrust::exp(-2.0 * eta[m] * L.l[m]);
      const zc X = (e - 1.0) / (e + 1.0);
      const zc al = g == 0 ? zc(1.0) : sig(L, m + 1) / sig(L, m);
      const zc ra = al * eta[m] / eta[m + 1];
      p[m + 1] = (1.0 + ra * X) / (1.0 - ra * X);
    }
    q[L.L] = 0.0;
    for (int m = L.L; m >= 1; --m) {
      const zc e = q[m] * thrust::exp(-2.0 * eta[m] * L.l[m]);
      const zc Y = (e - 1.0) / (e + 1.0);
      const zc be = g == 0 ? zc(1.0) : sig(L, m - 1) / sig(L, m);
      const zc rb = be * eta[m] / eta[m - 1];
      q[m - 1] = (1.0 + rb * Y) / (1.0 - rb * Y);
    }
    for (int m = 0; m < nl; ++m) {
      const zc ann = 1.0 / (eta[m] * (1.0 - p[m] * q[m] * thrust::exp(-2.0 * eta[m] * L.l[m])));
      const zc tf = m < L.L ? (1.0 + p[m + 1]) / (1.0 + p[m] * thrust::exp(-2.0 * eta[m] * L.l[m])) : zc(1.0);
      o[m * 5 + 0] = eta[m];
      o[m * 5 + 1] = p[m];
      o[m * 5 + 2] = q[m];
      o[m * 5 + 3] = ann;
      o[m * 5 + 4] = tf;
    }
  }
}

// ---------------------------------------------------------------------------
// 2. Vertical integrals for every (t, field cell a, source cell b)
// ---------------------------------------------------------------------------
struct Term {
  zc c, az, azs, k;
  int tag;  // 0: depends on z*-z and decays, 1: separable, 2: depends on z*-z and grows
};

struct Terms {
  Term t[4];
  int n;
};

// terms of U(z, z*) for z in layer r, z* in layer s; below: z > z*
__device__ Terms full_terms(const zc *sp, int nl, const LayDev &L, bool gsig, int r, int s, bool below) {
  const int up = below ? s : r, lo = below ? r : s;
  auto eta = [&](int m) { return sp[m * 5 + 0]; };
  zc amp = sp[lo * 5 + 3];
  for (int m = up; m < lo; ++m) amp *= sp[m * 5 + 4];
  if (below && gsig && r != s) amp *= sig(L, r) / sig(L, s);
  const zc eu = eta(up), el = eta(lo);
  zc c0 = 0.0;
  if (up != lo) {
    c0 = -eu * L.d[up + 1] + el * L.d[lo];
    for (int m = up + 1; m < lo; ++m) c0 -= eta(m) * L.l[m];
  }
  const zc pu = sp[up * 5 + 1], ql = sp[lo * 5 + 2];
  Terms T;
  T.n = 0;
  T.t[T.n++] = {amp, eu, -el, c0, 0};
  if (up >= 1) T.t[T.n++] = {amp * pu, -eu, -el, c0 + 2.0 * eu * L.d[up], 1};
  if (lo < L.L) T.t[T.n++] = {amp * ql, eu, el, c0 - 2.0 * el * L.d[lo + 1], 1};
  if (up >= 1 && lo < L.L) T.t[T.n++] = {amp * pu * ql, -eu, el, c0 + 2.0 * eu * L.d[up] - 2.0 * el * L.d[lo + 1], 2};
  if (below)
    for (int i = 0; i < T.n; ++i) { zc tmp = T.t[i].az; T.t[i].az = T.t[i].azs; T.t[i].azs = tmp; }
  return T;
}

// quasi-static U_sigma: c e^{-lam|z-z*|}/lam (+ images within one layer)
__device__ void static_coefs(const LayDev &L, int r, int s, zc &c, zc &pt, zc &pb) {
  c = 0.0; pt = 0.0; pb = 0.0;
  if (r == s) {
    c = 1.0;
    if (r >= 1) pt = (sig(L, r - 1) - sig(L, r)) / (sig(L, r - 1) + sig(L, r));
    if (r < L.L) pb = (sig(L, r + 1) - sig(L, r)) / (sig(L, r + 1) + sig(L, r));
  } else if (r - s == 1 || s - r == 1) {
    c = 2.0 * sig(L, r) / (sig(L, r) + sig(L, s));
  }
}

__device__ Terms static_terms(const LayDev &L, double lam, int r, int s, bool below) {
  zc c, pt, pb;
  static_coefs(L, r, s, c, pt, pb);
  Terms T;
  T.n = 0;
  if (c == zc(0.0)) return T;
  const double il = 1.0 / lam;
  T.t[T.n++] = below ? Term{c * il, -lam, lam, 0.0, 0} : Term{c * il, lam, -lam, 0.0, 0};
  if (r == s && pt != zc(0.0)) T.t[T.n++] = {pt * il, -lam, -lam, 2.0 * lam * L.d[r], 1};
  if (r == s && pb != zc(0.0)) T.t[T.n++] = {pb * il, lam, lam, -2.0 * lam * L.d[r + 1], 1};
  return T;
}

// int_{x1}^{x2} e^{a x} dx = e^{a ref} * f  (ref: end where Re(a x) is largest)
__device__ __forceinline__ void int_exp(zc a, double x1, double x2, double &ref, zc &f) {
  const double h = x2 - x1;
  if (thrust::abs(a) * h < 1e-9) { ref = x1; f = h * (1.0 + 0.5 * a * h); return; }
  if (a.real() >= 0) { ref = x2; f = (1.0 - thrust::exp(-a * h)) / a; }
  else { ref = x1; f = (thrust::exp(a * h) - 1.0) / a; }
}

// (x - 1 + e^{-x}) / x^2 and (1 - e^{-x}(1 + x)) / x^2 with series for small |x|
__device__ zc phi_ab(zc x) {
  if (thrust::abs(x) < 0.05) {
    zc s = 0.0, term = 0.5;
    for (int k = 2; k < 14; ++k) { s += term; term *= -x / double(k + 1); }
    return s;
  }
  return (x - 1.0 + thrust::exp(-x)) / (x * x);
}
__device__ zc psi_ab(zc x) {
  if (thrust::abs(x) < 0.05) {
    zc s = 0.0, pw = 1.0;
    double fact = 2.0;
    for (int k = 2; k < 16; ++k) {
      s += ((k % 2) ? -1.0 : 1.0) * double(k - 1) * pw / fact;
      pw *= x;
      fact *= double(k + 1);
    }
    return s * 1.0;
  }
  return (1.0 - thrust::exp(-x) * (1.0 + x)) / (x * x);
}

__device__ __forceinline__ zc eval_terms(const Terms &T, double z, double zs) {
  zc acc = 0.0;
  for (int i = 0; i < T.n; ++i) acc += T.t[i].c * thrust::exp(T.t[i].az * z + T.t[i].azs * zs + T.t[i].k);
  return acc;
}

__device__ __forceinline__ zc F_terms(const Terms &T, double z0, double w1, double w2, bool deriv) {
  zc acc = 0.0;
  for (int i = 0; i < T.n; ++i) {
    double wr;
    zc f;
    int_exp(T.t[i].azs, w1, w2, wr, f);
    zc v = T.t[i].c * thrust::exp(T.t[i].az * z0 + T.t[i].azs * wr + T.t[i].k) * f;
    acc += deriv ? T.t[i].az * v : v;
  }
  return acc;
}

__device__ zc DD_disjoint(const Terms &T, double z1, double z2, double w1, double w2) {
  zc acc = 0.0;
  for (int i = 0; i < T.n; ++i) {
    double zr, wr;
    zc fa, fb;
    int_exp(T.t[i].az, z1, z2, zr, fa);
    int_exp(T.t[i].azs, w1, w2, wr, fb);
    acc += T.t[i].c * thrust::exp(T.t[i].az * zr + T.t[i].azs * wr + T.t[i].k) * fa * fb;
  }
  return acc;
}

__device__ zc DD_self(const Terms &T, double z1, double z2) {
  const double h = z2 - z1;
  zc acc = 0.0;
  for (int i = 0; i < T.n; ++i) {
    const Term &q = T.t[i];
    if (q.tag == 0) {
      acc += q.c * thrust::exp(q.k) * 2.0 * h * h * phi_ab(q.az * h);
    } else if (q.tag == 2) {
      acc += q.c * thrust::exp(q.k + q.azs * h) * 2.0 * h * h * psi_ab(q.azs * h);
    } else {
      double zr, wr;
      zc fa, fb;
      int_exp(q.az, z1, z2, zr, fa);
      int_exp(q.azs, z1, z2, wr, fb);
      acc += q.c * thrust::exp(q.az * zr + q.azs * wr + q.k) * fa * fb;
    }
  }
  return acc;
}

struct PairQ {
  zc DD, F1, F2, Fz1, Fz2, U11, U12, U21, U22;
};

template <typename TF>
__device__ PairQ pair_q(TF terms, double z1, double z2, double w1, double w2) {
  PairQ Q;
  if (z2 <= w1 || z1 >= w2) {
    const Terms T = terms(!(z2 <= w1));
    Q.DD = DD_disjoint(T, z1, z2, w1, w2);
    Q.F1 = F_terms(T, z1, w1, w2, false);
    Q.F2 = F_terms(T, z2, w1, w2, false);
    Q.Fz1 = F_terms(T, z1, w1, w2, true);
    Q.Fz2 = F_terms(T, z2, w1, w2, true);
    Q.U11 = eval_terms(T, z1, w1);
    Q.U12 = eval_terms(T, z1, w2);
    Q.U21 = eval_terms(T, z2, w1);
    Q.U22 = eval_terms(T, z2, w2);
  } else {
    const Terms Ta = terms(false), Tb = terms(true);
    Q.DD = DD_self(Ta, z1, z2);
    Q.F1 = F_terms(Ta, z1, w1, w2, false);
    Q.F2 = F_terms(Tb, z2, w1, w2, false);
    Q.Fz1 = F_terms(Ta, z1, w1, w2, true);
    Q.Fz2 = F_terms(Tb, z2, w1, w2, true);
    Q.U11 = eval_terms(Ta, z1, w1);
    Q.U12 = eval_terms(Ta, z1, w2);
    Q.U21 = eval_terms(Tb, z2, w1);
    Q.U22 = eval_terms(Ta, z2, w2);
  }
  return Q;
}

// F layout: F[kind][t][a * Nz + b], kinds: 0 V1, 1 V2, 2 V3p (classical), 3 V4, 4 V5,
// 5 V3 - V3st (cell-face forms; the delta cancels), 6 V4 - V4st, 7 V5 - V5st
constexpr int kNF = 8;

__global__ void vertical_kernel(int T, double t0, double dt, double omega, LayDev L, GridDev G, const zc *spec,
                                zc *F) {
  const int nz = G.nz;
  const long long np = (long long)nz * nz;
  const long long tot = (long long)T * np;
  const int nl = L.L + 1;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot;
       id += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(id / np);
    const int pr = (int)(id % np);
    const int a = pr / nz, b = pr % nz;
    const double lam = exp(t0 + dt * t);
    const double z1 = G.ze[a], z2 = G.ze[a + 1], w1 = G.ze[b], w2 = G.ze[b + 1];
    const int r = G.lay[a], s = G.lay[b];
    const zc *sp1 = spec + ((size_t)0 * T + t) * nl * 5;
    const zc *sps = spec + ((size_t)1 * T + t) * nl * 5;
    const PairQ q1 = pair_q([&](bool below) { return full_terms(sp1, nl, L, false, r, s, below); }, z1, z2, w1, w2);
    const PairQ qs = pair_q([&](bool below) { return full_terms(sps, nl, L, true, r, s, below); }, z1, z2, w1, w2);
    const PairQ qt = pair_q([&](bool below) { return static_terms(L, lam, r, s, below); }, z1, z2, w1, w2);
    const zc iwm = zc(0.0, omega * kMu0);
    const zc inv = 1.0 / sig(L, r);
    const double ovl = (a == b) ? (z2 - z1) : 0.0;
    const zc V3w = -inv * (qs.U22 - qs.U21 - qs.U12 + qs.U11);
    const zc V3s = -inv * (qt.U22 - qt.U21 - qt.U12 + qt.U11);
    const zc V4 = inv * (qs.F2 - qs.F1), V4s = inv * (qt.F2 - qt.F1);
    const zc V5 = inv * (qs.Fz2 - qs.Fz1), V5s = inv * (qt.Fz2 - qt.Fz1);
    const long long st = (long long)T * np;
    const long long o = (long long)t * np + pr;
    F[0 * st + o] = iwm * q1.DD;
    F[1 * st + o] = iwm * qs.DD;
    F[2 * st + o] = V3w + 2.0 * inv * ovl;
    F[3 * st + o] = V4;
    F[4 * st + o] = V5;
    F[5 * st + o] = V3w - V3s;
    F[6 * st + o] = V4 - V4s;
    F[7 * st + o] = V5 - V5s;
  }
}

// ---------------------------------------------------------------------------
// 3. Lateral weights on the master grid
//    W[kind][offset][t], kinds: 0 K_J*lam, 1 K_xx/lam, 2 K_yy/lam, 3 K_xy/lam, 4 K_x*lam, 5 K_y*lam
// ---------------------------------------------------------------------------
constexpr int kNW = 6;
constexpr int kGL = 8;
__constant__ double c_glx[kGL], c_glw[kGL];

struct WParams {
  int nx, ny;          // offsets j in [0, nx), i in [0, ny) (the stored quadrant)
  double hx, hy, hmin;
  int T;
  double t0, dt;
  double near_lh, far_c, far_w, panel_rel, lam_low;
  int max_panels;
  int point;           // 1: a point seen from the source rectangle (box transform), 0: two cells (tent)
};

__device__ __forceinline__ double tent_hat(double k, double h) {
  const double x = 0.5 * k * h;
  if (fabs(x) < 1e-8) return h * h;
  const double s = sin(x) / x;
  return h * h * s * s;
}
// transform of the rectangle's indicator (point-to-cell lateral integrals)
__device__ __forceinline__ double box_hat(double k, double h) {
  const double x = 0.5 * k * h;
  if (fabs(x) < 1e-8) return h;
  return h * sin(x) / x;
}

// doffs (may be NULL): real offsets (Dy, Dx) in metres per offset in place of the cell
// offsets offs (i, j) -> (i hy, j hx) (receivers at arbitrary lateral sites)
__global__ void weights_kernel(WParams P, const int *offs, int n_off, double *W, double *edges_ws,
                               const double *doffs = nullptr) {
  extern __shared__ double smw[];  // [kNW][T]
  const int o = blockIdx.x;
  if (o >= n_off) return;
  const double Dx = doffs ? doffs[2 * o + 1] : offs[2 * o + 1] * P.hx;
  const double Dy = doffs ? doffs[2 * o] : offs[2 * o] * P.hy;
  const int T = P.T;
  for (int q = threadIdx.x; q < kNW * T; q += blockDim.x) smw[q] = 0.0;
  const double rmax = hypot(fabs(Dx) + P.hx, fabs(Dy) + P.hy);
  const bool near = fabs(Dx) <= P.hx * (1 + 1e-12) && fabs(Dy) <= P.hy * (1 + 1e-12);
  double lam_end, rmin = 0.0;
  if (near) lam_end = P.near_lh / P.hmin;
  else {
    rmin = hypot(fmax(fabs(Dx) - P.hx, 0.0), fmax(fabs(Dy) - P.hy, 0.0));
    lam_end = (P.far_c + 6.0 * P.far_w) / rmin;
  }
  // panel edges (sequential), kept in global scratch for this CTA
  double *edges = edges_ws + (size_t)blockIdx.x * (P.max_panels + 1);
  __shared__ int n_pan;
  if (threadIdx.x == 0) {
    const double cap = kPi / rmax;
    double e = P.lam_low;
    int n = 0;
    edges[0] = e;
    while (e < lam_end && n < P.max_panels) {
      e = fmin(lam_end, e + fmin(P.panel_rel * e, cap));
      edges[++n] = e;
    }
    n_pan = n;
  }
  __syncthreads();
  const int nn = n_pan * kGL;
  const double band0 = fabs(Dx) + fabs(Dy) + P.hx + P.hy;
  for (int n = threadIdx.x; n < nn; n += blockDim.x) {
    const int pan = n / kGL, g = n % kGL;
    const double a = edges[pan], b = edges[pan + 1];
    const double lam = 0.5 * (b - a) * c_glx[g] + 0.5 * (a + b);
    double w = 0.5 * (b - a) * c_glw[g];
    if (!near) w *= 0.5 * erfc((lam - P.far_c / rmin) / (P.far_w / rmin));
    // lateral kernels by the trapezoidal rule on [0, pi/2]
    const int nt = (int)ceil(0.32 * lam * band0) + 24;
    double kJ = 0, kxx = 0, kyy = 0, kxy = 0, kx = 0, ky = 0;
    for (int q = 0; q <= nt; ++q) {
      const double th = 0.5 * kPi * q / nt;
      double sn, cs;
      sincos(th, &sn, &cs);
      const double kxv = lam * cs, kyv = lam * sn;
      double base = P.point ? box_hat(kxv, P.hx) * box_hat(kyv, P.hy) : tent_hat(kxv, P.hx) * tent_hat(kyv, P.hy);
      if (q == 0 || q == nt) base *= 0.5;
      double sx, cx, sy, cy;
      sincos(kxv * Dx, &sx, &cx);
      sincos(kyv * Dy, &sy, &cy);
      const double bcc = base * cx * cy;
      kJ += bcc;
      kxx -= kxv * kxv * bcc;
      kyy -= kyv * kyv * bcc;
      kxy += kxv * kyv * base * sx * sy;
      kx -= kxv * base * sx * cy;
      ky -= kyv * base * cx * sy;
    }
    const double inv_nt = 1.0 / nt;
    const double vals[kNW] = {kJ * inv_nt * lam * w, kxx * inv_nt / lam * w, kyy * inv_nt / lam * w,
                              kxy * inv_nt / lam * w, kx * inv_nt * lam * w, ky * inv_nt * lam * w};
    // 8-point Lagrange interpolation in ln(lambda) onto the master grid
    const double pos = (log(lam) - P.t0) / P.dt;
    int k0 = (int)floor(pos) - 3;
    k0 = max(0, min(k0, T - 8));
    double Lw[8];
    for (int m = 0; m < 8; ++m) {
      double v = 1.0;
      for (int m2 = 0; m2 < 8; ++m2)
        if (m2 != m) v *= (pos - (k0 + m2)) / double(m - m2);
      Lw[m] = v;
    }
    for (int kind = 0; kind < kNW; ++kind)
      for (int m = 0; m < 8; ++m) atomicAdd(&smw[kind * T + k0 + m], vals[kind] * Lw[m]);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < kNW * T; q += blockDim.x) {
    const int kind = q / T, t = q % T;
    W[((size_t)kind * n_off + o) * T + t] = smw[q];
  }
}

// ---------------------------------------------------------------------------
// 4. Closed-form quasi-static parts for touching footprints
// ---------------------------------------------------------------------------
__device__ __forceinline__ double xlog(double m, double v, double r, double o2) {
  if (m == 0.0) return 0.0;
  if (v >= 0.0) return m * log(v + r);
  if (o2 <= 0.0) return 0.0;
  return m * (log(o2) - log(r - v));
}
__device__ __forceinline__ double xatan(double m, double num, double den) {
  if (den == 0.0) return 0.0;
  return m * atan(num / den);
}
// d^2/dy^2 d^2/dz^2 Pf(x; y, z) = 1/r
__device__ double Pf(double x, double y, double z) {
  const double x2 = x * x, y2 = y * y, z2 = z * z, r = sqrt(x2 + y2 + z2);
  return -0.5 * xlog(x2 * y, y, r, x2 + z2) - 0.5 * xlog(x2 * z, z, r, x2 + y2) + x2 * r / 3.0 -
         xatan(x * y * z, y * z, x * r) + 0.5 * xlog(y2 * z, z, r, x2 + y2) - y2 * r / 6.0 +
         0.5 * xlog(y * z2, y, r, x2 + z2) - z2 * r / 6.0;
}
// d/dx d/dz d^2/dy^2 Nf(x, z; y) = 1/r
__device__ double Nf(double x, double z, double y) {
  const double x2 = x * x, y2 = y * y, z2 = z * z, r = sqrt(x2 + y2 + z2);
  return -xlog(x2 * x, z, r, x2 + y2) / 6.0 - 0.5 * xatan(x2 * y, y * z, x * r) + 0.5 * xlog(x * y2, z, r, x2 + y2) +
         xlog(x * y * z, y, r, x2 + z2) - x * z * r / 3.0 - xatan(y2 * y, x * z, y * r) / 6.0 +
         0.5 * xlog(y2 * z, x, r, y2 + z2) - 0.5 * xatan(y * z2, x * y, z * r) - xlog(z2 * z, x, r, y2 + z2) / 6.0;
}
// kinds: 0 xx, 1 yy, 2 zz, 3 xy, 4 xz, 5 yz
__device__ double box_d2(int kind, double Dx, double Dy, double hx, double hy, double zf1, double zf2, double zs1,
                         double zs2) {
  const double lx[3] = {-1, 0, 1}, lw[3] = {1, -2, 1};
  const double Zs[4] = {zf2 - zs1, zf2 - zs2, zf1 - zs1, zf1 - zs2}, Zw[4] = {1, -1, -1, 1};
  double acc = 0.0;
  for (int ix = 0; ix < 3; ++ix)
    for (int iy = 0; iy < 3; ++iy)
      for (int iz = 0; iz < 4; ++iz) {
        const double X = Dx + lx[ix] * hx, Y = Dy + lx[iy] * hy, Z = Zs[iz];
        double v;
        switch (kind) {
          case 0: v = Pf(X, Y, Z); break;
          case 1: v = Pf(Y, X, Z); break;
          case 2: v = Pf(Z, X, Y); break;
          case 3: v = Nf(X, Y, Z); break;
          case 4: v = Nf(X, Z, Y); break;
          default: v = Nf(Y, Z, X); break;
        }
        acc += lw[ix] * lw[iy] * Zw[iz] * v;
      }
  return acc;
}

// S[near][kind][a][b] (complex), kinds xx, yy, zz, xy, xz, yz
__global__ void statics_kernel(LayDev L, GridDev G, double hx, double hy, const int *offs, int n_near, zc *S) {
  const int nz = G.nz;
  const long long tot = (long long)n_near * 6 * nz * nz;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot;
       id += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(id % nz), a = (int)((id / nz) % nz);
    const int kind = (int)((id / ((long long)nz * nz)) % 6);
    const int o = (int)(id / (6LL * nz * nz));
    const double Dx = offs[2 * o + 1] * hx, Dy = offs[2 * o] * hy;
    const int r = G.lay[a], s = G.lay[b];
    zc c, pt, pb;
    static_coefs(L, r, s, c, pt, pb);
    const double z1 = G.ze[a], z2 = G.ze[a + 1], w1 = G.ze[b], w2 = G.ze[b + 1];
    zc acc = 0.0;
    if (c != zc(0.0)) {
      acc += c * box_d2(kind, Dx, Dy, hx, hy, z1, z2, w1, w2);
      const double img = (kind == 0 || kind == 1 || kind == 3) ? -1.0 : 1.0;
      if (r == s && pt != zc(0.0)) {
        const double dd = L.d[r];
        acc += img * pt * box_d2(kind, Dx, Dy, hx, hy, z1, z2, 2 * dd - w2, 2 * dd - w1);
      }
      if (r == s && pb != zc(0.0)) {
        const double dd = L.d[r + 1];
        acc += img * pb * box_d2(kind, Dx, Dy, hx, hy, z1, z2, 2 * dd - w2, 2 * dd - w1);
      }
      acc /= sig(L, r);
    }
    S[id] = acc;
  }
}

// ---------------------------------------------------------------------------
// 5. Assembly: Q[i][j][blk][a][b] from the products and the statics
//    P[g][offset][col]: g = product index (see generate()), col = 2 * (kindcol * np + pair) + re/im
// ---------------------------------------------------------------------------
__global__ void assemble_kernel(const double *Pfar, const double *Pnear, const zc *S, const int *offs, int n_off,
                                const int *near_idx, int nx, int nz, zc *Q) {
  const long long np = (long long)nz * nz;
  const long long tot = (long long)n_off * 6 * np;
  const double inv4pi = 1.0 / (4.0 * kPi);
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot;
       id += (long long)gridDim.x * blockDim.x) {
    const long long pr = id % np;
    const int blk = (int)((id / np) % 6);
    const int o = (int)(id / (6 * np));
    const int ni = near_idx[o];
    const double *Pm = ni >= 0 ? Pnear : Pfar;
    const long long oo = ni >= 0 ? ni : o;
    const long long nrow = ni >= 0 ? 0 : 0;
    (void)nrow;
    // product layout: for each offset row, 8 complex column groups of np:
    //   0: WJ*V1, 1: WJ*V2, 2: WJ*V5, 3: Wxx*X, 4: Wyy*X, 5: Wxy*X, 6: Wx*V4, 7: Wy*V4
    const double *row = Pm + oo * (8 * 2 * np);
    auto get = [&](int g) { return zc(row[2 * (g * np + pr)], row[2 * (g * np + pr) + 1]); };
    zc v;
    int sk = -1;
    switch (blk) {
      case 0: v = get(0) + get(3); sk = 0; break;
      case 1: v = get(0) + get(4); sk = 1; break;
      case 2: v = get(1) + get(2); sk = 2; break;
      case 3: v = get(5); sk = 3; break;
      case 4: v = get(6); sk = 4; break;
      default: v = get(7); sk = 5; break;
    }
    if (ni >= 0) v += S[((long long)ni * 6 + sk) * np + pr];
    const int i = offs[2 * o], j = offs[2 * o + 1];
    Q[(((long long)i * nx + j) * 6 + blk) * np + pr] = v * inv4pi;
  }
}

// ---------------------------------------------------------------------------
// 6. Receiver kernels (eq. (APR_lab)): E and H at a point at depth z_r above the grid
//    from a cell of uniform current.  Vertical functions of U(z_r, z*) over the source
//    cell [w1, w2] (zero unless w1 > z_r), sigma_r the conductivity at the receiver:
//      0 P1 = i w mu0 int U_1        1 X = P1 - (1/sigma_r) d/dz [U_s(z, w2) - U_s(z, w1)]
//      2 P4 = (1/sigma_r) d/dz int U_s   3 P1z = d/dz int U_1
//      4 Pg = U_s(z_r, w2) - U_s(z_r, w1) + P1z   5 Ps = int U_s
//    Fr layout: Fr[kind][t][b].  With the point lateral weights W (box transform):
//      4 pi E_xx = WJ.P1 + Wxx.X,  4 pi E_yy = WJ.P1 + Wyy.X,  4 pi E_xy = Wxy.X,
//      4 pi E_xz = Wx.P4,          4 pi E_yz = Wy.P4,
//      4 pi H_xx = -Wxy.Pg (= -4 pi H_yy),  4 pi H_yx = WJ.P1z + Wxx.Pg,
//      4 pi H_xy = -WJ.P1z - Wyy.Pg,  4 pi H_xz = Wy.Ps,  4 pi H_yz = -Wx.Ps
//    (GE = (1/k^2)-weighted derivatives of (Ge2); GH = curl of (green_tensor) / (i w mu0)).
// ---------------------------------------------------------------------------
constexpr int kNR = 6;
constexpr int kNRP = 12;  // products
constexpr int kRecEntries = 10;

__global__ void receiver_vertical_kernel(int T, double t0, double dt, double omega, LayDev L, GridDev G,
                                         const zc *spec, double z_r, int r, zc *F) {
  const int nz = G.nz;
  const long long tot = (long long)T * nz;
  const int nl = L.L + 1;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot;
       id += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(id / nz), b = (int)(id % nz);
    const double w1 = G.ze[b], w2 = G.ze[b + 1];
    const long long st = (long long)T * nz, o = (long long)t * nz + b;
    if (!(w1 > z_r)) {
      for (int k = 0; k < kNR; ++k) F[k * st + o] = 0.0;
      continue;
    }
    const int s = G.lay[b];
    const zc *sp1 = spec + ((size_t)0 * T + t) * nl * 5;
    const zc *sps = spec + ((size_t)1 * T + t) * nl * 5;
    const Terms T1 = full_terms(sp1, nl, L, false, r, s, false);
    const Terms Ts = full_terms(sps, nl, L, true, r, s, false);
    const zc F1 = F_terms(T1, z_r, w1, w2, false), F1z = F_terms(T1, z_r, w1, w2, true);
    const zc Fs = F_terms(Ts, z_r, w1, w2, false), Fsz = F_terms(Ts, z_r, w1, w2, true);
    zc dU = 0.0, Ud = 0.0;
    for (int i = 0; i < Ts.n; ++i) {
      const Term &q = Ts.t[i];
      const zc e2 = q.c * thrust::exp(q.az * z_r + q.azs * w2 + q.k);
      const zc e1 = q.c * thrust::exp(q.az * z_r + q.azs * w1 + q.k);
      dU += q.az * (e2 - e1);
      Ud += e2 - e1;
    }
    const zc iwm = zc(0.0, omega * kMu0);
    const zc inv = 1.0 / sig(L, r);
    const zc P1 = iwm * F1;
    F[0 * st + o] = P1;
    F[1 * st + o] = P1 - inv * dU;
    F[2 * st + o] = inv * Fsz;
    F[3 * st + o] = F1z;
    F[4 * st + o] = Ud + F1z;
    F[5 * st + o] = Fs;
  }
}

// tab[((i * nx + j) * nz + b) * 10 + e], e: E_xx, E_yy, E_xy, E_xz, E_yz, H_xx, H_yx, H_xy, H_xz, H_yz
__global__ void receiver_assemble_kernel(const double *P, int n_off, int nz, zc *tab) {
  const long long tot = (long long)n_off * nz;
  const double inv4pi = 1.0 / (4.0 * kPi);
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot;
       id += (long long)gridDim.x * blockDim.x) {
    const int o = (int)(id / nz), b = (int)(id % nz);
    const double *row = P + (size_t)o * kNRP * 2 * nz;
    auto g = [&](int k) { return zc(row[2 * (k * nz + b)], row[2 * (k * nz + b) + 1]); };
    zc *t = tab + ((size_t)o * nz + b) * kRecEntries;
    t[0] = (g(0) + g(1)) * inv4pi;
    t[1] = (g(0) + g(2)) * inv4pi;
    t[2] = g(3) * inv4pi;
    t[3] = g(4) * inv4pi;
    t[4] = g(5) * inv4pi;
    t[5] = -g(6) * inv4pi;
    t[6] = (g(7) + g(8)) * inv4pi;
    t[7] = (-g(7) - g(9)) * inv4pi;
    t[8] = g(10) * inv4pi;
    t[9] = -g(11) * inv4pi;
  }
}

// Gauss-Legendre nodes on [-1, 1] by Newton's iteration on P_n.
void gauss_legendre(int n, double *x, double *w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      const double dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) {
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
        break;
      }
    }
  }
}

int grid1d(long long n) {
  long long g = (n + 255) / 256;
  return (int)std::max<long long>(1, std::min<long long>(g, 152LL * 32));
}

}  // namespace

CoefGenStatus generate_coefficients(const CoefGenInput &in, double2 *q_dev, cudaStream_t s) {
  const int nx = in.nx, ny = in.ny, nz = in.nz;
  if (in.n_interfaces < 1 || in.n_interfaces > kMaxLay || nz > 256) return CoefGenStatus::kUnsupported;
  LayDev L{};
  L.L = in.n_interfaces;
  for (int k = 0; k < L.L; ++k) L.d[k + 1] = in.interfaces[k];
  L.d[0] = L.d[1];
  L.d[L.L + 1] = L.d[L.L];
  for (int m = 0; m <= L.L; ++m) {
    L.l[m] = (m >= 1 && m < L.L) ? L.d[m + 1] - L.d[m] : 0.0;
    L.sr[m] = in.sigma[2 * m];
    L.si[m] = in.sigma[2 * m + 1];
  }
  GridDev G{};
  G.nz = nz;
  for (int k = 0; k <= nz; ++k) G.ze[k] = in.z_edges[k];
  for (int k = 0; k < nz; ++k) G.lay[k] = in.cell_layer[k];
  double hz_min = 1e300;
  for (int k = 0; k < nz; ++k) hz_min = std::min(hz_min, G.ze[k + 1] - G.ze[k]);
  const double hmin = std::min({in.hx, in.hy, hz_min});
  // master grid in ln(lambda)
  const double dt = 0.02, near_lh = 300.0, lam_low = 1e-9;
  const double t0 = std::log(lam_low) - 5 * dt;
  const double t1 = std::log(near_lh / hmin) + 5 * dt;
  const int T = (int)std::ceil((t1 - t0) / dt) + 1;
  const double omega = 2.0 * kPi * in.freq;
  const long long np = (long long)nz * nz;
  CoefGenStatus st = CoefGenStatus::kOk;
  auto ck = [&](cudaError_t e) { if (e != cudaSuccess && st == CoefGenStatus::kOk) st = CoefGenStatus::kCuda; };

  // offsets of the stored quadrant; near ones first in a separate list
  std::vector<int> offs, near_offs, near_idx;
  for (int i = 0; i < ny; ++i)
    for (int j = 0; j < nx; ++j) {
      offs.push_back(i);
      offs.push_back(j);
      if (i <= 1 && j <= 1) {
        near_idx.push_back((int)near_offs.size() / 2);
        near_offs.push_back(i);
        near_offs.push_back(j);
      } else {
        near_idx.push_back(-1);
      }
    }
  const int n_off = nx * ny, n_near = (int)near_offs.size() / 2;

  zc *spec = nullptr, *F = nullptr, *S = nullptr;
  double *W = nullptr, *Wn = nullptr, *edges = nullptr, *Pfar = nullptr, *Pnear = nullptr, *Fr = nullptr;
  int *d_offs = nullptr, *d_near = nullptr, *d_nidx = nullptr;
  const int max_panels = 4000;
  const long long ncol = 8 * 2 * np;  // real columns of one offset row of the products
  ck(cudaMalloc(&spec, sizeof(zc) * 2 * T * (L.L + 1) * 5));
  ck(cudaMalloc(&F, sizeof(zc) * kNF * T * np));
  ck(cudaMalloc(&W, sizeof(double) * kNW * (size_t)n_off * T));
  ck(cudaMalloc(&Wn, sizeof(double) * kNW * (size_t)n_near * T));
  ck(cudaMalloc(&edges, sizeof(double) * (size_t)std::max(n_off, n_near) * (max_panels + 1)));
  ck(cudaMalloc(&Fr, sizeof(double) * (size_t)T * ncol));
  ck(cudaMalloc(&Pfar, sizeof(double) * (size_t)n_off * ncol));
  ck(cudaMalloc(&Pnear, sizeof(double) * (size_t)n_near * ncol));
  ck(cudaMalloc(&S, sizeof(zc) * (size_t)n_near * 6 * np));
  ck(cudaMalloc(&d_offs, sizeof(int) * offs.size()));
  ck(cudaMalloc(&d_near, sizeof(int) * near_offs.size()));
  ck(cudaMalloc(&d_nidx, sizeof(int) * near_idx.size()));
  cublasHandle_t hb = nullptr;
  if (st == CoefGenStatus::kOk && cublasCreate(&hb) != CUBLAS_STATUS_SUCCESS) st = CoefGenStatus::kCuda;
  if (st == CoefGenStatus::kOk) {
    ck(cudaMemcpyAsync(d_offs, offs.data(), sizeof(int) * offs.size(), cudaMemcpyHostToDevice, s));
    ck(cudaMemcpyAsync(d_near, near_offs.data(), sizeof(int) * near_offs.size(), cudaMemcpyHostToDevice, s));
    ck(cudaMemcpyAsync(d_nidx, near_idx.data(), sizeof(int) * near_idx.size(), cudaMemcpyHostToDevice, s));
    double gx[kGL], gw[kGL];
    gauss_legendre(kGL, gx, gw);
    ck(cudaMemcpyToSymbolAsync(c_glx, gx, sizeof(gx), 0, cudaMemcpyHostToDevice, s));
    ck(cudaMemcpyToSymbolAsync(c_glw, gw, sizeof(gw), 0, cudaMemcpyHostToDevice, s));
    count_launches(5);
    spectra_kernel<<<(T + 127) / 128, 128, 0, s>>>(T, t0, dt, omega, L, spec);
    vertical_kernel<<<grid1d((long long)T * np), 256, 0, s>>>(T, t0, dt, omega, L, G, spec, F);
    WParams P{nx, ny, in.hx, in.hy, hmin, T, t0, dt, near_lh, 80.0, 10.0, 0.25, lam_low, max_panels, 0};
    const size_t smw = sizeof(double) * kNW * T;
    cudaFuncSetAttribute(weights_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw);
    weights_kernel<<<n_off, 256, smw, s>>>(P, d_offs, n_off, W, edges);
    weights_kernel<<<n_near, 256, smw, s>>>(P, d_near, n_near, Wn, edges);
    statics_kernel<<<grid1d((long long)n_near * 6 * np), 256, 0, s>>>(L, G, in.hx, in.hy, d_near, n_near, S);
    ck(cudaGetLastError());
    cublasSetStream(hb, s);
    const double one = 1.0, zero = 0.0;
    // real views: F kind k as doubles [t][2*np]
    const long long fst = (long long)T * np;  // complex elements per kind
    auto Fk = [&](int k) { return reinterpret_cast<const double *>(F + (size_t)k * fst); };
    // products: P[o][g*2np + col] = sum_t Wkind[o][t] * F[t][col]
    struct G8 { int wk; int fk; };
    const G8 far8[8] = {{0, 0}, {0, 1}, {0, 4}, {1, -1}, {2, -1}, {3, -1}, {4, 3}, {5, 3}};
    const G8 near8[8] = {{0, 0}, {0, 1}, {0, 7}, {1, -2}, {2, -2}, {3, -2}, {4, 6}, {5, 6}};
    // X = V1 + V3 (classical) for far, V1 + (V3 - V3st) for near, built into Fr
    for (int pass = 0; pass < 2 && st == CoefGenStatus::kOk; ++pass) {
      const bool nearp = pass == 1;
      const int no = nearp ? n_near : n_off;
      if (no == 0) continue;
      const double *Wm = nearp ? Wn : W;
      double *Pm = nearp ? Pnear : Pfar;
      const G8 *tab = nearp ? near8 : far8;
      // X in Fr[t][2np] = V1 + V3x
      {
        const double *v1 = Fk(0);
        const double *v3 = Fk(nearp ? 5 : 2);
        // Fr = v1 + v3 with cuBLAS geam (column-major m = 2np, n = T)
        cublasDgeam(hb, CUBLAS_OP_N, CUBLAS_OP_N, (int)(2 * np), T, &one, v1, (int)(2 * np), &one, v3,
                    (int)(2 * np), Fr, (int)(2 * np));
      }
      for (int g = 0; g < 8; ++g) {
        const double *Bm = tab[g].fk >= 0 ? Fk(tab[g].fk) : Fr;
        const double *Am = Wm + (size_t)tab[g].wk * no * T;
        // row-major C[no][ncol] block at column offset g*2np: C^T (col-major) = B^T A^T
        const cublasStatus_t cs =
            cublasDgemm(hb, CUBLAS_OP_N, CUBLAS_OP_N, (int)(2 * np), no, T, &one, Bm, (int)(2 * np), Am, T, &zero,
                        Pm + (size_t)g * 2 * np, (int)ncol);
        if (cs != CUBLAS_STATUS_SUCCESS) st = CoefGenStatus::kCuda;
      }
    }
    count_launches(1);
    assemble_kernel<<<grid1d((long long)n_off * 6 * np), 256, 0, s>>>(Pfar, Pnear, S, d_offs, n_off, d_nidx, nx, nz,
                                                                      reinterpret_cast<zc *>(q_dev));
    ck(cudaGetLastError());
    ck(cudaStreamSynchronize(s));
  }
  if (hb) cublasDestroy(hb);
  cudaFree(spec); cudaFree(F); cudaFree(W); cudaFree(Wn); cudaFree(edges); cudaFree(Fr);
  cudaFree(Pfar); cudaFree(Pnear); cudaFree(S); cudaFree(d_offs); cudaFree(d_near); cudaFree(d_nidx);
  return st;
}

CoefGenStatus generate_receiver_tables(const CoefGenInput &in, double z_r, int r_layer, double2 *tab_dev,
                                       cudaStream_t s, const double *offs_host, int n_off_host) {
  const int nx = in.nx, ny = in.ny, nz = in.nz;
  if (in.n_interfaces < 1 || in.n_interfaces > kMaxLay || nz > 256) return CoefGenStatus::kUnsupported;
  LayDev L{};
  L.L = in.n_interfaces;
  for (int k = 0; k < L.L; ++k) L.d[k + 1] = in.interfaces[k];
  L.d[0] = L.d[1];
  L.d[L.L + 1] = L.d[L.L];
  for (int m = 0; m <= L.L; ++m) {
    L.l[m] = (m >= 1 && m < L.L) ? L.d[m + 1] - L.d[m] : 0.0;
    L.sr[m] = in.sigma[2 * m];
    L.si[m] = in.sigma[2 * m + 1];
  }
  GridDev G{};
  G.nz = nz;
  for (int k = 0; k <= nz; ++k) G.ze[k] = in.z_edges[k];
  for (int k = 0; k < nz; ++k) G.lay[k] = in.cell_layer[k];
  double hz_min = 1e300;
  for (int k = 0; k < nz; ++k) hz_min = std::min(hz_min, G.ze[k + 1] - G.ze[k]);
  const double hmin = std::min({in.hx, in.hy, hz_min});
  const double dt = 0.02, near_lh = 300.0, lam_low = 1e-9;
  const double t0 = std::log(lam_low) - 5 * dt;
  const double t1 = std::log(near_lh / hmin) + 5 * dt;
  const int T = (int)std::ceil((t1 - t0) / dt) + 1;
  const double omega = 2.0 * kPi * in.freq;
  CoefGenStatus st = CoefGenStatus::kOk;
  auto ck = [&](cudaError_t e) { if (e != cudaSuccess && st == CoefGenStatus::kOk) st = CoefGenStatus::kCuda; };
  std::vector<int> offs;
  for (int i = 0; i < ny; ++i)
    for (int j = 0; j < nx; ++j) { offs.push_back(i); offs.push_back(j); }
  const bool real_offs = offs_host != nullptr;
  if (real_offs && n_off_host < 1) return CoefGenStatus::kUnsupported;
  const int n_off = real_offs ? n_off_host : nx * ny;
  const int max_panels = 4000;
  const long long ncol = (long long)kNRP * 2 * nz;
  zc *spec = nullptr, *F = nullptr;
  double *W = nullptr, *edges = nullptr, *Pm = nullptr, *d_doffs = nullptr;
  int *d_offs = nullptr;
  ck(cudaMalloc(&spec, sizeof(zc) * 2 * T * (L.L + 1) * 5));
  ck(cudaMalloc(&F, sizeof(zc) * kNR * (size_t)T * nz));
  ck(cudaMalloc(&W, sizeof(double) * kNW * (size_t)n_off * T));
  ck(cudaMalloc(&edges, sizeof(double) * (size_t)n_off * (max_panels + 1)));
  ck(cudaMalloc(&Pm, sizeof(double) * (size_t)n_off * ncol));
  ck(cudaMalloc(&d_offs, sizeof(int) * offs.size()));
  if (real_offs) ck(cudaMalloc(&d_doffs, sizeof(double) * 2 * (size_t)n_off));
  cublasHandle_t hb = nullptr;
  if (st == CoefGenStatus::kOk && cublasCreate(&hb) != CUBLAS_STATUS_SUCCESS) st = CoefGenStatus::kCuda;
  if (st == CoefGenStatus::kOk) {
    ck(cudaMemcpyAsync(d_offs, offs.data(), sizeof(int) * offs.size(), cudaMemcpyHostToDevice, s));
    if (real_offs)
      ck(cudaMemcpyAsync(d_doffs, offs_host, sizeof(double) * 2 * (size_t)n_off, cudaMemcpyHostToDevice, s));
    double gx[kGL], gw[kGL];
    gauss_legendre(kGL, gx, gw);
    ck(cudaMemcpyToSymbolAsync(c_glx, gx, sizeof(gx), 0, cudaMemcpyHostToDevice, s));
    ck(cudaMemcpyToSymbolAsync(c_glw, gw, sizeof(gw), 0, cudaMemcpyHostToDevice, s));
    count_launches(4);
    spectra_kernel<<<(T + 127) / 128, 128, 0, s>>>(T, t0, dt, omega, L, spec);
    receiver_vertical_kernel<<<grid1d((long long)T * nz), 256, 0, s>>>(T, t0, dt, omega, L, G, spec, z_r, r_layer, F);
    WParams P{nx, ny, in.hx, in.hy, hmin, T, t0, dt, near_lh, 80.0, 10.0, 0.25, lam_low, max_panels, 1};
    const size_t smw = sizeof(double) * kNW * T;
    cudaFuncSetAttribute(weights_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw);
    weights_kernel<<<n_off, 256, smw, s>>>(P, d_offs, n_off, W, edges, d_doffs);
    ck(cudaGetLastError());
    cublasSetStream(hb, s);
    const double one = 1.0, zero = 0.0;
    const long long fst = (long long)T * nz;
    auto Fk = [&](int k) { return reinterpret_cast<const double *>(F + (size_t)k * fst); };
    // (W kind, F kind) of each product, in the order the assembly expects
    const int prod[kNRP][2] = {{0, 0}, {1, 1}, {2, 1}, {3, 1}, {4, 2}, {5, 2},
                               {3, 4}, {0, 3}, {1, 4}, {2, 4}, {5, 5}, {4, 5}};
    for (int g = 0; g < kNRP && st == CoefGenStatus::kOk; ++g) {
      const double *Am = W + (size_t)prod[g][0] * n_off * T;
      const cublasStatus_t cs = cublasDgemm(hb, CUBLAS_OP_N, CUBLAS_OP_N, (int)(2 * nz), n_off, T, &one,
                                            Fk(prod[g][1]), (int)(2 * nz), Am, T, &zero,
                                            Pm + (size_t)g * 2 * nz, (int)ncol);
      if (cs != CUBLAS_STATUS_SUCCESS) st = CoefGenStatus::kCuda;
    }
    receiver_assemble_kernel<<<grid1d((long long)n_off * nz), 256, 0, s>>>(Pm, n_off, nz,
                                                                           reinterpret_cast<zc *>(tab_dev));
    ck(cudaGetLastError());
    ck(cudaStreamSynchronize(s));
  }
  if (hb) cublasDestroy(hb);
  cudaFree(spec); cudaFree(F); cudaFree(W); cudaFree(edges); cudaFree(Pm); cudaFree(d_offs); cudaFree(d_doffs);
  return st;
}

}  // namespace ie
