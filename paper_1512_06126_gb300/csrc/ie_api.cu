// C ABI of the GB300 integral-equation solver: context, setup, the FFT matrix-vector
// product A = S + R1 B R2 (eq. (matrix_convolv)), GMRES and the mixed-precision
// iterative refinement.  See include/ie.h for the contract of every entry point.
#include "../../include/ie.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <limits>
#include <complex>
#include <cstring>
#include <new>
#include <vector>

#include "blas.cuh"
#include "coefgen.cuh"
#include "receivers.cuh"
#include "contract.cuh"
#include "fft.cuh"
#include "setup.cuh"

using cd = std::complex<double>;

#include <atomic>
namespace ie {
static std::atomic<long long> g_launches{0};
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace ie

namespace {

constexpr double kMu0 = 4e-7 * M_PI;

struct DiagSet {  // per-cell complex scales of one precision
  void *in_f = nullptr, *out_f = nullptr, *diag = nullptr, *in_t = nullptr, *out_t = nullptr;
};

struct Instance {
  double freq = 0.0;
  double2 *q64 = nullptr;
  float2 *q32 = nullptr;
  float4 *qdf = nullptr;           // double-float copy of q64 (residuals of the mixed solver)
  int *qexp = nullptr;             // per folded wavenumber: the scale exponent of its c64 block
  void *qh = nullptr;              // the c64 blocks scaled and split into FP16 pairs (Nz in {16, 32})
  double2 *rtab = nullptr;         // receiver kernels [Ny][Nx][Nz][10] (ie_set_receivers) or, for sites,
                                   // [group][2 Ny][2 Nx][Nz][10] (ie_set_receivers_xy)
  size_t rtab_cap = 0;             // its allocated elements
  double2 en{0.0, 0.0}, hn{0.0, 0.0};  // normal E^N and E^N'/(i w mu0) at the receiver depth
};

}  // namespace

struct ie_ctx {
  int nx = 0, ny = 0, nz = 0;
  double hx = 0, hy = 0, x0 = 0, y0 = 0;
  std::vector<double> ze, d;
  std::vector<cd> sig, sigma_a;
  std::vector<int> lay;
  ie::FftPlan px{}, py{};
  double fft_ms[2] = {0.0, 0.0};  // plan autotuner: ms of the chosen c128 pass (x rows, y columns)
  int max_rhs = 1;
  int cvar[5] = {-1, -1, -1, -1, -1};          // c64 contraction variant per right-hand sides per instance
  double tune_ms[5][ie::kContractVariants] = {};  // autotuner timings (ms per launch, 0: not timed)
  bool autotune = true;
  int restart = 30, max_iter = 2000, max_outer = 50;
  double inner_tol = 1e-3;
  std::vector<Instance> inst;
  DiagSet d64, d32;
  cudaStream_t stream = nullptr;
  void *t1 = nullptr, *spec = nullptr;        // FFT workspaces (sized for c128, max_rhs)
  float2 *x32 = nullptr, *y32 = nullptr;       // c64 right-hand side and correction of the inner solves
  // Krylov basis V [restart + 1][R][3N] and work vector w: sized for c128, used as c64
  // by the inner solves of the mixed solver; r: c128 residual; part / nrmpart: partial
  // sums of the Gram-Schmidt passes and norms; hdev: Hessenberg columns and solutions;
  // dx: c128 correction of the IE_MIXED_FP64K inner solves
  double2 *V = nullptr, *w = nullptr, *r = nullptr, *dx = nullptr, *part = nullptr, *hdev = nullptr;
  double *nrmpart = nullptr, *nrm = nullptr;
  int *gsflag = nullptr;                       // 48 ints: second-projection flags, reduction tickets, a counter
  ie::GivensState gst{};                       // device least-squares state of GMRES
  int *pin_active = nullptr;                   // pinned: active counts (slot 0: cycle start, 1..4: iterations),
                                               // slot 5: the contraction error word
  int *err = nullptr;                          // device: contraction error word of this context's launches
  bool gs_df = true;                           // IE_MIXED_FP64K inner Gram-Schmidt in double-float arithmetic
  float4 *Vs = nullptr;                        // split copy of the FP64 basis [restart + 1][R][3N] (gs_df)
  cudaEvent_t pin_ev[4] = {};
  // the Givens steps of a Krylov iteration run on a second stream, overlapping the next
  // product: gs_ev (Gram-Schmidt of the iteration done) orders them after their
  // column, giv_ev (Givens step done) orders the next Gram-Schmidt pass after them
  cudaStream_t side = nullptr;
  cudaEvent_t gs_ev = nullptr, giv_ev = nullptr;
  void *jfac = nullptr, *gdiv = nullptr;       // per cell: 2 s gamma; (dgamma/dln sigma_a) / gamma (0 off the anomaly)
  void *efac = nullptr;                        // per cell: 1 / a = 2 s / (sigma_a + conj sigma_b) (E = U / a)
  int n_rec = 0;                               // receivers (ie_set_receivers)
  int *rec_ix = nullptr, *rec_iy = nullptr;
  int *rec_grp = nullptr;                      // sites (ie_set_receivers_xy): table group of every receiver
  bool rec_sites = false;                      // the receivers are arbitrary sites
  double z_rec = 0.0;
  double *phi_r = nullptr;                     // per-receiver misfit terms
  std::vector<void *> allocs;
  long long dev_bytes = 0;
  // profiling: event pairs recorded around each contraction launch (level 1) and also
  // around the steps of every Krylov iteration (level 2)
  int prof = 0;
  struct ProfRec { cudaEvent_t a, b; int dtype; };
  std::vector<ProfRec> prof_rec;

  long long ncell() const { return (long long)nx * ny * nz; }
  long long nvec() const { return 3 * ncell(); }
};

namespace {

ie_status cuda_status(cudaError_t e) { return e == cudaSuccess ? IE_OK : (e == cudaErrorMemoryAllocation ? IE_ERR_OOM : IE_ERR_CUDA); }

template <typename P> ie_status dalloc(ie_ctx *c, P **p, size_t bytes) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? IE_ERR_OOM : IE_ERR_CUDA;
  }
  c->allocs.push_back(q);
  c->dev_bytes += (long long)bytes;
  *p = reinterpret_cast<P *>(q);
  return IE_OK;
}

#define IE_TRY(x)                      \
  do {                                 \
    ie_status _s = (x);                \
    if (_s != IE_OK) return _s;        \
  } while (0)
#define IE_CUDA(x) IE_TRY(cuda_status(x))

// ---------------------------------------------------------------------------
// Geometry and diagonals
// ---------------------------------------------------------------------------

int layer_of_cell(const std::vector<double> &d, double z1, double z2) {
  // layer m holds (d_m, d_{m+1}); layer 0 is the air above d_1
  int ra = 0, rb = 0;
  for (size_t k = 0; k < d.size(); ++k) {
    if (z1 >= d[k]) ra = (int)k + 1;
    if (z2 > d[k]) rb = (int)k + 1;
  }
  return ra == rb ? ra : -1;
}

template <typename T>
ie_status upload_cplx(ie_ctx *c, const std::vector<cd> &h, void **dst) {
  using V = ie::C<T>;
  std::vector<V> tmp(h.size());
  for (size_t i = 0; i < h.size(); ++i) tmp[i] = ie::mk<T>((T)h[i].real(), (T)h[i].imag());
  V *p = static_cast<V *>(*dst);
  if (!p) IE_TRY(dalloc(c, &p, tmp.size() * sizeof(V)));  // an existing buffer is overwritten in place
  IE_CUDA(cudaMemcpy(p, tmp.data(), tmp.size() * sizeof(V), cudaMemcpyHostToDevice));
  *dst = p;
  return IE_OK;
}

ie_status build_diagonals(ie_ctx *c) {
  const long long N = c->ncell();
  const double norm = 1.0 / (4.0 * c->nx * c->ny);
  std::vector<cd> in_f(N), out_f(N), diag(N), in_t(N), out_t(N), jfac(N), gdiv(N), efac(N);
  for (int z = 0; z < c->nz; ++z) {
    const cd sb = c->sig[c->lay[z]];
    const double s = std::sqrt(sb.real());
    const double V = c->hx * c->hy * (c->ze[z + 1] - c->ze[z]);
    for (long long q = 0; q < (long long)c->ny * c->nx; ++q) {
      const long long i = (long long)z * c->ny * c->nx + q;
      const cd sa = c->sigma_a[i];
      const cd g = (sa - sb) / (sa + std::conj(sb));
      in_f[i] = s * g;
      out_f[i] = -2.0 * s / V * norm;
      diag[i] = 1.0 - g;
      in_t[i] = -2.0 * s / V;
      out_t[i] = s * g * norm;
      jfac[i] = 2.0 * s * g;
      efac[i] = 2.0 * s / (sa + std::conj(sb));
      // dgamma/dln(sigma_a) = sigma_a 2 Re(sigma_b) / (sigma_a + conj sigma_b)^2, divided by gamma
      const cd den = sa + std::conj(sb);
      gdiv[i] = g == 0.0 ? cd(0.0) : sa * 2.0 * sb.real() / (den * den) / g;
    }
  }
  IE_TRY(upload_cplx<double>(c, in_f, &c->d64.in_f));
  IE_TRY(upload_cplx<double>(c, out_f, &c->d64.out_f));
  IE_TRY(upload_cplx<double>(c, diag, &c->d64.diag));
  IE_TRY(upload_cplx<double>(c, in_t, &c->d64.in_t));
  IE_TRY(upload_cplx<double>(c, out_t, &c->d64.out_t));
  IE_TRY(upload_cplx<float>(c, in_f, &c->d32.in_f));
  IE_TRY(upload_cplx<float>(c, out_f, &c->d32.out_f));
  IE_TRY(upload_cplx<float>(c, diag, &c->d32.diag));
  IE_TRY(upload_cplx<float>(c, in_t, &c->d32.in_t));
  IE_TRY(upload_cplx<float>(c, out_t, &c->d32.out_t));
  IE_TRY(upload_cplx<double>(c, jfac, &c->jfac));
  IE_TRY(upload_cplx<double>(c, gdiv, &c->gdiv));
  IE_TRY(upload_cplx<double>(c, efac, &c->efac));
  return IE_OK;
}

// E^N(z) and E^N'(z) / (i w mu0) of the 1-D profile (normalised H(0) = 1) at a depth z
// in layer m >= 1; same propagation as mt_cell_average.
void mt_point(const ie_ctx *c, double omega, double z, cd *E_out, cd *H_out) {
  const int L = (int)c->d.size();
  std::vector<cd> kap(L + 1), Eb(L + 1), Epb(L + 1);
  for (int m = 0; m <= L; ++m) kap[m] = std::sqrt(cd(0.0, -omega * kMu0) * c->sig[m]);
  cd E = 1.0, Ep = -kap[L];
  for (int m = L - 1; m >= 1; --m) {
    Eb[m] = E;
    Epb[m] = Ep;
    const double l = c->d[m] - c->d[m - 1];
    const cd ch = std::cosh(kap[m] * l), sh = std::sinh(kap[m] * l);
    const cd Et = E * ch - Ep * sh / kap[m];
    const cd Ept = -E * kap[m] * sh + Ep * ch;
    E = Et;
    Ep = Ept;
  }
  const cd a = cd(0.0, omega * kMu0) / Ep;
  int m = 1;
  for (int k = 0; k < L; ++k)
    if (z >= c->d[k]) m = k + 1;
  cd e, ep;
  const cd k = kap[m];
  if (m == L) {
    e = a * std::exp(-k * (z - c->d[L - 1]));
    ep = -k * e;
  } else {
    const double zb = c->d[m];
    e = a * (Eb[m] * std::cosh(k * (z - zb)) + Epb[m] * std::sinh(k * (z - zb)) / k);
    ep = a * (Eb[m] * k * std::sinh(k * (z - zb)) + Epb[m] * std::cosh(k * (z - zb)));
  }
  *E_out = e;
  *H_out = ep / cd(0.0, omega * kMu0);
}

// IE_ERR_GEOMETRY if an anomalous cell touches or rises above the receiver plane
ie_status check_receiver_geometry(const ie_ctx *c) {
  if (c->n_rec == 0) return IE_OK;
  const long long plane = (long long)c->nx * c->ny;
  for (int z = 0; z < c->nz; ++z) {
    if (c->ze[z] > c->z_rec) continue;
    const cd sb = c->sig[c->lay[z]];
    for (long long q = 0; q < plane; ++q)
      if (c->sigma_a[(long long)z * plane + q] != sb) return IE_ERR_GEOMETRY;
  }
  return IE_OK;
}

// Coefficient DFT: real-space compressed tensor (c128, on the host or already on the
// device) -> folded spectral c128 + c64.  If both pointers are null the tensor is
// generated on the device (Appendices A-C).
ie_status build_spectral(ie_ctx *c, Instance &in, const double *q_host) {
  const int Nx = c->nx, Ny = c->ny, Nz = c->nz;
  const long long NE = 6LL * Nz * Nz;
  const long long nq = (long long)Nx * Ny * NE;
  const long long BS = 2LL * Nz * (2 * Nz + 1);
  const long long nf = (long long)(Nx + 1) * (Ny + 1);
  IE_TRY(dalloc(c, &in.q64, nf * BS * sizeof(double2)));
  IE_TRY(dalloc(c, &in.q32, nf * BS * sizeof(float2)));
  double2 *dq = nullptr, *buf = nullptr;
  IE_CUDA(cudaMalloc(&dq, nq * sizeof(double2)));
  cudaError_t e = cudaSuccess;
  if (q_host) {
    e = cudaMemcpyAsync(dq, q_host, nq * sizeof(double2), cudaMemcpyHostToDevice, c->stream);
  } else {
    std::vector<double> sg(2 * c->sig.size());
    for (size_t k = 0; k < c->sig.size(); ++k) { sg[2 * k] = c->sig[k].real(); sg[2 * k + 1] = c->sig[k].imag(); }
    ie::CoefGenInput gi{c->nx, c->ny, c->nz, c->hx, c->hy, c->ze.data(), c->lay.data(), (int)c->d.size(),
                        c->d.data(), sg.data(), in.freq};
    const ie::CoefGenStatus gs = ie::generate_coefficients(gi, dq, c->stream);
    if (gs != ie::CoefGenStatus::kOk) {
      cudaFree(dq);
      return gs == ie::CoefGenStatus::kUnsupported ? IE_ERR_ARG : IE_ERR_CUDA;
    }
  }
  const long long plane = 4LL * Nx * Ny;
  long long E = std::max<long long>(1, std::min<long long>(NE, (1LL << 30) / (plane * (long long)sizeof(double2))));
  if (e == cudaSuccess) e = cudaMalloc(&buf, plane * E * sizeof(double2));
  if (e != cudaSuccess) { cudaFree(dq); return cuda_status(e); }
  for (long long e0 = 0; e == cudaSuccess && e0 < NE; e0 += E) {
    const long long Ec = std::min(E, NE - e0);
    ie::launch_embed(dq, buf, Nx, Ny, Nz, e0, Ec, c->stream);
    ie::launch_fft_axis<double, false>(buf, buf, 2 * Ny, 2 * Nx, 2 * Nx, Ec, c->px, 1.0, c->stream);
    ie::launch_fft_axis<double, false>(buf, buf, 1, 2 * Ny, 2 * Ny, 2LL * Nx * Ec, c->py, 1.0, c->stream);
    ie::launch_pack(buf, in.q64, in.q32, Nx, Ny, Nz, e0, Ec, c->stream);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(dq);
  cudaFree(buf);
  IE_TRY(cuda_status(e));
  IE_TRY(dalloc(c, &in.qdf, nf * BS * sizeof(float4)));
  ie::launch_split_df(in.q64, in.qdf, nf * BS, c->stream);
  IE_TRY(dalloc(c, &in.qexp, nf * sizeof(int)));
  ie::launch_block_exponents(in.q32, in.qexp, nf, Nz, c->stream);
  if (ie::contract_variant_available(ie::kContractTc16, Nz, 1, true)) {
    IE_TRY(dalloc(c, &in.qh, nf * BS * sizeof(uint2)));
    ie::launch_split_f16(in.q32, in.qexp, in.qh, nf, Nz, c->stream);
  }
  return cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// The matrix-vector product
// ---------------------------------------------------------------------------

template <typename T> const DiagSet &diags(const ie_ctx *c);
template <> const DiagSet &diags<double>(const ie_ctx *c) { return c->d64; }
template <> const DiagSet &diags<float>(const ie_ctx *c) { return c->d32; }
template <typename T> const ie::C<T> *qf(const Instance &in);
template <> const double2 *qf<double>(const Instance &in) { return in.q64; }
template <> const float2 *qf<float>(const Instance &in) { return in.q32; }

// The right-hand sides of one product: n blocks of rpi right-hand sides, block k with
// the coefficients of instance inst[k] (layout [n][rpi][3][Nz][Ny][Nx]).  The
// diagonal scalings do not depend on the frequency, so all blocks share the row
// passes; each block gets its own contraction on its slice of the spectrum.
struct Group {
  std::vector<int> inst;
  int rpi = 1;
  int R() const { return (int)inst.size() * rpi; }
};

template <typename T>
ie_status contract_group(ie_ctx *c, const Group &g, ie::C<T> *spec, cudaStream_t s, bool df = false) {
  const int CZ = g.R() * 3 * c->nz;
  cudaEvent_t ea = nullptr, eb = nullptr;
  if (c->prof) {
    cudaEventCreate(&ea);
    cudaEventCreate(&eb);
    cudaEventRecord(ea, s);
  }
  const int variant = sizeof(T) == 4 ? c->cvar[g.rpi] : ie::kContractPanel;
  for (size_t k = 0; k < g.inst.size(); ++k) {
    ie::C<T> *sk = spec + k * (size_t)g.rpi * 3 * c->nz;
    if constexpr (sizeof(T) == 8) {
      if (df && ie::launch_contract_df(sk, c->inst[g.inst[k]].qdf, c->nx, c->ny, c->nz, g.rpi, CZ, s) == 0) continue;
    }
    if (ie::launch_contract<T>(sk, qf<T>(c->inst[g.inst[k]]), c->nx, c->ny, c->nz, g.rpi, CZ, variant, c->err, s,
                               c->inst[g.inst[k]].qexp, c->inst[g.inst[k]].qh) != 0)
      return IE_ERR_CUDA;
  }
  if (c->prof) {
    cudaEventRecord(eb, s);
    c->prof_rec.push_back({ea, eb, sizeof(T) == 8 ? IE_C128 : IE_C64});
  }
  return IE_OK;
}

// df (c128 only): the contraction in double-float arithmetic (launch_contract_df)
template <typename T>
ie_status apply(ie_ctx *c, const Group &g, const ie::C<T> *x, ie::C<T> *y, int transpose, cudaStream_t s,
                bool df = false) {
  using V = ie::C<T>;
  const int Nx = c->nx, Ny = c->ny, Nz = c->nz;
  const int CZ = g.R() * 3 * Nz;
  const DiagSet &D = diags<T>(c);
  const V *in_s = (const V *)(transpose ? D.in_t : D.in_f);
  const V *out_s = (const V *)(transpose ? D.out_t : D.out_f);
  const V *dg = (const V *)D.diag;
  V *t1 = (V *)c->t1;
  V *spec = (V *)c->spec;
  ie::launch_fft_rows_fwd<T>(x, in_s, t1, CZ, Nz, Ny, Nx, c->px, s);
  ie::launch_fft_axis<T, false>(t1, spec, 1, Ny, 2 * Ny, 2LL * Nx * CZ, c->py, (T)1, s);
  IE_TRY(contract_group<T>(c, g, spec, s, df));
  ie::launch_fft_axis<T, true>(spec, t1, 1, 2 * Ny, Ny, 2LL * Nx * CZ, c->py, (T)1, s);
  ie::launch_fft_rows_inv<T>(t1, x, dg, out_s, y, CZ, Nz, Ny, Nx, c->px, s);
  return cuda_status(cudaGetLastError());
}

// c64 product on FP64 vectors (the inner solves of IE_MIXED_FP64K): the c64 operator
// applied in FP32 arithmetic throughout (the FP32 scales), the row passes reading the
// FP64 vector (rounded to FP32 on load) and writing the FP64 result.
ie_status apply_mixed(ie_ctx *c, const Group &g, const double2 *x, double2 *y, int transpose, cudaStream_t s) {
  const int Nx = c->nx, Ny = c->ny, Nz = c->nz;
  const int CZ = g.R() * 3 * Nz;
  const DiagSet &D = c->d32;
  const float2 *in_s = (const float2 *)(transpose ? D.in_t : D.in_f);
  const float2 *out_s = (const float2 *)(transpose ? D.out_t : D.out_f);
  float2 *t1 = (float2 *)c->t1;
  float2 *spec = (float2 *)c->spec;
  ie::launch_fft_rows_fwd<float, double>(x, in_s, t1, CZ, Nz, Ny, Nx, c->px, s);
  ie::launch_fft_axis<float, false>(t1, spec, 1, Ny, 2 * Ny, 2LL * Nx * CZ, c->py, 1.0f, s);
  IE_TRY(contract_group<float>(c, g, spec, s));
  ie::launch_fft_axis<float, true>(spec, t1, 1, 2 * Ny, Ny, 2LL * Nx * CZ, c->py, 1.0f, s);
  ie::launch_fft_rows_inv<float, double>(t1, x, (const float2 *)D.diag, out_s, y, CZ, Nz, Ny, Nx, c->px, s);
  return cuda_status(cudaGetLastError());
}

// The operator the Krylov solver applies: the c128 product on c128 vectors (T =
// double), the c64 product on c64 vectors (T = float), or the c64 product on c128
// vectors (T = double with single).
template <typename T>
struct Op {
  ie_ctx *c;
  const Group *g;
  int transpose;
  bool df = false;      // c128: double-float contraction
  bool single = false;  // T = double: the c64 product (apply_mixed)
  ie_status operator()(const ie::C<T> *x, ie::C<T> *y, int R) const {
    if (R != g->R()) return IE_ERR_ARG;
    if constexpr (sizeof(T) == 8) {
      if (single) return apply_mixed(c, *g, x, y, transpose, c->stream);
    }
    return apply<T>(c, *g, x, y, transpose, c->stream, df);
  }
};

// A pair of events around one step of a Krylov iteration (profiling level 2).
struct ProfSpan {
  ie_ctx *c;
  int kind;
  cudaEvent_t a = nullptr;
  ProfSpan(ie_ctx *c_, int kind_) : c(c_), kind(kind_) {
    if (c->prof >= 2 && cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, c->stream);
  }
  void end() {
    cudaEvent_t b = nullptr;
    if (a && cudaEventCreate(&b) == cudaSuccess) {
      cudaEventRecord(b, c->stream);
      c->prof_rec.push_back({a, b, kind});
      a = nullptr;
    }
  }
};

// ---------------------------------------------------------------------------
// GMRES(m), classical Gram-Schmidt with selective reorthogonalisation, all right-hand
// sides in lockstep.
// Solves op(x) = b until ||b - op x|| <= tol ||b|| for every right-hand side (the
// Givens recurrence ends a cycle; a true residual at the next restart confirms it).
// ---------------------------------------------------------------------------

constexpr int kGivensLag = 2;   // iterations between issuing a Givens step and reading its count
constexpr int kPinSlots = 4;
constexpr int kPinErr = 1 + kPinSlots;  // pinned slot of the contraction error word

// Queue a copy of the contraction error word into its pinned slot (read after the
// caller's next synchronisation).
ie_status queue_err_read(ie_ctx *c, cudaStream_t s) {
  IE_CUDA(cudaMemcpyAsync(c->pin_active + kPinErr, c->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  return IE_OK;
}
// After that synchronisation: IE_ERR_TIMEOUT (and the word cleared) if a contraction
// kernel recorded a wait that ran out, whose product is then incomplete.
ie_status take_err(ie_ctx *c, cudaStream_t s) {
  if (c->pin_active[kPinErr] == 0) return IE_OK;
  c->pin_active[kPinErr] = 0;
  IE_CUDA(cudaMemsetAsync(c->err, 0, sizeof(int), s));
  IE_CUDA(cudaStreamSynchronize(s));
  return IE_ERR_TIMEOUT;
}

struct GmresResult {
  int iters = 0;
  int cycles = 0;
  bool converged = false;
  bool breakdown = false;
};

// Swap the blocks p and q (elem elements each) of a, through the scratch tmp.
template <typename V>
ie_status swap_blocks(V *a, int p, int q, long long elem, V *tmp, cudaStream_t s) {
  const size_t bytes = (size_t)elem * sizeof(V);
  IE_CUDA(cudaMemcpyAsync(tmp, a + p * elem, bytes, cudaMemcpyDeviceToDevice, s));
  IE_CUDA(cudaMemcpyAsync(a + p * elem, a + q * elem, bytes, cudaMemcpyDeviceToDevice, s));
  IE_CUDA(cudaMemcpyAsync(a + q * elem, tmp, bytes, cudaMemcpyDeviceToDevice, s));
  return IE_OK;
}

// Restarted GMRES on the group g0 (its instances' blocks of rpi right-hand sides).
// With compact (several instances; b then is scratch the solver may reorder), an
// instance whose right-hand sides have all converged leaves the lockstep at the next
// restart: its blocks of b and x swap places with an active instance's, and the
// remaining cycles run on the smaller group.  x is back in the original order on
// return.  T = double: c128 vectors and operator; T = float: c64 vectors and
// operator, the basis in the same storage (half of it used).
// x_zero: x is zero on entry (the first residual is b).  For c64 vectors the residual
// at a restart comes from the Krylov relation (b - A x = V_{k+1} Q^H g_{k+1} e_{k+1},
// one combination of the basis instead of a product); c128 solves recompute it.
template <typename T>
ie_status gmres(ie_ctx *c, const Group &g0, int transpose, ie::C<T> *b, ie::C<T> *x, double tol, int max_iter,
                GmresResult *res, bool compact, bool x_zero, bool single = false) {
  using Vt = ie::C<T>;
  Vt *const Vb = (Vt *)c->V;
  Vt *const w = (Vt *)c->w;
  const long long n = c->nvec();
  const int m = c->restart;
  const int ldh = m + 1;
  const int rpi = g0.rpi;
  const long long blk = n * rpi;
  cudaStream_t s = c->stream;
  Group g = g0;
  const Op<T> op{c, &g, transpose, false, single};
  int R = g.R();
  long long nR = n * R;
  const int G = (int)g0.inst.size();
  std::vector<int> inst_at(G);  // original block index of the block now at each position
  for (int k = 0; k < G; ++k) inst_at[k] = k;
  compact = compact && G > 1;
  double2 *h1 = c->hdev, *h2 = c->hdev + (size_t)R * ldh, *yd = c->hdev + 2 * (size_t)R * ldh;
  const ie::GivensState &st = c->gst;
  std::vector<double> bnorm(R), thr(R);
  ie::gmres_norm<T>(b, c->nrmpart, c->nrm, R, n, s);
  IE_CUDA(cudaMemcpyAsync(bnorm.data(), c->nrm, R * sizeof(double), cudaMemcpyDeviceToHost, s));
  IE_CUDA(cudaStreamSynchronize(s));
  auto upload_thr = [&]() -> ie_status {
    for (int r = 0; r < R; ++r) thr[r] = tol * bnorm[r];
    IE_CUDA(cudaMemcpyAsync(st.thr, thr.data(), R * sizeof(double), cudaMemcpyHostToDevice, s));
    return IE_OK;
  };
  IE_TRY(upload_thr());
  std::vector<int> kr(R), brk(R), act(R);
  res->converged = false;
  res->breakdown = false;
  int it = 0;  // iterations issued (including the few issued after the last right-hand side stopped)
  bool pending = false;  // a finished cycle's column counts are being copied
  int R_prev = R;
  bool have_res = false;  // w holds b - A x from the Krylov relation
  while (true) {
    h1 = c->hdev;
    h2 = c->hdev + (size_t)R * ldh;
    yd = c->hdev + 2 * (size_t)R * ldh;
    if (x_zero) {
      IE_CUDA(cudaMemcpyAsync(w, b, nR * sizeof(Vt), cudaMemcpyDeviceToDevice, s));
      x_zero = false;
    } else if (!have_res) {
      IE_TRY(op(x, w, R));
      ie::vec_sub<T>(b, w, w, nR, s);
    }
    have_res = false;
    ie::gmres_norm<T>(w, c->nrmpart, c->nrm, R, n, s);
    ie::gmres_scale<T>(w, Vb, c->nrm, R, n, s);
    if constexpr (sizeof(T) == 8) {
      if (single && c->gs_df) ie::gmres_split((const double2 *)Vb, c->Vs, nR, s);
    }
    ie::givens_init(st, c->nrm, R, ldh, s);
    IE_CUDA(cudaMemcpyAsync(c->pin_active, st.n_active, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (compact) IE_CUDA(cudaMemcpyAsync(act.data(), st.active, R * sizeof(int), cudaMemcpyDeviceToHost, s));
    IE_TRY(queue_err_read(c, s));
    IE_CUDA(cudaStreamSynchronize(s));
    IE_TRY(take_err(c, s));
    if (pending) {
      int kmx = 0;
      for (int r = 0; r < R_prev; ++r) {
        kmx = std::max(kmx, kr[r]);
        if (brk[r]) res->breakdown = true;
      }
      res->iters += kmx;
      pending = false;
    }
    if (c->pin_active[0] == 0) { res->converged = true; break; }
    if (it >= max_iter) break;
    if (compact) {
      // instances with no right-hand side left above its threshold leave the group
      const int Gc = (int)g.inst.size();
      std::vector<char> ia(Gc, 0);
      int n_act = 0;
      for (int p = 0; p < Gc; ++p) {
        for (int j = 0; j < rpi; ++j) ia[p] |= act[p * rpi + j] ? 1 : 0;
        n_act += ia[p];
      }
      if (n_act < Gc) {
        int p = 0, q = Gc - 1;
        while (p < q) {
          if (ia[p]) { ++p; continue; }
          if (!ia[q]) { --q; continue; }
          IE_TRY(swap_blocks(b, p, q, blk, w, s));
          IE_TRY(swap_blocks(x, p, q, blk, w, s));
          std::swap(inst_at[p], inst_at[q]);
          std::swap(g.inst[p], g.inst[q]);
          for (int j = 0; j < rpi; ++j) std::swap(bnorm[p * rpi + j], bnorm[q * rpi + j]);
          std::swap(ia[p], ia[q]);
          ++p;
          --q;
        }
        g.inst.resize(n_act);
        R = n_act * rpi;
        nR = n * R;
        IE_TRY(upload_thr());
        have_res = false;
        continue;  // residual of the smaller group
      }
    }
    res->cycles++;
    // the cycle: products, Gram-Schmidt and Givens steps stay on the device; the host
    // learns the number of right-hand sides still iterating from a pinned copy made
    // kLag iterations earlier, so it never waits for the iteration it just issued.  The
    // Givens step of iteration k runs on the side stream, beside the product of
    // iteration k + 1 (which does not depend on it); the Gram-Schmidt pass of k + 1, which
    // rewrites the column and norm the step reads, waits for it.  With per-step
    // profiling everything stays on the main stream.
    const bool overlap = c->prof < 2;
    bool giv_pending = false;
    int kmax = 0;
    for (int k = 0; k < m && it < max_iter; ++k) {
      if (k >= kGivensLag) {
        const int slot = (k - kGivensLag) % kPinSlots;
        IE_CUDA(cudaEventSynchronize(c->pin_ev[slot]));
        if (c->pin_active[1 + slot] == 0) break;
      }
      ProfSpan sp_op(c, sizeof(T) == 4 ? IE_PROF_PRODUCT_C64 : IE_PROF_PRODUCT_C128);
      IE_TRY(op(Vb + (long long)k * nR, w, R));
      sp_op.end();
      if (giv_pending) IE_CUDA(cudaStreamWaitEvent(s, c->giv_ev, 0));
      ProfSpan sp_gs(c, sizeof(T) == 4 ? IE_PROF_GS_C64 : IE_PROF_GS_C128);
      if (ie::gmres_orthogonalize<T>(Vb, w, Vb + (long long)(k + 1) * nR, h1, h2, c->part, c->nrmpart, c->nrm,
                                  c->gsflag, k + 1, R, n, ldh, s, single && c->gs_df, c->Vs,
                                  c->Vs + (long long)(k + 1) * nR) != 0)
        return IE_ERR_ARG;
      sp_gs.end();
      cudaStream_t sg = s;
      if (overlap) {
        IE_CUDA(cudaEventRecord(c->gs_ev, s));
        IE_CUDA(cudaStreamWaitEvent(c->side, c->gs_ev, 0));
        sg = c->side;
      }
      ProfSpan sp_gv(c, IE_PROF_GIVENS);
      ie::givens_step(st, h1, h2, c->nrm, k, R, m, ldh, sizeof(T) == 4, sg);
      sp_gv.end();
      const int slot = k % kPinSlots;
      IE_CUDA(cudaMemcpyAsync(c->pin_active + 1 + slot, st.n_active, sizeof(int), cudaMemcpyDeviceToHost, sg));
      IE_CUDA(cudaEventRecord(c->pin_ev[slot], sg));
      if (overlap) {
        IE_CUDA(cudaEventRecord(c->giv_ev, sg));
        giv_pending = true;
      }
      ++it;
      kmax = k + 1;
    }
    if (giv_pending) IE_CUDA(cudaStreamWaitEvent(s, c->giv_ev, 0));  // the cycle's last Givens step
    // x += V y with y from the rotated least-squares problem (zero beyond each kr); the
    // FP64 vectors of the IE_MIXED_FP64K inner solves in double-float from the split basis
    const bool dfk = sizeof(T) == 8 && single && c->gs_df;
    ie::givens_solve(st, yd, R, m, ldh, s);
    if (dfk) ie::gmres_maxpy_df(c->Vs, yd, (double2 *)x, kmax, R, n, ldh, s);
    else ie::gmres_maxpy<T>(Vb, yd, x, kmax, R, n, ldh, 1.0, s);
    if (sizeof(T) == 4 || dfk) {
      // the next cycle's residual from the basis (the inner solves of both mixed modes):
      // w = V_0..V_kmax z
      ie::givens_residual(st, h1, R, m, ldh, s);
      IE_CUDA(cudaMemsetAsync(w, 0, nR * sizeof(Vt), s));
      if (dfk) ie::gmres_maxpy_df(c->Vs, h1, (double2 *)w, kmax + 1, R, n, ldh, s);
      else ie::gmres_maxpy<T>(Vb, h1, w, kmax + 1, R, n, ldh, 1.0, s);
      have_res = true;
    }
    IE_CUDA(cudaMemcpyAsync(kr.data(), st.kr, R * sizeof(int), cudaMemcpyDeviceToHost, s));
    IE_CUDA(cudaMemcpyAsync(brk.data(), st.brk, R * sizeof(int), cudaMemcpyDeviceToHost, s));
    pending = true;
    R_prev = R;
    IE_CUDA(cudaGetLastError());
  }
  if (pending) {  // only reached when the loop left before the next synchronisation
    IE_TRY(queue_err_read(c, s));
    IE_CUDA(cudaStreamSynchronize(s));
    IE_TRY(take_err(c, s));
    int kmx = 0;
    for (int r = 0; r < R_prev; ++r) {
      kmx = std::max(kmx, kr[r]);
      if (brk[r]) res->breakdown = true;
    }
    res->iters += kmx;
  }
  // blocks back to their original positions
  for (int p = 0; p < G; ++p)
    while (inst_at[p] != p) {
      const int q = inst_at[p];
      IE_TRY(swap_blocks(x, p, q, blk, w, s));
      IE_TRY(swap_blocks(b, p, q, blk, w, s));
      std::swap(inst_at[p], inst_at[q]);
    }
  return IE_OK;
}

// max over right-hand sides of ||b - A128 u|| / ||b||; leaves the residual in c->r.  df:
// the product's contraction in double-float arithmetic (the residuals of the mixed
// solver), else FP64.
ie_status true_residual(ie_ctx *c, const Group &g, int transpose, const double2 *b, const double2 *u,
                        std::vector<double> &rel, bool df = false) {
  const long long n = c->nvec();
  const int R = g.R();
  Op<double> op{c, &g, transpose, df};
  IE_TRY(op(u, c->r, R));
  ie::vec_sub<double>(b, c->r, c->r, n * R, c->stream);
  std::vector<double> rn(R), bn(R);
  ie::gmres_norm<double>(c->r, c->nrmpart, c->nrm, R, n, c->stream);
  IE_CUDA(cudaMemcpyAsync(rn.data(), c->nrm, R * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  ie::gmres_norm<double>(b, c->nrmpart, c->nrm + R, R, n, c->stream);
  IE_CUDA(cudaMemcpyAsync(bn.data(), c->nrm + R, R * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  IE_TRY(queue_err_read(c, c->stream));
  IE_CUDA(cudaStreamSynchronize(c->stream));
  IE_TRY(take_err(c, c->stream));
  rel.resize(R);
  for (int r = 0; r < R; ++r) rel[r] = bn[r] > 0 ? rn[r] / bn[r] : rn[r];
  return IE_OK;
}

ie_status solve_impl(ie_ctx *c, const Group &g, const double2 *b, double2 *u, double tol, int precision,
                     int use_x0, int transpose, ie_solve_info *info) {
  const int R = g.R();
  if (!c || !b || !u || g.inst.empty() || g.rpi < 1 || g.rpi > 4 || R > c->max_rhs || !(tol > 0)) return IE_ERR_ARG;
  for (int k : g.inst)
    if (k < 0 || k >= (int)c->inst.size()) return IE_ERR_ARG;
  if (precision != IE_FP64 && precision != IE_MIXED && precision != IE_MIXED_FP64K) return IE_ERR_ARG;
  const bool k64 = precision == IE_MIXED_FP64K;  // inner solves with FP64 Krylov vectors
  const long long n = c->nvec();
  const auto t0 = std::chrono::steady_clock::now();
  if (!use_x0) IE_CUDA(cudaMemsetAsync(u, 0, n * R * sizeof(double2), c->stream));
  IE_CUDA(cudaMemsetAsync(c->gsflag + 32, 0, sizeof(int), c->stream));
  ie_solve_info inf{};
  bool conv = false, brk = false;
  std::vector<double> rel;
  if (precision == IE_FP64) {
    GmresResult gr;
    // several instances: GMRES reorders the right-hand sides, so it works on a copy of b
    const bool comp = g.inst.size() > 1;
    double2 *bw = const_cast<double2 *>(b);
    if (comp) {
      IE_CUDA(cudaMemcpyAsync(c->r, b, n * R * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
      bw = c->r;
    }
    IE_TRY(gmres<double>(c, g, transpose, bw, u, tol, c->max_iter, &gr, comp, !use_x0));
    inf.inner_iters = gr.iters;
    inf.outer_iters = gr.cycles;
    conv = gr.converged;
    brk = gr.breakdown;
  } else {  // IE_MIXED, IE_MIXED_FP64K: iterative refinement
    int inner_total = 0;
    const long long blk = n * g.rpi;  // elements of one instance's block
    for (int outer = 0; outer <= c->max_outer; ++outer) {
      if (outer == 0 && !use_x0) {
        // u = 0: the residual is b itself (no c128 product needed)
        std::vector<double> bn(R);
        ie::gmres_norm<double>(b, c->nrmpart, c->nrm, R, n, c->stream);
        IE_CUDA(cudaMemcpyAsync(bn.data(), c->nrm, R * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        IE_CUDA(cudaStreamSynchronize(c->stream));
        rel.assign(R, 0.0);
        for (int r = 0; r < R; ++r) rel[r] = !std::isfinite(bn[r]) ? bn[r] : (bn[r] > 0 ? 1.0 : 0.0);
      } else {
        IE_TRY(true_residual(c, g, transpose, b, u, rel, !k64));
      }
      inf.outer_iters = outer + 1;
      // instances with a right-hand side above the tolerance stay in the inner solve;
      // the others are done and drop out of the group
      Group act;
      act.rpi = g.rpi;
      std::vector<int> pos;
      double worst = 0;
      bool finite = true;
      for (size_t k = 0; k < g.inst.size(); ++k) {
        double wk = 0;
        for (int p = 0; p < g.rpi; ++p) {
          wk = std::max(wk, rel[k * g.rpi + p]);
          finite = finite && std::isfinite(rel[k * g.rpi + p]);
        }
        worst = std::max(worst, wk);
        if (wk > tol) { act.inst.push_back(g.inst[k]); pos.push_back((int)k); }
      }
      if (!finite) { brk = true; break; }  // a non-finite residual ends the refinement, unconverged
      if (act.inst.empty()) { conv = true; break; }
      if (outer == c->max_outer || inner_total >= c->max_iter) break;
      const double2 *rsrc = (outer == 0 && !use_x0) ? b : c->r;
      const int Ra = act.R();
      const double itol = std::max(c->inner_tol, 0.5 * tol / std::max(worst, 1e-300));
      if (k64) {
        // the residual blocks of the active instances packed in order into r (a block
        // only moves to a lower position, so source and target never overlap); inner
        // GMRES with FP64 Krylov vectors on the c64 operator
        for (size_t a = 0; a < pos.size(); ++a)
          if (rsrc != c->r || (int)a != pos[a])
            IE_CUDA(cudaMemcpyAsync(c->r + (long long)a * blk, rsrc + (long long)pos[a] * blk,
                                    blk * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
        IE_CUDA(cudaMemsetAsync(c->dx, 0, n * Ra * sizeof(double2), c->stream));
        GmresResult gr;
        IE_TRY(gmres<double>(c, act, transpose, c->r, c->dx, std::min(itol, 0.5), c->max_iter - inner_total, &gr,
                             act.inst.size() > 1, true, true));
        inner_total += gr.iters;
        brk = brk || gr.breakdown;
        for (size_t a = 0; a < pos.size(); ++a)
          ie::vec_add<double>(c->dx + (long long)a * blk, u + (long long)pos[a] * blk, blk, c->stream);
        continue;
      }
      // the residual blocks of the active instances, rounded to c64, packed in order
      for (size_t a = 0; a < pos.size(); ++a)
        ie::vec_round(rsrc + (long long)pos[a] * blk, c->x32 + (long long)a * blk, blk, c->stream);
      // inner: A64 d = r in c64 (relative tolerance inner_tol, bounded below so as not
      // to over-solve)
      IE_CUDA(cudaMemsetAsync(c->y32, 0, n * Ra * sizeof(float2), c->stream));
      GmresResult gr;
      IE_TRY(gmres<float>(c, act, transpose, c->x32, c->y32, std::min(itol, 0.5), c->max_iter - inner_total, &gr,
                          act.inst.size() > 1, true));
      inner_total += gr.iters;
      brk = brk || gr.breakdown;
      for (size_t a = 0; a < pos.size(); ++a)
        ie::vec_add<float>(c->y32 + (long long)a * blk, u + (long long)pos[a] * blk, blk, c->stream);
    }
    inf.inner_iters = inner_total;
  }
  // the refinement loop ends on a true residual of the final iterate when it converged;
  // otherwise (and after a plain FP64 solve) measure it here
  if (!(precision != IE_FP64 && conv)) IE_TRY(true_residual(c, g, transpose, b, u, rel, precision == IE_MIXED));
  double worst = 0;
  for (double v : rel) worst = std::isfinite(v) ? std::max(worst, v) : std::numeric_limits<double>::infinity();
  inf.final_rel_res = worst;
  IE_CUDA(cudaMemcpyAsync(&inf.reorth, c->gsflag + 32, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  IE_TRY(queue_err_read(c, c->stream));
  IE_CUDA(cudaStreamSynchronize(c->stream));
  IE_TRY(take_err(c, c->stream));
  inf.t_solve = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  if (worst <= tol) return IE_OK;
  return brk ? IE_BREAKDOWN : IE_NOT_CONVERGED;
}

// ---------------------------------------------------------------------------
// Magnetotelluric normal field (1-D plane wave), integrated over the cells.
// E'' = kappa^2 E in each layer, kappa = sqrt(-i w mu0 sigma); E decays in the
// basement; E and E' continuous; E'(0) = i w mu0 (H(0) = 1).  Propagated upwards
// from the basement with the layer transfer (cosh, sinh) relations.
// ---------------------------------------------------------------------------

std::vector<cd> mt_cell_average(const ie_ctx *c, double omega) {
  const int L = (int)c->d.size();
  std::vector<cd> kap(L + 1), Eb(L + 1), Epb(L + 1);
  for (int m = 0; m <= L; ++m) kap[m] = std::sqrt(cd(0.0, -omega * kMu0) * c->sig[m]);
  cd E = 1.0, Ep = -kap[L];
  for (int m = L - 1; m >= 1; --m) {
    Eb[m] = E;
    Epb[m] = Ep;
    const double l = c->d[m] - c->d[m - 1];
    const cd ch = std::cosh(kap[m] * l), sh = std::sinh(kap[m] * l);
    const cd Et = E * ch - Ep * sh / kap[m];
    const cd Ept = -E * kap[m] * sh + Ep * ch;
    E = Et;
    Ep = Ept;
  }
  const cd a = cd(0.0, omega * kMu0) / Ep;  // E'(0) = i w mu0
  const cd EL = a;                          // E at the top of the basement before scaling was 1
  std::vector<cd> out(c->nz);
  for (int z = 0; z < c->nz; ++z) {
    const int m = c->lay[z];
    const double z1 = c->ze[z], z2 = c->ze[z + 1];
    const cd k = kap[m];
    cd integral;
    if (m == L) {
      const double dL = c->d[L - 1];
      integral = EL * (std::exp(-k * (z1 - dL)) - std::exp(-k * (z2 - dL))) / k;
    } else {
      const double zb = c->d[m];
      auto F = [&](double zz) {
        return a * (Eb[m] * std::sinh(k * (zz - zb)) / k + Epb[m] * std::cosh(k * (zz - zb)) / (k * k));
      };
      integral = F(z2) - F(z1);
    }
    out[z] = integral / (z2 - z1);
  }
  return out;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

const char *ie_status_str(ie_status s) {
  switch (s) {
    case IE_OK: return "ok";
    case IE_NOT_CONVERGED: return "not converged";
    case IE_BREAKDOWN: return "Krylov breakdown";
    case IE_ERR_ARG: return "invalid argument";
    case IE_ERR_GEOMETRY: return "invalid geometry";
    case IE_ERR_COEFF: return "invalid coefficient tensor";
    case IE_ERR_OOM: return "out of device memory";
    case IE_ERR_CUDA: return "CUDA error";
    case IE_ERR_SCRATCH: return "problem larger than the fixed work space of ie_matvec_noalloc";
    case IE_ERR_TIMEOUT: return "a wait inside a contraction kernel ran out; the product is incomplete";
  }
  return "unknown status";
}

static void prof_clear(ie_ctx *c);
void ie_destroy(ie_ctx *c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  prof_clear(c);
  for (void *p : c->allocs) cudaFree(p);
  if (c->pin_active) cudaFreeHost(c->pin_active);
  if (c->side) cudaStreamSynchronize(c->side);
  for (auto &e : c->pin_ev)
    if (e) cudaEventDestroy(e);
  if (c->gs_ev) cudaEventDestroy(c->gs_ev);
  if (c->giv_ev) cudaEventDestroy(c->giv_ev);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

void *ie_ctx_stream(ie_ctx *c) { return c ? (void *)c->stream : nullptr; }

long long ie_kernel_launches(void) { return ie::launches(); }

ie_status ie_generate_coefficients(const ie_grid *g, const ie_layers *lay, double freq, void *q_dev, void *stream) {
  if (!g || !lay || !q_dev || !(freq > 0) || g->nx < 1 || g->ny < 1 || g->nz < 1 || !g->z_edges_host ||
      lay->n_interfaces < 1 || !lay->interfaces_host || !lay->sigma_host)
    return IE_ERR_ARG;
  std::vector<double> ze(g->z_edges_host, g->z_edges_host + g->nz + 1);
  std::vector<double> d(lay->interfaces_host, lay->interfaces_host + lay->n_interfaces);
  std::vector<int> cl(g->nz);
  for (int z = 0; z < g->nz; ++z) {
    if (!(ze[z + 1] > ze[z])) return IE_ERR_ARG;
    cl[z] = layer_of_cell(d, ze[z], ze[z + 1]);
    if (cl[z] < 0 || !(lay->sigma_host[2 * cl[z]] > 0.0)) return IE_ERR_GEOMETRY;
  }
  ie::CoefGenInput gi{g->nx, g->ny, g->nz, g->hx, g->hy, ze.data(), cl.data(), lay->n_interfaces, d.data(),
                      lay->sigma_host, freq};
  const ie::CoefGenStatus gs = ie::generate_coefficients(gi, (double2 *)q_dev, (cudaStream_t)stream);
  if (gs == ie::CoefGenStatus::kUnsupported) return IE_ERR_ARG;
  return gs == ie::CoefGenStatus::kOk ? IE_OK : IE_ERR_CUDA;
}

static void prof_clear(ie_ctx *c) {
  for (auto &r : c->prof_rec) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  c->prof_rec.clear();
}

ie_status ie_profile(ie_ctx *c, int enable) {
  if (!c) return IE_ERR_ARG;
  IE_CUDA(cudaStreamSynchronize(c->stream));
  prof_clear(c);
  c->prof = enable < 0 ? 0 : (enable > 2 ? 2 : enable);
  return IE_OK;
}

ie_status ie_profile_read(ie_ctx *c, int dtype, double *total_ms, long long *n_launch) {
  if (!c || !total_ms || !n_launch) return IE_ERR_ARG;
  double tot = 0.0;
  long long n = 0;
  for (auto &r : c->prof_rec) {
    if (r.dtype != dtype) continue;
    IE_CUDA(cudaEventSynchronize(r.b));
    float ms = 0.f;
    IE_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    tot += ms;
    ++n;
  }
  *total_ms = tot;
  *n_launch = n;
  return IE_OK;
}

ie_status ie_profile_matvec(ie_ctx *c, int inst, int nrhs, int dtype, int n_iter, double *ms_out) {
  if (!c || !ms_out || inst < 0 || inst >= (int)c->inst.size() || nrhs < 1 || nrhs > std::min(4, c->max_rhs) ||
      n_iter < 1)
    return IE_ERR_ARG;
  if (dtype != IE_C64 && dtype != IE_C128) return IE_ERR_ARG;
  const int Nx = c->nx, Ny = c->ny, Nz = c->nz, CZ = nrhs * 3 * Nz;
  cudaStream_t s = c->stream;
  cudaEvent_t ev[6];
  for (auto &e : ev) IE_CUDA(cudaEventCreate(&e));
  double acc[5] = {0, 0, 0, 0, 0};
  int bad = 0;
  for (int it = 0; it < n_iter; ++it) {
    if (dtype == IE_C128) {
      const double2 *x = c->w;
      double2 *y = c->r, *t1 = (double2 *)c->t1, *sp = (double2 *)c->spec;
      cudaEventRecord(ev[0], s);
      ie::launch_fft_rows_fwd<double>(x, (const double2 *)c->d64.in_f, t1, CZ, Nz, Ny, Nx, c->px, s);
      cudaEventRecord(ev[1], s);
      ie::launch_fft_axis<double, false>(t1, sp, 1, Ny, 2 * Ny, 2LL * Nx * CZ, c->py, 1.0, s);
      cudaEventRecord(ev[2], s);
      bad |= ie::launch_contract<double>(sp, c->inst[inst].q64, Nx, Ny, Nz, nrhs, CZ, ie::kContractPanel, c->err, s);
      cudaEventRecord(ev[3], s);
      ie::launch_fft_axis<double, true>(sp, t1, 1, 2 * Ny, Ny, 2LL * Nx * CZ, c->py, 1.0, s);
      cudaEventRecord(ev[4], s);
      ie::launch_fft_rows_inv<double>(t1, x, (const double2 *)c->d64.diag, (const double2 *)c->d64.out_f, y, CZ, Nz,
                                      Ny, Nx, c->px, s);
      cudaEventRecord(ev[5], s);
    } else {
      const float2 *x = c->x32;
      float2 *y = c->y32, *t1 = (float2 *)c->t1, *sp = (float2 *)c->spec;
      cudaEventRecord(ev[0], s);
      ie::launch_fft_rows_fwd<float>(x, (const float2 *)c->d32.in_f, t1, CZ, Nz, Ny, Nx, c->px, s);
      cudaEventRecord(ev[1], s);
      ie::launch_fft_axis<float, false>(t1, sp, 1, Ny, 2 * Ny, 2LL * Nx * CZ, c->py, 1.0f, s);
      cudaEventRecord(ev[2], s);
      bad |= ie::launch_contract<float>(sp, c->inst[inst].q32, Nx, Ny, Nz, nrhs, CZ, c->cvar[nrhs], c->err, s,
                                        c->inst[inst].qexp, c->inst[inst].qh);
      cudaEventRecord(ev[3], s);
      ie::launch_fft_axis<float, true>(sp, t1, 1, 2 * Ny, Ny, 2LL * Nx * CZ, c->py, 1.0f, s);
      cudaEventRecord(ev[4], s);
      ie::launch_fft_rows_inv<float>(t1, x, (const float2 *)c->d32.diag, (const float2 *)c->d32.out_f, y, CZ, Nz, Ny,
                                     Nx, c->px, s);
      cudaEventRecord(ev[5], s);
    }
    IE_CUDA(cudaEventSynchronize(ev[5]));
    for (int k = 0; k < 5; ++k) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
      acc[k] += ms;
    }
  }
  for (auto &e : ev) cudaEventDestroy(e);
  for (int k = 0; k < 5; ++k) ms_out[k] = acc[k] / n_iter;
  const ie_status st = cuda_status(cudaGetLastError());
  if (bad) return IE_ERR_CUDA;
  if (st == IE_OK && ie::contract_take_error(c->err, s) != 0) return IE_ERR_TIMEOUT;
  return st;
}
long long ie_ctx_device_bytes(ie_ctx *c) { return c ? c->dev_bytes : 0; }

// FFT plan autotuner: time every candidate stage order (candidate_plans) of the two
// transform lengths in the c128 passes the refinement residuals and FP64 solves run (the
// forward row pass over x, the column pass over y; four launches each on the context's
// workspaces, zeroed) and keep the fastest.  The c64 passes use the same plans where no
// register-blocked kernel applies.
ie_status autotune_fft(ie_ctx *c) {
  const int Nx = c->nx, Ny = c->ny, Nz = c->nz;
  const int CZ = 3 * Nz;  // one right-hand side
  cudaEvent_t e0, e1;
  IE_CUDA(cudaEventCreate(&e0));
  IE_CUDA(cudaEventCreate(&e1));
  const double2 *x = (const double2 *)c->w;
  double2 *t1 = (double2 *)c->t1, *spec = (double2 *)c->spec;
  cudaMemsetAsync(c->w, 0, (size_t)c->nvec() * sizeof(double2), c->stream);
  cudaMemsetAsync(c->t1, 0, (size_t)Ny * 2 * Nx * CZ * sizeof(double2), c->stream);
  ie_status st = IE_OK;
  for (int axis = 0; axis < 2 && st == IE_OK; ++axis) {
    const std::vector<ie::FftPlan> cand = ie::candidate_plans(axis == 0 ? 2 * Nx : 2 * Ny);
    if (cand.size() < 2) continue;
    double best_ms = 1e300;
    ie::FftPlan best = axis == 0 ? c->px : c->py;
    for (const ie::FftPlan &p : cand) {
      auto run = [&]() {
        if (axis == 0)
          ie::launch_fft_rows_fwd<double>(x, nullptr, t1, CZ, Nz, Ny, Nx, p, c->stream);
        else
          ie::launch_fft_axis<double, false>(t1, spec, 1, Ny, 2 * Ny, 2LL * Nx * CZ, p, 1.0, c->stream);
      };
      run();
      cudaEventRecord(e0, c->stream);
      for (int k = 0; k < 4; ++k) run();
      cudaEventRecord(e1, c->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) { st = IE_ERR_CUDA; break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms / 4.0 < best_ms) { best_ms = ms / 4.0; best = p; }
    }
    if (st != IE_OK) break;
    if (axis == 0) c->px = best; else c->py = best;
    c->fft_ms[axis] = best_ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == IE_OK) st = cuda_status(cudaGetLastError());
  return st;
}

// Autotuner: time every contraction variant that applies to this grid (c64, one and two
// right-hand sides per instance) on the context's own coefficients and workspaces, and
// keep the fastest.  The spectrum workspace is zeroed first; the values do not change
// the work.
ie_status autotune_contraction(ie_ctx *c) {
  const int Nx = c->nx, Ny = c->ny, Nz = c->nz;
  cudaEvent_t e0, e1;
  IE_CUDA(cudaEventCreate(&e0));
  IE_CUDA(cudaEventCreate(&e1));
  ie_status st = IE_OK;
  for (int rpi = 1; rpi <= std::min(2, c->max_rhs) && st == IE_OK; ++rpi) {
    const int CZ = rpi * 3 * Nz;
    float2 *spec = (float2 *)c->spec;
    cudaMemsetAsync(spec, 0, (size_t)4 * Nx * Ny * CZ * sizeof(float2), c->stream);
    int best = ie::kContractPanel;
    double best_ms = 1e300;
    int n_avail = 0;
    for (int v = 0; v < ie::kContractVariants; ++v)
      if (ie::contract_variant_available(v, Nz, rpi, true)) ++n_avail;
    for (int v = 0; v < ie::kContractVariants && n_avail > 1; ++v) {
      if (!ie::contract_variant_available(v, Nz, rpi, true)) continue;
      const int *qe = c->inst[0].qexp;
      const void *qh = c->inst[0].qh;
      bool ok =
          ie::launch_contract<float>(spec, c->inst[0].q32, Nx, Ny, Nz, rpi, CZ, v, c->err, c->stream, qe, qh) == 0;
      cudaEventRecord(e0, c->stream);
      for (int k = 0; k < 3 && ok; ++k)
        ok = ie::launch_contract<float>(spec, c->inst[0].q32, Nx, Ny, Nz, rpi, CZ, v, c->err, c->stream, qe, qh) ==
             0;
      cudaEventRecord(e1, c->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) { st = IE_ERR_CUDA; break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (!ok || ie::contract_take_error(c->err, c->stream) != 0) continue;
      c->tune_ms[rpi][v] = ms / 3.0;
      if (ms / 3.0 < best_ms) { best_ms = ms / 3.0; best = v; }
    }
    if (n_avail == 1) best = ie::kContractPanel;
    if (n_avail > 1 || ie::contract_variant_available(ie::kContractPanel, Nz, rpi, true)) c->cvar[rpi] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == IE_OK) st = cuda_status(cudaGetLastError());
  return st;
}

static ie_status setup_impl(const ie_grid *g, const ie_layers *lay, const double *sigma_a, int n_freq,
                            const double *freq, const double *q_real, int max_rhs, const ie_options *opt,
                            ie_ctx *c) {
  c->nx = g->nx; c->ny = g->ny; c->nz = g->nz;
  c->hx = g->hx; c->hy = g->hy; c->x0 = g->x0; c->y0 = g->y0;
  c->ze.assign(g->z_edges_host, g->z_edges_host + g->nz + 1);
  for (int k = 0; k < g->nz; ++k)
    if (!(c->ze[k + 1] > c->ze[k])) return IE_ERR_ARG;
  c->d.assign(lay->interfaces_host, lay->interfaces_host + lay->n_interfaces);
  for (int k = 0; k + 1 < lay->n_interfaces; ++k)
    if (!(c->d[k + 1] > c->d[k])) return IE_ERR_ARG;
  c->sig.resize(lay->n_interfaces + 1);
  for (int k = 0; k <= lay->n_interfaces; ++k) c->sig[k] = cd(lay->sigma_host[2 * k], lay->sigma_host[2 * k + 1]);
  c->lay.resize(g->nz);
  for (int z = 0; z < g->nz; ++z) {
    const int m = layer_of_cell(c->d, c->ze[z], c->ze[z + 1]);
    if (m < 0) return IE_ERR_GEOMETRY;
    if (!(c->sig[m].real() > 0.0)) return IE_ERR_GEOMETRY;
    c->lay[z] = m;
  }
  const long long N = c->ncell();
  c->sigma_a.resize(N);
  for (long long i = 0; i < N; ++i) c->sigma_a[i] = cd(sigma_a[2 * i], sigma_a[2 * i + 1]);
  c->max_rhs = max_rhs;
  if (opt) {
    if (opt->restart > 0) c->restart = opt->restart;
    if (opt->max_iter > 0) c->max_iter = opt->max_iter;
    if (opt->inner_tol > 0) c->inner_tol = opt->inner_tol;
    if (opt->max_outer > 0) c->max_outer = opt->max_outer;
    if (opt->autotune < 0) c->autotune = false;
  }
  if (c->restart < 2) return IE_ERR_ARG;
  // every product of up to four right-hand sides must fit the panel contraction (c128)
  if (!ie::contract_fits(c->nz, std::min(4, max_rhs), false)) return IE_ERR_ARG;
  try {
    c->px = ie::make_plan(2 * c->nx);
    c->py = ie::make_plan(2 * c->ny);
  } catch (...) {
    return IE_ERR_ARG;
  }
  IE_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
  IE_TRY(build_diagonals(c));
  c->inst.resize(n_freq);
  const long long nq = (long long)c->nx * c->ny * 6LL * c->nz * c->nz;
  for (int f = 0; f < n_freq; ++f) {
    if (!(freq[f] > 0)) return IE_ERR_ARG;
    c->inst[f].freq = freq[f];
    IE_TRY(build_spectral(c, c->inst[f], q_real ? q_real + 2 * nq * f : nullptr));
  }
  // workspaces (sized for c128 and max_rhs)
  const long long CZ = (long long)max_rhs * 3 * c->nz;
  IE_TRY(dalloc(c, &c->t1, (size_t)c->ny * 2 * c->nx * CZ * sizeof(double2)));
  IE_TRY(dalloc(c, &c->spec, (size_t)4 * c->ny * c->nx * CZ * sizeof(double2)));
  const long long nv = c->nvec() * max_rhs;
  IE_TRY(dalloc(c, &c->x32, nv * sizeof(float2)));
  IE_TRY(dalloc(c, &c->y32, nv * sizeof(float2)));
  IE_TRY(dalloc(c, &c->V, (size_t)(c->restart + 1) * nv * sizeof(double2)));
  IE_TRY(dalloc(c, &c->w, nv * sizeof(double2)));
  IE_TRY(dalloc(c, &c->r, nv * sizeof(double2)));
  IE_TRY(dalloc(c, &c->dx, nv * sizeof(double2)));  // correction of IE_MIXED_FP64K inner solves
  // the split copy of the FP64 Krylov basis read by the double-float Gram-Schmidt passes
  IE_TRY(dalloc(c, &c->Vs, (size_t)(c->restart + 1) * nv * sizeof(float4)));
  if (c->restart > 63) return IE_ERR_ARG;
  const long long nbp = std::max<long long>(ie::mdot_nb(c->nvec()), ie::gs_partial_blocks(c->nvec()));
  IE_TRY(dalloc(c, &c->part, (size_t)max_rhs * (c->restart + 1) * nbp * sizeof(double2)));
  IE_TRY(dalloc(c, &c->hdev, (size_t)3 * max_rhs * (c->restart + 1) * sizeof(double2)));
  IE_TRY(dalloc(c, &c->nrmpart, (size_t)2 * max_rhs * std::max<long long>(1024, nbp) * sizeof(double)));
  IE_TRY(dalloc(c, &c->gsflag, (size_t)48 * sizeof(int)));  // flags, reduction tickets, a counter
  IE_CUDA(cudaMemset(c->gsflag, 0, (size_t)48 * sizeof(int)));
  IE_TRY(dalloc(c, &c->nrm, (size_t)2 * max_rhs * sizeof(double)));
  {
    const int m = c->restart, ldh = m + 1;
    IE_TRY(dalloc(c, &c->gst.Rm, (size_t)max_rhs * m * ldh * sizeof(double2)));
    IE_TRY(dalloc(c, &c->gst.sn, (size_t)max_rhs * m * sizeof(double2)));
    IE_TRY(dalloc(c, &c->gst.g, (size_t)max_rhs * ldh * sizeof(double2)));
    IE_TRY(dalloc(c, &c->gst.cs, (size_t)max_rhs * m * sizeof(double)));
    IE_TRY(dalloc(c, &c->gst.thr, (size_t)max_rhs * sizeof(double)));
    IE_TRY(dalloc(c, &c->gst.active, (size_t)max_rhs * sizeof(int)));
    IE_TRY(dalloc(c, &c->gst.kr, (size_t)max_rhs * sizeof(int)));
    IE_TRY(dalloc(c, &c->gst.brk, (size_t)max_rhs * sizeof(int)));
    IE_TRY(dalloc(c, &c->gst.n_active, sizeof(int)));
    IE_CUDA(cudaHostAlloc((void **)&c->pin_active, (2 + kPinSlots) * sizeof(int), cudaHostAllocDefault));
    for (int k = 0; k < 2 + kPinSlots; ++k) c->pin_active[k] = 0;
    IE_TRY(dalloc(c, &c->err, sizeof(int)));
    IE_CUDA(cudaMemset(c->err, 0, sizeof(int)));
    for (int k = 0; k < kPinSlots; ++k) IE_CUDA(cudaEventCreateWithFlags(&c->pin_ev[k], cudaEventDisableTiming));
    IE_CUDA(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    IE_CUDA(cudaEventCreateWithFlags(&c->gs_ev, cudaEventDisableTiming));
    IE_CUDA(cudaEventCreateWithFlags(&c->giv_ev, cudaEventDisableTiming));
  }
  IE_CUDA(cudaStreamSynchronize(c->stream));
  if (c->autotune) {
    IE_TRY(autotune_fft(c));
    IE_TRY(autotune_contraction(c));
  }
  return IE_OK;
}

ie_status ie_setup(const ie_grid *g, const ie_layers *lay, const double *sigma_a, int n_freq, const double *freq,
                   const double *q_real, int max_rhs, const ie_options *opt, ie_ctx **out) {
  if (!out) return IE_ERR_ARG;
  *out = nullptr;
  if (!g || !lay || !sigma_a || !freq || n_freq < 1 || max_rhs < 1 || max_rhs > 16) return IE_ERR_ARG;
  if (g->nx < 1 || g->ny < 1 || g->nz < 1 || !(g->hx > 0) || !(g->hy > 0) || !g->z_edges_host) return IE_ERR_ARG;
  if (lay->n_interfaces < 1 || !lay->interfaces_host || !lay->sigma_host) return IE_ERR_ARG;
  ie_ctx *c = new (std::nothrow) ie_ctx();
  if (!c) return IE_ERR_OOM;
  const ie_status st = setup_impl(g, lay, sigma_a, n_freq, freq, q_real, max_rhs, opt, c);
  if (st != IE_OK) {
    ie_destroy(c);
    return st;
  }
  *out = c;
  return IE_OK;
}

ie_status ie_matvec(ie_ctx *c, int inst, const void *x, void *y, int nrhs, int dtype, int transpose, void *stream) {
  if (!c || !x || !y || x == y || inst < 0 || inst >= (int)c->inst.size() || nrhs < 1 ||
      nrhs > std::min(4, c->max_rhs))
    return IE_ERR_ARG;
  cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
  transpose = transpose ? 1 : 0;
  Group g;
  g.inst = {inst};
  g.rpi = nrhs;
  if (dtype == IE_C128) return apply<double>(c, g, (const double2 *)x, (double2 *)y, transpose, s);
  if (dtype == IE_C128_DF) return apply<double>(c, g, (const double2 *)x, (double2 *)y, transpose, s, true);
  if (dtype == IE_C64) return apply<float>(c, g, (const float2 *)x, (float2 *)y, transpose, s);
  return IE_ERR_ARG;
}

ie_status ie_sync(ie_ctx *c, void *stream) {
  if (!c) return IE_ERR_ARG;
  cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
  IE_CUDA(cudaStreamSynchronize(s));
  const int e = ie::contract_take_error(c->err, s);
  if (e < 0) return IE_ERR_CUDA;
  return e ? IE_ERR_TIMEOUT : IE_OK;
}

void ie_debug_set_wait_limit(long long polls) { ie::set_wait_limit(polls); }

ie_status ie_solve(ie_ctx *c, int inst, const void *b, void *u, int nrhs, double tol, int precision, int use_x0,
                   ie_solve_info *info) {
  Group g;
  g.inst = {inst};
  g.rpi = nrhs;
  return solve_impl(c, g, (const double2 *)b, (double2 *)u, tol, precision, use_x0, 0, info);
}

ie_status ie_adjoint_solve(ie_ctx *c, int inst, const void *b, void *w, int nrhs, double tol, int precision,
                           int use_x0, ie_solve_info *info) {
  Group g;
  g.inst = {inst};
  g.rpi = nrhs;
  return solve_impl(c, g, (const double2 *)b, (double2 *)w, tol, precision, use_x0, 1, info);
}

ie_status ie_solve_batch(ie_ctx *c, int n_inst, const int *inst_host, const void *b, void *u, int nrhs, double tol,
                         int precision, int use_x0, int transpose, ie_solve_info *info) {
  if (!c || n_inst < 1 || !inst_host) return IE_ERR_ARG;
  Group g;
  g.inst.assign(inst_host, inst_host + n_inst);
  g.rpi = nrhs;
  return solve_impl(c, g, (const double2 *)b, (double2 *)u, tol, precision, use_x0, transpose ? 1 : 0, info);
}

ie_status ie_contract_tuning(ie_ctx *c, int *variant_host, double *ms_host) {
  if (!c || !variant_host) return IE_ERR_ARG;
  for (int r = 1; r <= 4; ++r) {
    variant_host[r - 1] = c->cvar[r];
    if (ms_host)
      for (int v = 0; v < ie::kContractVariants; ++v) ms_host[(r - 1) * ie::kContractVariants + v] = c->tune_ms[r][v];
  }
  return IE_OK;
}

ie_status ie_fft_plan(ie_ctx *c, int axis, int *radix_host, int *n_stages, double *ms) {
  if (!c || axis < 0 || axis > 1 || !radix_host || !n_stages) return IE_ERR_ARG;
  const ie::FftPlan &p = axis == 0 ? c->px : c->py;
  *n_stages = p.n_stages;
  for (int k = 0; k < p.n_stages; ++k) radix_host[k] = p.radix[k];
  if (ms) *ms = c->fft_ms[axis];
  return IE_OK;
}

ie_status ie_set_fft_plan(ie_ctx *c, int axis, const int *radix_host, int n_stages) {
  if (!c || axis < 0 || axis > 1 || !radix_host || n_stages < 1 || n_stages > ie::kMaxStages) return IE_ERR_ARG;
  ie::FftPlan p{};
  p.L = axis == 0 ? 2 * c->nx : 2 * c->ny;
  long long prod = 1;
  for (int k = 0; k < n_stages; ++k) {
    const int r = radix_host[k];
    if (r != 2 && r != 3 && r != 4 && r != 5 && r != 7 && r != 8 && r != 11 && r != 13) return IE_ERR_ARG;
    prod *= r;
    p.radix[k] = r;
  }
  if (prod != p.L) return IE_ERR_ARG;
  p.n_stages = n_stages;
  if (axis == 0) c->px = p; else c->py = p;
  c->fft_ms[axis] = 0.0;
  return IE_OK;
}

ie_status ie_set_contract_variant(ie_ctx *c, int nrhs, int variant) {
  if (!c || nrhs < 1 || nrhs > 4 || variant < -1 || variant >= ie::kContractVariants) return IE_ERR_ARG;
  if (variant >= 0 && !ie::contract_variant_available(variant, c->nz, nrhs, true)) return IE_ERR_ARG;
  c->cvar[nrhs] = variant;
  return IE_OK;
}

ie_status ie_set_sigma(ie_ctx *c, const double *sigma_a_host) {
  if (!c || !sigma_a_host) return IE_ERR_ARG;
  const long long N = c->ncell();
  std::vector<cd> sa(N);
  for (long long i = 0; i < N; ++i) sa[i] = cd(sigma_a_host[2 * i], sigma_a_host[2 * i + 1]);
  std::swap(sa, c->sigma_a);
  if (check_receiver_geometry(c) != IE_OK) {
    std::swap(sa, c->sigma_a);
    return IE_ERR_GEOMETRY;
  }
  IE_CUDA(cudaStreamSynchronize(c->stream));  // no product may be reading the diagonals
  return build_diagonals(c);
}

namespace {
// layer of the receiver depth and the layer stack as (re, im) pairs for the generator
int receiver_layer_of(const ie_ctx *c, double z_rec) {
  int r_layer = 0;
  for (size_t k = 0; k < c->d.size(); ++k)
    if (z_rec >= c->d[k]) r_layer = (int)k + 1;
  return r_layer;
}
std::vector<double> sigma_pairs(const ie_ctx *c) {
  std::vector<double> sg(2 * c->sig.size());
  for (size_t k = 0; k < c->sig.size(); ++k) { sg[2 * k] = c->sig[k].real(); sg[2 * k + 1] = c->sig[k].imag(); }
  return sg;
}
ie_status ensure_rtab(ie_ctx *c, Instance &in, size_t elems) {
  if (in.rtab && in.rtab_cap >= elems) return IE_OK;
  IE_TRY(dalloc(c, &in.rtab, elems * sizeof(double2)));
  in.rtab_cap = elems;
  return IE_OK;
}
}  // namespace

ie_status ie_set_receivers_xy(ie_ctx *c, int n_rec, const double *x, const double *y, double z_rec) {
  if (!c || n_rec < 1 || n_rec > (1 << 16) || !x || !y) return IE_ERR_ARG;
  if (z_rec > c->ze[0] || z_rec < c->d[0]) return IE_ERR_ARG;
  const int nx = c->nx, ny = c->ny, nz = c->nz;
  std::vector<int> ix(n_rec), iy(n_rec), grp(n_rec);
  std::vector<double> gfx, gfy;
  for (int r = 0; r < n_rec; ++r) {
    const double ux = (x[r] - c->x0) / c->hx - 0.5, uy = (y[r] - c->y0) / c->hy - 0.5;
    if (!(ux >= -0.5 && ux <= nx - 0.5 && uy >= -0.5 && uy <= ny - 0.5)) return IE_ERR_ARG;
    // the cell centre at or before the site, and the site's position beyond it in cells
    const int jr = (int)std::floor(ux), ir = (int)std::floor(uy);
    const double fx = ux - jr, fy = uy - ir;
    int gsel = -1;
    for (size_t g = 0; g < gfx.size(); ++g)
      if (std::fabs(gfx[g] - fx) < 1e-9 && std::fabs(gfy[g] - fy) < 1e-9) { gsel = (int)g; break; }
    if (gsel < 0) {
      gsel = (int)gfx.size();
      gfx.push_back(fx);
      gfy.push_back(fy);
    }
    ix[r] = jr;
    iy[r] = ir;
    grp[r] = gsel;
  }
  const int n_grp = (int)gfx.size();
  const int old_n = c->n_rec;
  const double old_z = c->z_rec;
  c->n_rec = n_rec;
  c->z_rec = z_rec;
  if (check_receiver_geometry(c) != IE_OK) {
    c->n_rec = old_n;
    c->z_rec = old_z;
    return IE_ERR_GEOMETRY;
  }
  IE_CUDA(cudaStreamSynchronize(c->stream));
  if (old_n < n_rec || !c->rec_grp) {
    IE_TRY(dalloc(c, &c->rec_ix, (size_t)n_rec * sizeof(int)));
    IE_TRY(dalloc(c, &c->rec_iy, (size_t)n_rec * sizeof(int)));
    IE_TRY(dalloc(c, &c->rec_grp, (size_t)n_rec * sizeof(int)));
    IE_TRY(dalloc(c, &c->phi_r, (size_t)n_rec * sizeof(double)));
  }
  IE_CUDA(cudaMemcpy(c->rec_ix, ix.data(), (size_t)n_rec * sizeof(int), cudaMemcpyHostToDevice));
  IE_CUDA(cudaMemcpy(c->rec_iy, iy.data(), (size_t)n_rec * sizeof(int), cudaMemcpyHostToDevice));
  IE_CUDA(cudaMemcpy(c->rec_grp, grp.data(), (size_t)n_rec * sizeof(int), cudaMemcpyHostToDevice));
  c->rec_sites = true;
  const int r_layer = receiver_layer_of(c, z_rec);
  std::vector<double> sg = sigma_pairs(c);
  const int n_off = 4 * nx * ny;
  const size_t gstride = (size_t)n_off * nz * 10;
  std::vector<double> offs(2 * (size_t)n_off);
  for (auto &in : c->inst) {
    IE_TRY(ensure_rtab(c, in, gstride * n_grp));
    ie::CoefGenInput gi{nx, ny, nz, c->hx, c->hy, c->ze.data(), c->lay.data(), (int)c->d.size(), c->d.data(),
                        sg.data(), in.freq};
    for (int g = 0; g < n_grp; ++g) {
      // offsets (receiver minus cell centre) of the group: row di + Ny, column dj + Nx
      for (int di = -ny; di < ny; ++di)
        for (int dj = -nx; dj < nx; ++dj) {
          const size_t o = (size_t)(di + ny) * 2 * nx + (dj + nx);
          offs[2 * o] = (di + gfy[g]) * c->hy;
          offs[2 * o + 1] = (dj + gfx[g]) * c->hx;
        }
      const ie::CoefGenStatus gs =
          ie::generate_receiver_tables(gi, z_rec, r_layer, in.rtab + g * gstride, c->stream, offs.data(), n_off);
      if (gs != ie::CoefGenStatus::kOk) return gs == ie::CoefGenStatus::kUnsupported ? IE_ERR_ARG : IE_ERR_CUDA;
    }
    cd E, H;
    mt_point(c, 2.0 * M_PI * in.freq, z_rec, &E, &H);
    in.en = make_double2(E.real(), E.imag());
    in.hn = make_double2(H.real(), H.imag());
  }
  return IE_OK;
}

ie_status ie_mt_apparent(ie_ctx *c, int inst, const void *z_dev, int n_rec, void *rho_dev, void *phase_dev) {
  if (!c || !z_dev || !rho_dev || !phase_dev || inst < 0 || inst >= (int)c->inst.size() || n_rec < 1)
    return IE_ERR_ARG;
  ie::launch_mt_apparent((const double2 *)z_dev, 4 * n_rec, 2.0 * M_PI * c->inst[inst].freq, (double *)rho_dev,
                         (double *)phase_dev, c->stream);
  IE_CUDA(cudaGetLastError());
  IE_CUDA(cudaStreamSynchronize(c->stream));
  return IE_OK;
}

ie_status ie_set_receivers(ie_ctx *c, int n_rec, const int *ix, const int *iy, double z_rec) {
  if (!c || n_rec < 1 || n_rec > (1 << 16) || !ix || !iy) return IE_ERR_ARG;
  if (z_rec > c->ze[0] || z_rec < c->d[0]) return IE_ERR_ARG;
  for (int r = 0; r < n_rec; ++r)
    if (ix[r] < 0 || ix[r] >= c->nx || iy[r] < 0 || iy[r] >= c->ny) return IE_ERR_ARG;
  const int old_n = c->n_rec;
  const double old_z = c->z_rec;
  c->n_rec = n_rec;
  c->z_rec = z_rec;
  if (check_receiver_geometry(c) != IE_OK) {
    c->n_rec = old_n;
    c->z_rec = old_z;
    return IE_ERR_GEOMETRY;
  }
  IE_CUDA(cudaStreamSynchronize(c->stream));
  if (old_n < n_rec) {  // grow the per-receiver arrays
    IE_TRY(dalloc(c, &c->rec_ix, (size_t)n_rec * sizeof(int)));
    IE_TRY(dalloc(c, &c->rec_iy, (size_t)n_rec * sizeof(int)));
    IE_TRY(dalloc(c, &c->phi_r, (size_t)n_rec * sizeof(double)));
  }
  IE_CUDA(cudaMemcpy(c->rec_ix, ix, (size_t)n_rec * sizeof(int), cudaMemcpyHostToDevice));
  IE_CUDA(cudaMemcpy(c->rec_iy, iy, (size_t)n_rec * sizeof(int), cudaMemcpyHostToDevice));
  c->rec_sites = false;
  const int r_layer = receiver_layer_of(c, z_rec);
  std::vector<double> sg = sigma_pairs(c);
  const size_t tab_elems = (size_t)c->nx * c->ny * c->nz * 10;
  for (auto &in : c->inst) {
    IE_TRY(ensure_rtab(c, in, tab_elems));
    ie::CoefGenInput gi{c->nx, c->ny, c->nz, c->hx, c->hy, c->ze.data(), c->lay.data(), (int)c->d.size(),
                        c->d.data(), sg.data(), in.freq};
    const ie::CoefGenStatus gs = ie::generate_receiver_tables(gi, z_rec, r_layer, in.rtab, c->stream);
    if (gs != ie::CoefGenStatus::kOk) return gs == ie::CoefGenStatus::kUnsupported ? IE_ERR_ARG : IE_ERR_CUDA;
    cd E, H;
    mt_point(c, 2.0 * M_PI * in.freq, z_rec, &E, &H);
    in.en = make_double2(E.real(), E.imag());
    in.hn = make_double2(H.real(), H.imag());
  }
  return IE_OK;
}

ie_status ie_receiver_fields(ie_ctx *c, int inst, const void *u_dev, int nrhs, const int *pol_host, void *f_dev) {
  if (!c || !u_dev || !f_dev || !pol_host || inst < 0 || inst >= (int)c->inst.size() || nrhs < 1 || nrhs > 4)
    return IE_ERR_ARG;
  if (c->n_rec == 0 || !c->inst[inst].rtab) return IE_ERR_ARG;
  int pol[4] = {0, 0, 0, 0};
  for (int p = 0; p < nrhs; ++p) {
    if (pol_host[p] != 0 && pol_host[p] != 1) return IE_ERR_ARG;
    pol[p] = pol_host[p];
  }
  const Instance &in = c->inst[inst];
  ie::launch_receiver_fields(in.rtab, c->rec_ix, c->rec_iy, c->rec_sites ? c->rec_grp : nullptr, c->n_rec,
                             (const double2 *)u_dev, (const double2 *)c->jfac, nrhs, c->nx, c->ny, c->nz, pol[0],
                             pol[1], pol[2], pol[3], in.en, in.hn, (double2 *)f_dev, c->stream);
  IE_CUDA(cudaGetLastError());
  IE_CUDA(cudaStreamSynchronize(c->stream));
  return IE_OK;
}

ie_status ie_mt_misfit(ie_ctx *c, const void *f_dev, const void *zobs_dev, void *z_dev, double *phi_host,
                       void *c_dev) {
  if (!c || !f_dev || !zobs_dev || !z_dev || !phi_host || !c_dev || c->n_rec == 0) return IE_ERR_ARG;
  ie::launch_mt_misfit((const double2 *)f_dev, (const double2 *)zobs_dev, c->n_rec, (double2 *)z_dev, c->phi_r,
                       (double2 *)c_dev, c->stream);
  IE_CUDA(cudaGetLastError());
  std::vector<double> ph(c->n_rec);
  IE_CUDA(cudaMemcpyAsync(ph.data(), c->phi_r, ph.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  IE_CUDA(cudaStreamSynchronize(c->stream));
  double acc = 0.0;
  for (double v : ph) acc += v;
  *phi_host = acc;
  return IE_OK;
}

ie_status ie_receiver_adjoint(ie_ctx *c, int inst, const void *c_dev, int nrhs, void *rhs_dev) {
  if (!c || !c_dev || !rhs_dev || inst < 0 || inst >= (int)c->inst.size() || nrhs < 1 || nrhs > 4)
    return IE_ERR_ARG;
  if (c->n_rec == 0 || !c->inst[inst].rtab) return IE_ERR_ARG;
  ie::launch_receiver_adjoint(c->inst[inst].rtab, c->rec_ix, c->rec_iy, c->rec_sites ? c->rec_grp : nullptr,
                              c->n_rec, (const double2 *)c_dev, (const double2 *)c->jfac, nrhs, c->nx, c->ny, c->nz,
                              (double2 *)rhs_dev, c->stream);
  IE_CUDA(cudaGetLastError());
  IE_CUDA(cudaStreamSynchronize(c->stream));
  return IE_OK;
}

ie_status ie_gradient_accumulate(ie_ctx *c, const void *u_dev, const void *w_dev, int nrhs, void *grad_dev) {
  if (!c || !u_dev || !w_dev || !grad_dev || nrhs < 1 || nrhs > 4) return IE_ERR_ARG;
  ie::launch_gradient_accumulate((const double2 *)u_dev, (const double2 *)w_dev, (const double2 *)c->gdiv, nrhs,
                                 c->ncell(), (double *)grad_dev, c->stream);
  IE_CUDA(cudaGetLastError());
  IE_CUDA(cudaStreamSynchronize(c->stream));
  return IE_OK;
}

ie_status ie_fields(ie_ctx *c, const void *u_dev, void *e_dev, int nrhs, void *stream) {
  if (!c || !u_dev || !e_dev || nrhs < 1 || nrhs > c->max_rhs) return IE_ERR_ARG;
  cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
  ie::launch_cell_scale((const double2 *)u_dev, (const double2 *)c->efac, 3 * nrhs, c->ncell(), (double2 *)e_dev, s);
  return cuda_status(cudaGetLastError());
}

ie_status ie_rhs_mt(ie_ctx *c, int inst, int pol, void *u0) {
  if (!c || !u0 || inst < 0 || inst >= (int)c->inst.size() || (pol != 0 && pol != 1)) return IE_ERR_ARG;
  const double omega = 2.0 * M_PI * c->inst[inst].freq;
  const std::vector<cd> avg = mt_cell_average(c, omega);
  const long long plane = (long long)c->nx * c->ny;
  std::vector<double2> h((size_t)c->nvec(), make_double2(0.0, 0.0));
  for (int z = 0; z < c->nz; ++z) {
    const cd v = std::sqrt(c->sig[c->lay[z]].real()) * avg[z];
    for (long long q = 0; q < plane; ++q) h[((size_t)pol * c->nz + z) * plane + q] = make_double2(v.real(), v.imag());
  }
  IE_CUDA(cudaMemcpyAsync(u0, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
  IE_CUDA(cudaStreamSynchronize(c->stream));
  return IE_OK;
}

}  // extern "C"
