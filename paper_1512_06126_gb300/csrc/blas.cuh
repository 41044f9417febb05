#pragma once
#include "ie_common.cuh"

namespace ie {

// number of partial blocks used by gmres_norm for length n
int mdot_nb(long long n);
// Vectors are C<T>: c128 (T = double) or c64 (T = float); h, norms and partial sums
// are FP64 in both.
// w[r] += sign * sum_i h[r * ldh + i] V_i[r]
template <typename T>
void gmres_maxpy(const C<T> *V, const double2 *h, C<T> *w, int k1, int R, long long n, int ldh, double sign,
                 cudaStream_t s);
// out[r] = ||w[r]||_2
template <typename T>
void gmres_norm(const C<T> *w, double *part, double *out, int R, long long n, cudaStream_t s);
// Classical Gram-Schmidt against V_0..V_{k1-1} (k1 <= 64) with selective
// reorthogonalisation, ending with the next basis vector: h1 = V^H w; where
// ||w - V h1|| >= ||w|| / 16 (from ||w||^2 - |h1|^2) vnext = (w - V h1) / ||w - V h1||
// directly; elsewhere a second projection h2 = V^H w', w'' = w' - V h2 and
// vnext = w'' / ||w''|| (h2 = 0 where it did not run).  nrm = the norm used.  w is
// overwritten only where the second projection ran.
// R <= 16.  part: R * k1 * gs_partial_blocks(n) complex; npart: R * gs_partial_blocks(n)
// + R * 1024 doubles; nrm: 2 R doubles; flag: 48 ints, zero before the first call (flags
// [0, R): 1 where the second projection ran; [16, 16 + R): reduction tickets, left zero;
// [32]: incremented by every second projection).
// df (FP64 vectors only, with Vs and vs_next): the dot and subtract passes of the first
// projection in double-float arithmetic on the FP32 pipe (about 2^-46 relative to the
// sums of magnitudes; the second projection, the norms and all cross-thread sums stay
// FP64).  They read the basis from its split copy Vs (same layout as V, one float4 per
// complex entry: gmres_split of it, so the same numbers the FP64 basis would give when
// split on the fly) and write the split copy of vnext to vs_next.
// Returns -1 (nothing launched) for arguments out of range or a failed launch.
template <typename T>
int gmres_orthogonalize(const C<T> *V, C<T> *w, C<T> *vnext, double2 *h1, double2 *h2, double2 *part, double *npart,
                        double *nrm, int *flag, int k1, int R, long long n, int ldh, cudaStream_t s, bool df = false,
                        const float4 *Vs = nullptr, float4 *vs_next = nullptr);
// vs[e] = (re hi, re lo, im hi, im lo) of v[e] (hi: the leading 24 significant bits, lo
// the next 23), the split copy of a basis vector for the double-float passes
void gmres_split(const double2 *v, float4 *vs, long long n, cudaStream_t s);
// x[r] += sum_{i<k1} h[r * ldh + i] V_i[r] for FP64 vectors in double-float arithmetic,
// V read from its split copy Vs (k1 <= 64; gmres_maxpy with sign +1, on the FP32 pipe)
void gmres_maxpy_df(const float4 *Vs, const double2 *h, double2 *x, int k1, int R, long long n, int ldh,
                    cudaStream_t s);
int gs_partial_blocks(long long n);

// GMRES least-squares state on the device, per right-hand side r (m < 64):
// Rm [R][m][ldh] (rotated Hessenberg columns), cs [R][m], sn [R][m], g [R][ldh],
// active / kr / brk [R] (still iterating, columns so far, breakdown), thr [R] (stop
// when |g_{k+1}| <= thr), n_active [1] (right-hand sides still iterating).
struct GivensState {
  double2 *Rm, *sn, *g;
  double *cs, *thr;
  int *active, *kr, *brk, *n_active;
};
// start of a cycle from the residual norms nrm[R]
void givens_init(const GivensState &st, const double *nrm, int R, int ldh, cudaStream_t s);
// Hessenberg column k (h1 + h2 above the diagonal, nrm[r] below) for every active r;
// fp32: the recurrence in FP32 arithmetic (the state stays FP64)
void givens_step(const GivensState &st, const double2 *h1, const double2 *h2, const double *nrm, int k, int R, int m,
                 int ldh, bool fp32, cudaStream_t s);
// z[r * ldh + i], i <= kr[r]: coefficients of the residual of the cycle's least-squares
// solution in the basis V_0..V_kr (zero beyond kr): b - A x = sum_i z_i V_i
void givens_residual(const GivensState &st, double2 *z, int R, int m, int ldh, cudaStream_t s);
// yd[r * ldh + i] = the least-squares solution over the kr[r] columns (zero beyond)
void givens_solve(const GivensState &st, double2 *yd, int R, int m, int ldh, cudaStream_t s);
// dst[r] = src[r] / nrm[r]
template <typename T>
void gmres_scale(const C<T> *src, C<T> *dst, const double *nrm, int R, long long n, cudaStream_t s);
// out = a - b
template <typename T>
void vec_sub(const C<T> *a, const C<T> *b, C<T> *out, long long n, cudaStream_t s);
// y += x (y c128)
template <typename T>
void vec_add(const C<T> *x, double2 *y, long long n, cudaStream_t s);
// y = x rounded to c64
void vec_round(const double2 *x, float2 *y, long long n, cudaStream_t s);

}  // namespace ie
