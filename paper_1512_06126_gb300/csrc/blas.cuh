#pragma once
#include "ie_common.cuh"

namespace ie {

// number of partial blocks used by gmres_mdot / gmres_norm for length n
int mdot_nb(long long n);
// h_out[r * ldh + i] (+)= <V_i[r], w[r]> for i < k1 (conjugate-linear in V)
void gmres_mdot(const double2 *V, const double2 *w, double2 *part, double2 *h_out, int k1, int R, long long n, int ldh,
                int accumulate, cudaStream_t s);
// w[r] += sign * sum_i h[r * ldh + i] V_i[r]
void gmres_maxpy(const double2 *V, const double2 *h, double2 *w, int k1, int R, long long n, int ldh, double sign,
                 cudaStream_t s);
// out[r] = ||w[r]||_2
void gmres_norm(const double2 *w, double *part, double *out, int R, long long n, cudaStream_t s);
// Classical Gram-Schmidt applied twice against V_0..V_{k1-1} in three fused passes:
// h1 = V^H w; w -= V h1 and h2 = V^H w; w -= V h2 and nrm = ||w||.  k1 <= 64.
// part: R * k1 * cgs2_partial_blocks(n) complex; npart: R * cgs2_partial_blocks(n).
int gmres_cgs2(const double2 *V, double2 *w, double2 *h1, double2 *h2, double2 *part, double *npart, double *nrm,
               int k1, int R, long long n, int ldh, cudaStream_t s);
int cgs2_partial_blocks(long long n);
// dst[r] = src[r] / nrm[r]
void gmres_scale(const double2 *src, double2 *dst, const double *nrm, int R, long long n, cudaStream_t s);
void vec_sub(const double2 *a, const double2 *b, double2 *out, long long n, cudaStream_t s);
void vec_add(const double2 *x, double2 *y, long long n, cudaStream_t s);

}  // namespace ie
